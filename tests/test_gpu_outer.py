"""Barycenter (Alg. 2) and k-means (Sec. 5) on the GPU vs the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_08331_gb300 import api, inputs
from gpu_util import dev, hists_to_gpu, masses

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    api.load(build_if_missing=True)
    c = api.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("d,gamma,lam,steps,T", [(16, 1e-2, 2.0, 5, 200), (32, 5e-3, 5.0, 4, 300)])
def test_barycenter_matches_oracle(ctx, d, gamma, lam, steps, T):
    """Same inner iteration counts on both sides (tol 0, max_iter T, warm starts),
    so the outer iterates must agree to the inner solves' rounding."""
    b, t, o = inputs.random_diagrams(4, nmin=8, nmax=25, seed=d, log_uniform=False)
    h, m = oracle.rasterize(b, t, o, d)
    z_ref, e_ref = oracle.barycenter(d, gamma, h, lam, steps, T, 0.0)
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=T, tol=0.0)
    z, e = api.pd_barycenter(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, lam, steps)
    torch.cuda.synchronize()
    z, e = z.cpu().numpy(), e.cpu().numpy()
    assert np.allclose(e, e_ref, rtol=1e-6, atol=0)
    assert np.allclose(z, z_ref, rtol=1e-5, atol=1e-9 * z_ref.max())
    assert abs(z.sum() - z_ref.sum()) <= 1e-6 * z_ref.sum()


@pytest.mark.parametrize("d,gamma,lam,steps,T", [(16, 1e-2, 2.0, 5, 200), (32, 5e-3, 5.0, 4, 300)])
def test_sharpened_barycenter_matches_oracle(ctx, d, gamma, lam, steps, T):
    """NEXT-2 entropic sharpening after every Alg. 2 step (target: the largest
    input entropy): same outer iterates as the oracle, and z's entropy stays at
    or below the target."""
    b, t, o, _ = inputs.mode_diagrams(4, 1, 15, 30, sigma=0.04, seed=d)
    h, m = oracle.rasterize(b, t, o, d)
    z_ref, e_ref = oracle.barycenter(d, gamma, h, lam, steps, T, 0.0, sharpen=True)
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=T, tol=0.0, bary_sharpen=1)
    z, e = api.pd_barycenter(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, lam, steps)
    torch.cuda.synchronize()
    z, e = z.cpu().numpy(), e.cpu().numpy()
    assert np.allclose(e, e_ref, rtol=1e-6, atol=0)
    assert np.allclose(z, z_ref, rtol=1e-5, atol=1e-9 * z_ref.max())
    w = z[z > 0] / z.sum()
    H = -(w * np.log(w)).sum()
    H0 = max(-(x[x > 0] / x.sum() * np.log(x[x > 0] / x.sum())).sum() for x in h.astype(np.float64))
    assert H <= H0 + 1e-9


def test_barycenter_from_given_start_and_zero_steps(ctx):
    d, gamma = 16, 1e-2
    b, t, o = inputs.random_diagrams(3, nmin=10, nmax=10, seed=1)
    h, _ = oracle.rasterize(b, t, o, d)
    z0 = np.zeros((d, d))
    z0[np.triu_indices(d)] = np.linspace(0.1, 1.0, d * (d + 1) // 2)
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=150, tol=0.0)
    z, _ = api.pd_barycenter(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, 1.0, 0, z_init=dev(z0))
    assert np.array_equal(z.cpu().numpy(), z0)
    z, e = api.pd_barycenter(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, 1.0, 2, z_init=dev(z0))
    z_ref, e_ref = oracle.barycenter(d, gamma, h, 1.0, 2, 150, 0.0, z_init=z0)
    assert np.allclose(z.cpu().numpy(), z_ref, rtol=1e-5, atol=1e-12)


def test_kmeans_matches_oracle(ctx):
    d, gamma = 16, 5e-3
    b, t, o, lab = inputs.mode_diagrams(12, 3, 40, 60, sigma=0.02, seed=5)
    h, _ = oracle.rasterize(b, t, o, d)
    T = 300
    for seed in (2, 3):
        a_ref, c_ref, obj_ref = oracle.kmeans(d, gamma, h, 3, 5.0, 3, 2, T, 0.0, seed)
        p = api.pd_sinkhorn_default_params(gamma, d, max_iter=T, tol=0.0)
        a, c, obj = api.pd_kmeans(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), 3, p, 5.0, 3, 2, seed=seed)
        torch.cuda.synchronize()
        assert np.array_equal(a.cpu().numpy(), a_ref)
        assert np.allclose(obj.cpu().numpy(), obj_ref, rtol=1e-6)
        assert np.allclose(c.cpu().numpy(), c_ref, rtol=1e-5, atol=1e-9 * c_ref.max())


def test_outer_loops_reject_bad_arguments(ctx):
    h = np.zeros((2, 8, 8), np.uint32)
    h[:, 1, 2] = 1
    p = api.pd_sinkhorn_default_params(1e-2, 8)
    with pytest.raises(api.PdError):
        api.pd_barycenter(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, -1.0, 3)
    with pytest.raises(api.PdError):
        api.pd_kmeans(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), 3, p, 1.0, 2, 1)
    ps = api.pd_sinkhorn_default_params(1e-2, 8, bary_sharpen=1)
    with pytest.raises(api.PdError):
        api.pd_kmeans(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), 1, ps, 1.0, 1, 1)
