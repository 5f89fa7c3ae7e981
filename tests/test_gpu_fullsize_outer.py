"""The barycenter and k-means workloads at full size: 1000 diagrams from 3
modes at d = 100, gamma = 2e-3, 100 outer steps (Alg. 2), and k-means with
k = 10 on 5000 diagrams from 10 modes at d = 64, gamma = 5e-3, 10 rounds with
one Alg. 2 step per round (Sec. 5).

The oracle cannot redo these runs, so it checks sampled outputs one by one:
the transport costs between the GPU's final measures and sampled diagrams
(solved by both sides from the same measure), and the k-means assignment of
sampled diagrams (argmin of the oracle's costs to the GPU's centroids).  Every
output is checked against properties that hold at any size."""
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from paper_1805_08331_gb300 import api, inputs

pytestmark = pytest.mark.gpu

TOL, MAX_ITER = 1e-6, 20000


@pytest.fixture(scope="module")
def ctx():
    api.load(build_if_missing=True)
    c = api.Context(0)
    yield c
    c.close()


def _raster(ctx, b, t, o, d):
    db, dt, do = (torch.from_numpy(x).cuda() for x in (b, t, o))
    return api.pd_rasterize(ctx, db, dt, do, d)


def _oracle_costs(d, gamma, z_list, h_list):
    """FP64 oracle costs of the pairs (z + R a, a + R z), in parallel threads
    (the ctypes calls release the interpreter lock)."""
    def one(zh):
        z, h = zh
        a, b = oracle.augment(z.ravel(), h.astype(np.float64).ravel())
        return oracle.sinkhorn_w(d, gamma, a, b, MAX_ITER, TOL)["cost"]
    with ThreadPoolExecutor(max_workers=8) as ex:
        return np.array(list(ex.map(one, zip(z_list, h_list))))


def _upper_triangle_only(z):
    d = z.shape[-1]
    below = np.tril(np.ones((d, d), bool), -1)
    return np.all(z[..., below] == 0)


def test_barycenter_fullsize_1000_diagrams(ctx):
    d, gamma, lam, steps, N = 100, 2e-3, 5.0, 100, 1000
    b, t, o, _ = inputs.mode_diagrams(N, 3, 30, 300, sigma=0.03, seed=2)
    hist, mass = _raster(ctx, b, t, o, d)
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=MAX_ITER, tol=TOL)
    t0 = time.perf_counter()
    z, e = api.pd_barycenter(ctx, hist, mass, p, lam, steps)
    torch.cuda.synchronize()
    print(f"barycenter N={N} d={d} gamma={gamma} {steps} steps: {time.perf_counter() - t0:.2f} s")
    zn, en = z.cpu().numpy(), e.cpu().numpy()
    assert np.all(np.isfinite(zn)) and np.all(zn >= 0) and _upper_triangle_only(zn)
    assert np.all(np.isfinite(en)) and np.all(en > 0)
    assert en[-1] < en[0]                                   # the energy went down
    # sampled pairs (z + R a_i, a_i + R z) from the final z, both sides cold to tol
    h = hist.cpu().numpy().view(np.uint32).reshape(N, d, d)
    sample = [0, 377, N - 1]
    gpu = []
    for i in sample:
        _, _, csum = api.pd_barycenter_grad(ctx, hist[i:i + 1], mass[i:i + 1], p, z, 1)
        gpu.append(csum.item())
    ref = _oracle_costs(d, gamma, [zn] * len(sample), [h[i] for i in sample])
    rel = np.abs(np.array(gpu) - ref) / ref
    assert rel.max() <= 5e-6, rel


def test_kmeans_fullsize_5000_diagrams(ctx):
    d, gamma, k, lam, rounds, N = 64, 5e-3, 10, 5.0, 10, 5000
    b, t, o, labels = inputs.mode_diagrams(N, 10, 30, 300, sigma=0.03, seed=3)
    hist, mass = _raster(ctx, b, t, o, d)
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=MAX_ITER, tol=TOL)
    t0 = time.perf_counter()
    a, c, obj = api.pd_kmeans(ctx, hist, mass, k, p, lam, rounds, 1, seed=3)
    torch.cuda.synchronize()
    print(f"k-means N={N} k={k} d={d} gamma={gamma} {rounds} rounds: {time.perf_counter() - t0:.2f} s")
    an, cn, on = a.cpu().numpy(), c.cpu().numpy(), obj.cpu().numpy()
    assert an.min() >= 0 and an.max() < k
    assert np.all(np.isfinite(cn)) and np.all(cn >= 0) and _upper_triangle_only(cn)
    assert np.all(np.isfinite(on)) and on[-1] <= on[0]
    # how far seeding + 10 rounds recover the generative modes (reported, not a parity property)
    purity = sum(np.bincount(an[labels == m], minlength=k).max() for m in range(10)) / N
    print(f"k-means mode purity {purity:.3f}, clusters used {len(set(an.tolist()))}")
    # assignment against the final centroids: GPU costs vs the oracle's for
    # sampled diagrams, and the GPU's argmin where the oracle's is clear
    a2, _, cost = api.pd_kmeans_assign(ctx, hist, mass, p, c, want_cost=True)
    torch.cuda.synchronize()
    a2, cost = a2.cpu().numpy(), cost.cpu().numpy()
    assert np.array_equal(a2, np.argmin(cost, axis=1))
    h = hist.cpu().numpy().view(np.uint32).reshape(N, d, d)
    sample = [0, 2500, N - 1]
    ref = _oracle_costs(d, gamma, [cn[j] for _ in sample for j in range(k)],
                        [h[i] for i in sample for _ in range(k)]).reshape(len(sample), k)
    for r, i in enumerate(sample):
        rel = np.abs(cost[i] - ref[r]) / ref[r]
        assert rel.max() <= 5e-6, (i, rel)
        srt = np.sort(ref[r])
        if srt[1] - srt[0] > 1e-4 * srt[0]:
            assert a2[i] == int(np.argmin(ref[r])), (i, a2[i], ref[r])
