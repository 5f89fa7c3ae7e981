"""Sec. 3 "Upper and Lower Bounds" on the GPU, against the oracle at the same
iterate (fixed iteration counts, so both sides hold the same potentials):
the rounded plan's cost M_t = <R, C> (Prop. 3) against the oracle's literal
rounding of the dense plan, and the C-transform bound m_t against the
oracle's plain minimisation over the supports.  Early iterates have large
marginal errors, so the rank-one term is exercised; late ones check that the
bounds close in on the cost."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_08331_gb300 import api, inputs
from gpu_util import dev, hists_to_gpu, masses

pytestmark = pytest.mark.gpu

# The PD_FP32 path's potentials carry FP32-level error (cost parity 1e-6); the
# bound takes min() of the potentials and three more kernel applications from
# them (the rescalings X, Y and the residual row marginal), which turns that
# noise into a small rescaling bias; its agreement is stated at 5e-6
# (measured at most 3.4e-6 over these cases).
UPPER_REL = 5e-6


@pytest.fixture(scope="module")
def ctx():
    api.load(build_if_missing=True)
    c = api.Context(0)
    yield c
    c.close()


# m_t is exact FP64 min-plus arithmetic on the potentials; its agreement is set
# by the potentials' own error (f/gamma to ~1e-7 relative), well below this
LOWER_REL = 1e-6


def _gpu(ctx, hA, hB, d, gamma, T, tol=0.0):
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=T, tol=tol)
    out = api.pd_sinkhorn_bounds(ctx, hists_to_gpu(hA), dev(masses(hA).view(np.int32)), hists_to_gpu(hB),
                                      dev(masses(hB).view(np.int32)), p)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("d,gamma,nmin,nmax,T", [(16, 1e-2, 8, 20, 3), (16, 1e-2, 8, 20, 30), (16, 1e-2, 8, 20, 400),
                                                  (32, 5e-3, 20, 60, 2), (32, 5e-3, 20, 60, 100),
                                                  (64, 1e-3, 40, 120, 200)])
def test_upper_bound_matches_oracle_rounding(ctx, d, gamma, nmin, nmax, T):
    b, t, o = inputs.random_diagrams(6, nmin=nmin, nmax=nmax, seed=d + T)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    g = _gpu(ctx, hA, hB, d, gamma, T)
    assert np.all(g["iters"] == T)
    for k in range(3):
        a, bb = oracle.augment(hA[k], hB[k])
        r = oracle.sinkhorn_w(d, gamma, a, bb, T, 0.0)
        rb = oracle.round_bound(d, gamma, a, bb, r["f"], r["g"])
        lo = oracle.ctransform_bound(d, gamma, a, bb, r["f"])
        assert abs(g["cost"][k] - r["cost"]) <= 1e-6 * r["cost"]
        assert abs(g["lower"][k] - lo) <= LOWER_REL * abs(lo) + 1e-12, (k, g["lower"][k], lo)
        assert g["lower"][k] <= g["upper"][k]
        assert abs(g["upper"][k] - rb["upper"]) <= UPPER_REL * rb["upper"] + 1e-12, (k, g["upper"][k], rb["upper"])
        print(f"d={d} T={T} pair {k}: cost rel {abs(g['cost'][k] - r['cost']) / r['cost']:.2e}, "
              f"upper rel {abs(g['upper'][k] - rb['upper']) / rb['upper']:.2e}, upper-cost {rb['upper'] - r['cost']:.3e}")


def test_upper_bound_empty_side_and_converged(ctx):
    d, gamma = 32, 1e-2
    b, t, o = inputs.random_diagrams(2, nmin=15, nmax=15, seed=4)
    h, _ = oracle.rasterize(b, t, o, d)
    empty = np.zeros_like(h[:1])
    # B empty: the plan is forced (everything to the diagonal), R = P, both equal the closed form
    g = _gpu(ctx, h[:1], empty, d, gamma, 50, 1e-9)
    i, j = np.nonzero(h[0])
    expect = float(np.sum(h[0][i, j] * ((j - i) / d) ** 2 / 2))
    assert abs(g["cost"][0] - expect) <= 1e-7 * expect
    assert abs(g["upper"][0] - expect) <= 1e-7 * expect
    assert abs(g["lower"][0] - expect) <= 1e-12 * expect    # the forced plan: m_t is exact
    # converged to 1e-9: the exact gap is of the order of the marginal error;
    # the GPU's is bounded by the potentials' FP32-level noise (min() of two
    # noisy potentials in the rescaling), i.e. the stated UPPER_REL
    g = _gpu(ctx, h[:1], h[1:], d, gamma, 50000, 1e-9)
    assert g["status"][0] == api.PD_OK
    assert abs(g["upper"][0] - g["cost"][0]) <= UPPER_REL * g["cost"][0]
    assert g["lower"][0] <= g["cost"][0] + 1e-12
