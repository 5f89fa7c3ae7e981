"""Sec. 5 "A large scale approximation" / Fig. 3 (middle), on synthetic pairs:
100 pairs of diagrams with 100-150 points on a 100 x 100 grid, gamma from 1e-1
down to 5e-4, each solve stopped at a small marginal error, and the bounds
m_t <= L_C <= M_t of Sec. 3 around the exact cost L_C of the rasterised
diagrams (optimal partial matching of the snapped points, by an assignment
solver).  Checked on every pair and gamma: the bracket holds; the median gap
of each bound closes as gamma decreases.  The percentile table is printed
(pytest -s) as the experiment's output."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1805_08331_gb300 import api, inputs
from gpu_util import dev, hists_to_gpu, masses

pytestmark = pytest.mark.gpu

D, N = 100, 100
GAMMAS = [1e-1, 3e-2, 1e-2, 3e-3, 1e-3, 5e-4]


def _exact_cost(X, Y):
    from scipy.optimize import linear_sum_assignment
    nX, nY = len(X), len(Y)
    M = np.zeros((nX + nY, nX + nY))
    M[:nX, :nY] = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    M[:nX, nY:] = (((X[:, 1] - X[:, 0]) ** 2) / 2.0)[:, None]
    M[nX:, :nY] = (((Y[:, 1] - Y[:, 0]) ** 2) / 2.0)[None, :]
    r, c = linear_sum_assignment(M)
    return float(M[r, c].sum())


def test_fig3_bounds_bracket_and_close():
    api.load(build_if_missing=True)
    ctx = api.Context(0)
    b, t, o = inputs.random_diagrams(2 * N, nmin=100, nmax=150, seed=33, log_uniform=False)
    h, _ = oracle.rasterize(b, t, o, D)
    snap = lambda k: np.stack([np.minimum(np.floor(b[o[k]:o[k + 1]] * D), D - 1) / D,
                               np.minimum(np.floor(t[o[k]:o[k + 1]] * D), D - 1) / D], 1)
    L = np.array([_exact_cost(snap(2 * p), snap(2 * p + 1)) for p in range(N)])
    hA, hB = h[0::2], h[1::2]
    rows, med_up, med_lo = [], [], []
    for gamma in GAMMAS:
        prm = api.pd_sinkhorn_default_params(gamma, D, max_iter=20000, tol=4e-6)
        out = api.pd_sinkhorn_bounds(ctx, hists_to_gpu(hA), dev(masses(hA).view(np.int32)), hists_to_gpu(hB),
                                     dev(masses(hB).view(np.int32)), prm)
        lo, up = out["lower"].cpu().numpy(), out["upper"].cpu().numpy()
        assert np.all(lo <= L + 1e-12 * L), gamma                  # weak duality (exact FP64 min-plus)
        assert np.all(up >= L * (1 - 1e-5)), gamma                 # R is feasible (bound carries ~5e-6 error)
        gu, gl = (up - L) / L, (lo - L) / L
        med_up.append(np.median(gu))
        med_lo.append(np.median(gl))
        rows.append((gamma, np.percentile(gu, 10), np.median(gu), np.percentile(gu, 90),
                     np.percentile(gl, 10), np.median(gl), np.percentile(gl, 90)))
    ctx.close()
    print("\n gamma    | (M-L)/L p10   median     p90   | (m-L)/L p10   median     p90")
    for r in rows:
        print(" %-8g | %9.2e %9.2e %9.2e | %9.2e %9.2e %9.2e" % r)
    # both gaps close as gamma decreases (median over the pairs), at least half
    # as fast as gamma itself (the smoothing error is O(gamma n log n))
    assert all(a > b for a, b in zip(med_up, med_up[1:]))
    assert all(-a > -b for a, b in zip(med_lo, med_lo[1:]))
    for k in range(2, len(GAMMAS)):
        assert med_up[k] / med_up[k - 2] <= 2.0 * GAMMAS[k] / GAMMAS[k - 2]
        assert med_lo[k] / med_lo[k - 2] <= 2.0 * GAMMAS[k] / GAMMAS[k - 2]
