"""The benchmark's workload at full size, in the launch configuration the
benchmark times: 2048 pairs of 50-500-point diagrams (log-uniform), d = 128,
gamma = 1e-3, stop at relative marginal error 1e-6 or 20000 iterations, one
pd_sinkhorn_batch call over the rasterised batch with the pair list (2p, 2p+1).

The oracle cannot solve all 2048 pairs in a test, so it solves a sample one by
one (spread over the batch plus the largest pair) and every pair is checked
against properties that hold at any size: status, stopping error, the column
marginal of (u_t, v_t) equal to b, mass balance and a non-negative cost."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_08331_gb300 import api, inputs

pytestmark = pytest.mark.gpu

D, GAMMA, TOL, MAX_ITER, P, SEED = 128, 1e-3, 1e-6, 20000, 2048, 1


@pytest.fixture(scope="module")
def solved():
    api.load(build_if_missing=True)
    ctx = api.Context(0)
    b, t, o = inputs.random_diagrams(2 * P, nmin=50, nmax=500, exp_mean=0.2, seed=SEED)
    db, dt, do = (torch.from_numpy(x).cuda() for x in (b, t, o))
    hist, mass = api.pd_rasterize(ctx, db, dt, do, D)
    pairs = torch.arange(2 * P, dtype=torch.int32, device="cuda").view(P, 2).contiguous()
    prm = api.pd_sinkhorn_default_params(GAMMA, D, max_iter=MAX_ITER, tol=TOL)
    out = api.pd_sinkhorn_batch(ctx, hist, mass, hist, mass, prm, pairs=pairs, want_marginals=True)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    h = hist.cpu().numpy().view(np.uint32).reshape(2 * P, D, D)
    ctx.close()
    return h, res


def test_fullsize_invariants_every_pair(solved):
    h, r = solved
    st, it, err, cost = r["status"], r["iters"], r["err"], r["cost"]
    assert set(np.unique(st)) <= {api.PD_OK, api.PD_NOT_CONVERGED}
    assert np.all(err[st == api.PD_OK] <= TOL)
    assert np.all(it[st == api.PD_NOT_CONVERGED] == MAX_ITER)
    assert np.all(np.isfinite(cost)) and np.all(cost >= 0)
    nA = h[0::2].reshape(P, -1).sum(1).astype(np.float64)
    nB = h[1::2].reshape(P, -1).sum(1).astype(np.float64)
    b = np.concatenate([h[1::2].reshape(P, -1).astype(np.float64), nA[:, None]], 1)
    total = nA + nB
    # (u_t, v_t): the v-update makes the column marginal equal to b
    col_err = np.abs(r["col_marg"].astype(np.float64) - b).sum(1) / total
    assert col_err.max() <= 1e-5, col_err.max()
    # both marginals carry the same mass
    mass_gap = np.abs(r["row_marg"].astype(np.float64).sum(1) - r["col_marg"].astype(np.float64).sum(1)) / total
    assert mass_gap.max() <= 1e-5 + 2 * err.max(), mass_gap.max()


def test_fullsize_sampled_pairs_match_oracle(solved):
    h, r = solved
    nnz = (h.reshape(2 * P, -1) > 0).sum(1)
    largest = int(np.argmax(nnz[0::2] + nnz[1::2]))
    sample = sorted({0, 511, 1024, P - 1, largest})
    hA = h[[2 * p for p in sample]]
    hB = h[[2 * p + 1 for p in sample]]
    ref = oracle.sinkhorn_pd_batch(D, GAMMA, hA, hB, MAX_ITER, TOL)
    for k, p in enumerate(sample):
        rel = abs(r["cost"][p] - ref["cost"][k]) / ref["cost"][k]
        if r["iters"][p] == MAX_ITER and ref["iters"][k] == MAX_ITER:
            assert rel <= 1e-6, (p, rel)          # the same iterate on both sides
        else:
            assert rel <= 5e-6, (p, rel, r["iters"][p], ref["iters"][k])


def test_fullsize_upper_bound_within_rounding_distance(solved):
    """Prop. 3 on the full batch: the rounded plan R differs from P by at most
    2 (|r(P) - a|_1 + |c(P) - b|_1) in l1 (the rounding lemma of the
    supplementary), and C <= 2 on the grid, so |<R,C> - <P,C>| is at most
    4 x the plan's marginal error in mass units, for every pair."""
    h, r = solved
    api.load(build_if_missing=True)
    ctx = api.Context(0)
    hist = torch.from_numpy(h.reshape(2 * P, D, D).view(np.int32)).cuda()
    mass = torch.from_numpy(h.reshape(2 * P, -1).sum(1).astype(np.uint32).view(np.int32)).cuda()
    pairs = torch.arange(2 * P, dtype=torch.int32, device="cuda").view(P, 2).contiguous()
    prm = api.pd_sinkhorn_default_params(GAMMA, D, max_iter=MAX_ITER, tol=TOL)
    u = api.pd_sinkhorn_bounds(ctx, hist, mass, hist, mass, prm, pairs=pairs)
    torch.cuda.synchronize()
    cost, upper, lower = u["cost"].cpu().numpy(), u["upper"].cpu().numpy(), u["lower"].cpu().numpy()
    ctx.close()
    assert np.array_equal(u["iters"].cpu().numpy(), r["iters"])
    nA = h[0::2].reshape(P, -1).sum(1).astype(np.float64)
    nB = h[1::2].reshape(P, -1).sum(1).astype(np.float64)
    a = np.concatenate([h[0::2].reshape(P, -1).astype(np.float64), nB[:, None]], 1)
    b = np.concatenate([h[1::2].reshape(P, -1).astype(np.float64), nA[:, None]], 1)
    dev_l1 = np.abs(r["row_marg"] - a).sum(1) + np.abs(r["col_marg"] - b).sum(1)
    assert np.all(np.isfinite(upper)) and np.all(np.isfinite(lower))
    assert np.all(np.abs(upper - cost) <= 4.0 * dev_l1 + 1e-6 * cost + 1e-9)
    # m_t <= L_C <= M_t on every pair (weak duality and feasibility of R)
    assert np.all(lower <= upper + 1e-12 * upper)
