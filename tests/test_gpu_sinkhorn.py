"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1805_08331_gb300 import api, inputs
from gpu_util import dev, hists_to_gpu, masses, raster_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    api.load(build_if_missing=True)
    c = api.Context(0)
    yield c
    c.close()


def _solve(ctx, hA, hB, d, gamma, max_iter, tol, precision=api.PD_FP32, pairs=None, refine_iters=0, prm=None, **kw):
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=max_iter, tol=tol, precision=precision,
                                       refine_iters=refine_iters, **(prm or {}))
    out = api.pd_sinkhorn_batch(ctx, hists_to_gpu(hA), dev(masses(hA).view(np.int32)), hists_to_gpu(hB),
                                dev(masses(hB).view(np.int32)), p, pairs=pairs, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


# --------------------------------------------------------------------------- rasteriser (bit-exact)
@pytest.mark.parametrize("d", [2, 7, 32, 100, 128, 256])
def test_raster_bit_exact(ctx, d):
    b, t, o = inputs.random_diagrams(9, nmin=1, nmax=800, seed=d)
    # edge points: on the diagonal, death = 1, cell edges, the origin
    b = np.concatenate([b, [0.0, 0.5, 1.0, 0.25, 1 / d]])
    t = np.concatenate([t, [0.0, 0.5, 1.0, 1.0, 2 / d]])
    o = np.concatenate([o, [len(b)]])
    hg, mg = raster_gpu(ctx, b, t, o, d)
    ho, mo = oracle.rasterize(b, t, o, d)
    assert np.array_equal(hg.cpu().numpy().view(np.uint32), ho)
    assert np.array_equal(mg.cpu().numpy().view(np.uint32), mo)


def test_raster_empty_diagrams_and_invalid(ctx):
    b = np.array([0.1, 0.2]); t = np.array([0.3, 0.9]); o = np.array([0, 0, 2, 2])
    hg, mg = raster_gpu(ctx, b, t, o, 16)
    ho, mo = oracle.rasterize(b, t, o, 16)
    assert np.array_equal(hg.cpu().numpy().view(np.uint32), ho) and list(mg.cpu().numpy()) == [0, 2, 0]
    with pytest.raises(api.PdError) as e:
        raster_gpu(ctx, np.array([0.5]), np.array([0.4]), np.array([0, 1]), 16)
    assert e.value.status == api.PD_ERR_INVALID


# --------------------------------------------------------------------------- Sinkhorn parity
@pytest.mark.parametrize("engine", [api.PD_FP32, api.PD_FP32_DENSE, api.PD_FP32_PLAIN])
def test_config1_fp32_300_iterations(ctx, engine):
    """One pair of 20-point diagrams, d=32, gamma=1e-2, exactly 300 iterations."""
    d, gamma = 32, 1e-2
    b, t, o = inputs.random_diagrams(2, nmin=20, nmax=20, seed=0)
    h, _ = oracle.rasterize(b, t, o, d)
    r = oracle.sinkhorn_pd(d, gamma, h[0], h[1], 300, 0.0)
    g = _solve(ctx, h[:1], h[1:], d, gamma, 300, 0.0, precision=engine, want_marginals=True, want_potentials=True)
    assert g["iters"][0] == 300 and r["iters"] == 300
    assert g["status"][0] == api.PD_NOT_CONVERGED
    assert abs(g["cost"][0] - r["cost"]) <= 1e-6 * r["cost"]
    assert abs(g["err"][0] - r["err"]) <= 1e-6 + 1e-3 * r["err"]
    a, bb = oracle.augment(h[0], h[1])
    assert np.allclose(g["row_marg"][0], r["rmarg"], rtol=2e-6, atol=1e-6)
    assert np.allclose(g["col_marg"][0], r["cmarg"], rtol=2e-6, atol=1e-6)
    ma, mb = a > 0, bb > 0
    assert np.allclose(g["f"][0][ma], r["f"][ma], rtol=0, atol=gamma * 2e-5)
    assert np.allclose(g["g"][0][mb], r["g"][mb], rtol=0, atol=gamma * 2e-5)


@pytest.mark.parametrize("d,gamma", [(100, 1e-3), (128, 1e-3), (64, 5e-3)])
def test_small_gamma_fixed_iterations(ctx, d, gamma):
    """Paper-shaped pairs (50-500 points), log-stabilised small gamma, fixed 400
    iterations on both sides: relative cost error <= 1e-6."""
    b, t, o = inputs.random_diagrams(6, nmin=50, nmax=500, seed=d)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    ref = oracle.sinkhorn_pd_batch(d, gamma, hA, hB, 400, 0.0)
    g = _solve(ctx, hA, hB, d, gamma, 400, 0.0)
    assert np.all(g["iters"] == 400)
    rel = np.abs(g["cost"] - ref["cost"]) / ref["cost"]
    assert rel.max() <= 1e-6, rel


def test_marginals_and_potentials_elementwise_at_d128_gamma1e3(ctx):
    """The benchmark's grid and gamma, fixed 400 iterations on both sides:
    row and column marginals of the plan and the potentials f, g on the
    supports (and Delta) agree element by element with the FP64 oracle."""
    d, gamma, T = 128, 1e-3, 400
    b, t, o = inputs.random_diagrams(6, nmin=50, nmax=500, seed=5)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    g = _solve(ctx, hA, hB, d, gamma, T, 0.0, want_marginals=True, want_potentials=True)
    for p in range(3):
        r = oracle.sinkhorn_pd(d, gamma, hA[p], hB[p], T, 0.0)
        a, bb = oracle.augment(hA[p], hB[p])
        ma, mb = a > 0, bb > 0
        assert np.allclose(g["row_marg"][p], r["rmarg"], rtol=5e-6, atol=1e-6)
        assert np.allclose(g["col_marg"][p], r["cmarg"], rtol=5e-6, atol=1e-6)
        assert np.allclose(g["f"][p][ma], r["f"][ma], rtol=0, atol=gamma * 2e-5)
        assert np.allclose(g["g"][p][mb], r["g"][mb], rtol=0, atol=gamma * 2e-5)
        assert abs(g["cost"][p] - r["cost"]) <= 1e-6 * r["cost"]


def _pw_rule(h, pairs_a, pairs_b, ratio=5):
    """The automatic form rule of the iteration kernel, restated: a half-step
    (input side i, output side o) is pairwise while nnz(i) nnz(o) <=
    ratio (nnz(i) cols(o) + rows(i) nnz(o))."""
    nz = h > 0
    nnz = nz.reshape(len(h), -1).sum(1)
    rows, cols = nz.any(2).sum(1), nz.any(1).sum(1)
    out = []
    for a, b in zip(pairs_a, pairs_b):
        for i, o in ((b, a), (a, b)):
            out.append(nnz[i] * nnz[o] <= ratio * (nnz[i] * cols[o] + rows[i] * nnz[o]))
    return np.array(out)


@pytest.mark.parametrize("form", [1, 2])
def test_lse_forms_match_oracle_elementwise_at_d128_gamma1e3(ctx, form):
    """The separable (1) and pairwise (2) log-sum-exp forms each match the FP64
    oracle at the benchmark's grid and gamma after 400 fixed iterations:
    cost 1e-6 relative, marginals and potentials element by element."""
    d, gamma, T = 128, 1e-3, 400
    b, t, o = inputs.random_diagrams(8, nmin=50, nmax=500, seed=11)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    g = _solve(ctx, hA, hB, d, gamma, T, 0.0, prm={"lse_form": form}, want_marginals=True, want_potentials=True)
    assert np.all(g["iters"] == T)
    for p in range(4):
        r = oracle.sinkhorn_pd(d, gamma, hA[p], hB[p], T, 0.0)
        a, bb = oracle.augment(hA[p], hB[p])
        ma, mb = a > 0, bb > 0
        assert abs(g["cost"][p] - r["cost"]) <= 1e-6 * r["cost"]
        assert np.allclose(g["row_marg"][p], r["rmarg"], rtol=5e-6, atol=1e-6)
        assert np.allclose(g["col_marg"][p], r["cmarg"], rtol=5e-6, atol=1e-6)
        assert np.allclose(g["f"][p][ma], r["f"][ma], rtol=0, atol=gamma * 2e-5)
        assert np.allclose(g["g"][p][mb], r["g"][mb], rtol=0, atol=gamma * 2e-5)


@pytest.mark.parametrize("d,gamma,nmin,nmax", [(32, 1e-2, 5, 60), (64, 5e-3, 30, 300), (256, 2e-3, 20, 150)])
def test_lse_forms_converged_against_oracle(ctx, d, gamma, nmin, nmax):
    """Both forms run to a 1e-6 stop on small and large grids, as the oracle
    does: costs within 5e-6 of the oracle's and of each other (the stop's own
    effect), iteration counts within 15 %."""
    b, t, o = inputs.random_diagrams(8, nmin=nmin, nmax=nmax, seed=d + 3)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    ref = oracle.sinkhorn_pd_batch(d, gamma, hA, hB, 20000, 1e-6)
    res = {f: _solve(ctx, hA, hB, d, gamma, 20000, 1e-6, prm={"lse_form": f}) for f in (1, 2)}
    for f, g in res.items():
        assert np.all(g["status"] == api.PD_OK) and np.all(g["err"] <= 1e-6), (f, g["status"])
        rel = np.abs(g["cost"] - ref["cost"]) / ref["cost"]
        assert rel.max() <= 5e-6, (f, rel)
        assert np.all(np.abs(g["iters"] - ref["iters"]) <= 0.15 * ref["iters"] + 2), (f, g["iters"], ref["iters"])
    assert (np.abs(res[1]["cost"] - res[2]["cost"]) / ref["cost"]).max() <= 5e-6


def test_pair_alone_equals_pair_in_a_batch(ctx):
    """A pair's result does not depend on the batch around it: solved alone it
    equals the same pair solved inside a batch of 600 bit for bit (the batch
    orders its CTAs by support size and runs them side by side on the SMs)."""
    d, gamma = 128, 1e-3
    b, t, o = inputs.random_diagrams(1200, nmin=50, nmax=500, seed=21)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    big = _solve(ctx, hA, hB, d, gamma, 3000, 1e-6, want_potentials=True)
    for p in (0, 7, 599):
        one = _solve(ctx, hA[p:p + 1], hB[p:p + 1], d, gamma, 3000, 1e-6, want_potentials=True)
        for k in ("cost", "iters", "err", "status", "f", "g"):
            assert np.array_equal(one[k][0], big[k][p]), (p, k)


def test_pair_too_large_for_records_takes_the_separable_form(ctx):
    """A pair that fits in shared memory only without the pairwise records (a
    dense d = 100 histogram, ~4640 cells, against a small diagram: both
    half-steps pairwise by the rule, but the records alone take ~238 KB) takes
    the separable form on chip in the automatic rule: bit for bit the result
    of form 1, and the oracle's cost after 100 fixed iterations."""
    d, gamma, T = 100, 5e-3, 100
    b1, t1, o1 = inputs.random_diagrams(1, nmin=60000, nmax=60000, seed=31)
    b2, t2, o2 = inputs.random_diagrams(1, nmin=150, nmax=150, seed=32)
    hA, _ = oracle.rasterize(b1, t1, o1, d)
    hB, _ = oracle.rasterize(b2, t2, o2, d)
    assert (hA > 0).sum() > 4600 and _pw_rule(np.concatenate([hA, hB]), [0], [1]).all()
    r0, r1 = (_solve(ctx, hA, hB, d, gamma, T, 0.0, prm={"lse_form": f}, want_potentials=True) for f in (0, 1))
    for k in ("cost", "f", "g", "err"):
        assert np.array_equal(r0[k], r1[k]), k
    ref = oracle.sinkhorn_pd(d, gamma, hA[0], hB[0], T, 0.0)
    assert abs(r0["cost"][0] - ref["cost"]) <= 1e-6 * ref["cost"]


def test_automatic_form_follows_the_rule(ctx):
    """Form 0 chooses per half-step: on sparse diagrams at d = 128 (every
    half-step pairwise by the rule) it equals form 2 bit for bit; on dense
    histograms at d = 32 (every half-step separable) it equals form 1; for
    p != 2 the pairwise form is not used, so form 2 equals form 1."""
    d, gamma = 128, 1e-3
    b, t, o = inputs.random_diagrams(8, nmin=50, nmax=500, seed=12)
    h, _ = oracle.rasterize(b, t, o, d)
    assert _pw_rule(h, range(0, 8, 2), range(1, 8, 2)).all()
    r0, r1, r2 = (_solve(ctx, h[0::2], h[1::2], d, gamma, 200, 0.0, prm={"lse_form": f}, want_potentials=True)
                  for f in (0, 1, 2))
    for k in ("cost", "f", "g", "err"):
        assert np.array_equal(r0[k], r2[k]), k
    assert not np.array_equal(r0["f"], r1["f"])   # the forms round differently
    d = 32
    b, t, o = inputs.random_diagrams(4, nmin=3000, nmax=3000, seed=13)
    h, _ = oracle.rasterize(b, t, o, d)
    assert not _pw_rule(h, [0, 2], [1, 3]).any()
    r0, r1 = (_solve(ctx, h[0::2], h[1::2], d, 1e-2, 150, 0.0, prm={"lse_form": f}, want_potentials=True)
              for f in (0, 1))
    for k in ("cost", "f", "g", "err"):
        assert np.array_equal(r0[k], r1[k]), k
    b, t, o = inputs.random_diagrams(4, nmin=50, nmax=200, seed=14)
    h, _ = oracle.rasterize(b, t, o, 64)
    r1, r2 = (_solve(ctx, h[0::2], h[1::2], 64, 5e-3, 150, 0.0, prm={"lse_form": f, "p": 1.5}, want_potentials=True)
              for f in (1, 2))
    for k in ("cost", "f", "g", "err"):
        assert np.array_equal(r1[k], r2[k]), k


@pytest.mark.parametrize("tier", [0, 1, 2])
def test_d256_matches_oracle_on_every_tier(ctx, tier):
    """d = 256 (the largest grid) on small diagrams, so the FP64 oracle stays
    fast: the on-chip kernel, its global-memory variant and the FP64 kernel
    each match the oracle after 300 iterations (cost 1e-6 relative, marginals
    and potentials element by element)."""
    d, gamma, T = 256, 5e-3, 300
    b, t, o = inputs.random_diagrams(4, nmin=30, nmax=120, seed=256)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    g = _solve(ctx, hA, hB, d, gamma, T, 0.0, prm={"kernel_tier": tier}, want_marginals=True, want_potentials=True)
    assert np.all(g["iters"] == T)
    for p in range(2):
        r = oracle.sinkhorn_pd(d, gamma, hA[p], hB[p], T, 0.0)
        a, bb = oracle.augment(hA[p], hB[p])
        ma, mb = a > 0, bb > 0
        assert abs(g["cost"][p] - r["cost"]) <= 1e-6 * r["cost"]
        assert np.allclose(g["row_marg"][p], r["rmarg"], rtol=5e-6, atol=1e-6)
        assert np.allclose(g["col_marg"][p], r["cmarg"], rtol=5e-6, atol=1e-6)
        assert np.allclose(g["f"][p][ma], r["f"][ma], rtol=0, atol=gamma * 2e-5)
        assert np.allclose(g["g"][p][mb], r["g"][mb], rtol=0, atol=gamma * 2e-5)


@pytest.mark.parametrize("form", [0, 1, 2])
def test_cta_width_and_widening_leave_results_bitwise_equal(ctx, form):
    """The base-2 kernel sums in the same order at 256, 512 and 1024 threads
    per pair (stage-1 and stage-2 sums are per element or per 4-lane group,
    the Delta sum has a fixed 256-lane partition, the marginal error is an
    exact fixed-point sum; the pairwise form's lanes per cell are chosen from
    the supports at a fixed reference width), so costs, potentials, errors
    and iteration counts are bitwise equal across CTA widths, and handing the
    last pairs of a launch to wider CTAs (which pairs depends on timing)
    changes no result.  Every log-sum-exp form."""
    d, gamma, P = 32, 1e-2, 400
    b, t, o = inputs.random_diagrams(2 * P, nmin=10, nmax=150, seed=77)
    h, _ = oracle.rasterize(b, t, o, d)
    runs = {}
    for thr in (256, 128, 512, 1024, 0):
        ctx.profile_enable(True)
        before = ctx.profile_read().get("iter", (0.0, 0))[1]
        runs[thr] = _solve(ctx, h[0::2], h[1::2], d, gamma, 3000, 1e-6, prm={"cta_threads": thr, "lse_form": form},
                           want_potentials=True)
        runs[thr]["launches"] = ctx.profile_read().get("iter", (0.0, 0))[1] - before
        ctx.profile_enable(False)
    ref = runs[256]
    assert ref["launches"] == 1 and len(set(ref["iters"].tolist())) > 50   # one launch; varied stops
    # the widening (hand-over of the last pairs to wider CTAs) runs for the
    # separable form; pairwise-only batches keep their width
    assert (runs[0]["launches"] > 1) == (form == 1)
    for thr, r in runs.items():
        for k in ("cost", "iters", "err", "status", "f", "g"):
            assert np.array_equal(r[k], ref[k]), (thr, k)


@pytest.mark.parametrize("tier", [1, 2])
def test_kernel_tiers_match_oracle(ctx, tier):
    """Every pair forced into the global-memory variant of the base-2 kernel
    (gm) or into the FP64 global-memory kernel (fp64): same iterates as the
    oracle after 400 iterations at d=128, gamma=1e-3 (relative cost <= 1e-6)."""
    d, gamma = 128, 1e-3
    b, t, o = inputs.random_diagrams(4, nmin=50, nmax=500, seed=d)
    h, _ = oracle.rasterize(b, t, o, d)
    ref = oracle.sinkhorn_pd_batch(d, gamma, h[0::2], h[1::2], 400, 0.0)
    g = _solve(ctx, h[0::2], h[1::2], d, gamma, 400, 0.0, prm={"kernel_tier": tier})
    assert np.all(g["iters"] == 400)
    rel = np.abs(g["cost"] - ref["cost"]) / ref["cost"]
    assert rel.max() <= 1e-6, rel


def test_large_supports_global_variant_vs_fp64_kernel(ctx):
    """Pairs of 4000-point diagrams at d=256 have supports too large for shared
    memory, so the default path runs them in the global-memory base-2 variant;
    the independent FP64 global-memory kernel gives the same iterates."""
    d, gamma = 256, 5e-3
    b, t, o = inputs.random_diagrams(4, nmin=4000, nmax=4000, seed=11)
    h, _ = oracle.rasterize(b, t, o, d)
    nnz = (h.reshape(4, -1) > 0).sum(1)
    assert np.all(nnz[0::2] + nnz[1::2] > 5000)   # beyond the on-chip limit (~4.8k cells at d=256)
    g = _solve(ctx, h[0::2], h[1::2], d, gamma, 150, 0.0)
    r = _solve(ctx, h[0::2], h[1::2], d, gamma, 150, 0.0, prm={"kernel_tier": 2})
    assert np.all(g["iters"] == 150) and np.all(r["iters"] == 150)
    rel = np.abs(g["cost"] - r["cost"]) / r["cost"]
    assert rel.max() <= 1e-6, rel


def test_small_gamma_converged(ctx):
    """Stopping at relative marginal error 1e-6: costs agree with the converged
    oracle within the stopping tolerance's effect."""
    d, gamma = 100, 1e-3
    b, t, o = inputs.random_diagrams(4, nmin=50, nmax=500, seed=1)
    h, _ = oracle.rasterize(b, t, o, d)
    ref = oracle.sinkhorn_pd_batch(d, gamma, h[0::2], h[1::2], 20000, 1e-6)
    g = _solve(ctx, h[0::2], h[1::2], d, gamma, 20000, 1e-6)
    assert np.all(g["status"] == api.PD_OK)
    assert np.all(g["err"] <= 1e-6)
    rel = np.abs(g["cost"] - ref["cost"]) / ref["cost"]
    assert rel.max() <= 5e-6, rel
    # near err = tol the FP32-level potentials (~1e-7) make err_t uncertain by ~10%,
    # which moves the stopping iteration of very slowly converging pairs
    assert np.all(np.abs(g["iters"] - ref["iters"]) <= 0.15 * ref["iters"] + 2)


@pytest.fixture(scope="module")
def continuation_case():
    d, gamma = 64, 1e-3
    b, t, o = inputs.random_diagrams(6, nmin=50, nmax=200, seed=3)
    h, _ = oracle.rasterize(b, t, o, d)
    exact = oracle.sinkhorn_pd_batch(d, gamma, h[0::2], h[1::2], 200000, 1e-10)
    return d, gamma, h, exact


@pytest.mark.parametrize("stages", [2, 4])
def test_gamma_continuation_same_fixed_point(ctx, stages, continuation_case):
    """NEXT-2 (epsilon-scaling): stages at gamma * 4^k carry the potentials to
    the target gamma, which then stops at the same marginal tolerance (1e-6)
    as the plain solve.  Both stop on different paths to the same fixed point,
    so both are compared with the fixed point itself (the oracle converged to
    1e-10): a 1e-6 stop leaves cost errors of ~1e-5.  (Whether the stages save
    iterations depends on the pairs; the benchmark batch measures it.)"""
    d, gamma, h, exact = continuation_case
    plain = _solve(ctx, h[0::2], h[1::2], d, gamma, 20000, 1e-6)
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=20000, tol=1e-6, eps_stages=stages)
    out = api.pd_sinkhorn_batch(ctx, hists_to_gpu(h[0::2]), dev(masses(h[0::2]).view(np.int32)),
                                hists_to_gpu(h[1::2]), dev(masses(h[1::2]).view(np.int32)), p)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    assert np.all(exact["err"] <= 1e-10)
    assert np.all(g["status"] == api.PD_OK) and np.all(g["err"] <= 1e-6)
    rel_eps = np.abs(g["cost"] - exact["cost"]) / exact["cost"]
    rel_plain = np.abs(plain["cost"] - exact["cost"]) / exact["cost"]
    assert rel_plain.max() <= 3e-5 and rel_eps.max() <= 3e-5, (rel_plain, rel_eps)


@pytest.mark.parametrize("d,gamma,pw,T", [(32, 1e-2, 1.0, 300), (64, 5e-3, 1.5, 200), (128, 1e-3, 1.0, 150),
                                             (100, 2e-3, 3.0, 150)])
def test_ground_cost_p_fixed_iterations(ctx, d, gamma, pw, T):
    """NEXT-3: ground cost ||.||_p^p (separable on the grid, orthogonal
    projection to the diagonal) in the PD_FP32 engine: same iterates as the
    oracle with the explicit p-cost after T iterations (relative cost 1e-6)."""
    b, t, o = inputs.random_diagrams(6, nmin=30, nmax=300, seed=d + int(10 * pw))
    h, _ = oracle.rasterize(b, t, o, d)
    ref = oracle.sinkhorn_pd_batch(d, gamma, h[0::2], h[1::2], T, 0.0, p=pw)
    prm = api.pd_sinkhorn_default_params(gamma, d, max_iter=T, tol=0.0, p=pw)
    out = api.pd_sinkhorn_batch(ctx, hists_to_gpu(h[0::2]), dev(masses(h[0::2]).view(np.int32)),
                                hists_to_gpu(h[1::2]), dev(masses(h[1::2]).view(np.int32)), prm)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    assert np.all(g["iters"] == T)
    rel = np.abs(g["cost"] - ref["cost"]) / ref["cost"]
    assert rel.max() <= 1e-6, rel


def test_ground_cost_p_rejected_where_unsupported(ctx):
    h = np.zeros((2, 8, 8), np.uint32)
    h[:, 1, 2] = 1
    hh, mm = hists_to_gpu(h), dev(masses(h).view(np.int32))
    for kw in ({"p": 0.5}, {"p": 9.0}, {"p": 1.0, "precision": api.PD_BF16}, {"p": 1.0, "precision": api.PD_FP32_DENSE}):
        prm = api.pd_sinkhorn_default_params(1e-2, 8, **kw)
        with pytest.raises(api.PdError):
            api.pd_sinkhorn_batch(ctx, hh, mm, hh, mm, prm)
    prm = api.pd_sinkhorn_default_params(1e-2, 8, p=1.0)
    with pytest.raises(api.PdError):
        api.pd_sinkhorn_bounds(ctx, hh, mm, hh, mm, prm)


@pytest.mark.parametrize("form", [0, 1, 2])
def test_pairs_index_and_edge_cases(ctx, form):
    """Pair indexing, empty diagrams, a one-cell diagram and a diagram on the
    zero-cost diagonal cells (i = j), in every log-sum-exp form: the oracle's
    converged cost; both empty gives 0, and against an empty diagram every
    point goes to the diagonal bin."""
    d, gamma = 32, 1e-2
    b, t, o = inputs.random_diagrams(3, nmin=5, nmax=30, seed=3)
    h, _ = oracle.rasterize(b, t, o, d)
    empty = np.zeros((1, d, d), np.uint32)
    one = np.zeros((1, d, d), np.uint32); one[0, 3, 20] = 2
    diag = np.zeros((1, d, d), np.uint32); diag[0, 5, 5] = 3; diag[0, 30, 30] = 1
    H = np.concatenate([h, empty, one, diag])           # 0..2 random, 3 empty, 4 one cell, 5 diagonal cells
    pairs = np.array([[0, 1], [1, 0], [2, 2], [0, 3], [3, 0], [3, 3], [4, 1], [4, 4], [5, 0], [5, 3], [4, 5]],
                     dtype=np.int32)
    g = _solve(ctx, H, H, d, gamma, 5000, 1e-9, pairs=dev(pairs), prm={"lse_form": form})
    for k, (i, j) in enumerate(pairs):
        r = oracle.sinkhorn_pd(d, gamma, H[i], H[j], 5000, 1e-9)
        assert abs(g["cost"][k] - r["cost"]) <= 2e-6 * max(r["cost"], 1e-12) + 1e-9, (k, g["cost"][k], r["cost"])
    assert g["cost"][5] == 0.0 and g["status"][5] == api.PD_OK      # both empty
    ii, jj = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    assert g["cost"][3] == pytest.approx(float((h[0] * ((jj - ii) / d) ** 2 / 2).sum()), rel=1e-6)
    assert g["cost"][9] <= 1e-12                                    # diagonal cells to the diagonal bin


def _scaled_units(gamma, d):
    """The pairwise form's scaled units, restated: grid bits G of the base-2
    number format at gamma, n1 = rint(log2(e) / (gamma d^2) 2^G) and
    kappa = log2(e) / (gamma d^2) / (n1 2^-G) (None where n1 < 1)."""
    cmax = 2.0 / gamma * math.log2(math.e) + 64.0
    e = 0
    while 2.0 ** e < 8.0 * cmax:
        e += 1
    G = min(23 - e, 12)
    s = math.log2(math.e) / (gamma * d * d)
    n1 = round(s * 2.0 ** G)
    return None if n1 < 1 else s / (n1 * 2.0 ** -G)


@pytest.mark.parametrize("gamma", [0.242, 0.7, 1.0])
def test_pairwise_form_at_the_ends_of_its_scaled_units(ctx, gamma):
    """d = 128 at large gamma, where the scaled unit is one grid step (n1 = 1):
    kappa = 1.49 (gamma 0.242) and 0.515 (gamma 0.7) sit at the two ends of
    [1/2, 3/2], where the records' hi words carry the most rescaling; at
    gamma = 1 n1 rounds to 0, so the pairwise form is not available and form 2
    runs the separable form (bit for bit form 1).  Each matches the FP64
    oracle after 100 fixed iterations: cost, marginals and potentials."""
    d, T = 128, 100
    kap = _scaled_units(gamma, d)
    assert (kap is None) if gamma == 1.0 else (0.5 <= kap <= 1.5 and abs(kap - 1.0) > 0.45)
    b, t, o = inputs.random_diagrams(6, nmin=50, nmax=500, seed=41)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    g = _solve(ctx, hA, hB, d, gamma, T, 0.0, prm={"lse_form": 2}, want_marginals=True, want_potentials=True)
    assert np.all(g["iters"] == T)
    for p in range(3):
        r = oracle.sinkhorn_pd(d, gamma, hA[p], hB[p], T, 0.0)
        a, bb = oracle.augment(hA[p], hB[p])
        ma, mb = a > 0, bb > 0
        assert abs(g["cost"][p] - r["cost"]) <= 1e-6 * r["cost"], (p, g["cost"][p], r["cost"])
        assert np.allclose(g["row_marg"][p], r["rmarg"], rtol=5e-6, atol=1e-6)
        assert np.allclose(g["col_marg"][p], r["cmarg"], rtol=5e-6, atol=1e-6)
        assert np.allclose(g["f"][p][ma], r["f"][ma], rtol=0, atol=gamma * 2e-5)
        assert np.allclose(g["g"][p][mb], r["g"][mb], rtol=0, atol=gamma * 2e-5)
    if kap is None:
        g1 = _solve(ctx, hA, hB, d, gamma, T, 0.0, prm={"lse_form": 1}, want_potentials=True)
        for k in ("cost", "f", "g", "err"):
            assert np.array_equal(g[k], g1[k]), k


@pytest.mark.parametrize("d", [2, 7])
@pytest.mark.parametrize("form", [1, 2])
def test_smallest_and_odd_grids_every_form(ctx, d, form):
    """The smallest grid (d = 2: three cells with j >= i) and an odd one,
    iterated toward 1e-9 (at most 5000 iterations) on both sides in each form:
    the oracle's costs."""
    gamma = 1e-2
    b, t, o = inputs.random_diagrams(8, nmin=5, nmax=60, seed=50 + d)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    ref = oracle.sinkhorn_pd_batch(d, gamma, hA, hB, 5000, 1e-9)
    g = _solve(ctx, hA, hB, d, gamma, 5000, 1e-9, prm={"lse_form": form})
    # a pair whose points all sit on the zero-cost cells (i = j) has a cost of
    # ~1e-5 from the entropic spread alone: it is held to FP32 potentials'
    # accuracy on the scale of its mass times one grid step's cost
    floor = 1e-7 * (hA.reshape(len(hA), -1).sum(1) + hB.reshape(len(hB), -1).sum(1)) / d ** 2
    assert np.all(np.abs(g["cost"] - ref["cost"]) <= 2e-6 * ref["cost"] + floor), (g["cost"], ref["cost"])


def test_invalid_params(ctx):
    h = np.zeros((1, 8, 8), np.uint32); h[0, 1, 2] = 1
    for kw in (dict(gamma=-1.0), dict(d=300), dict(max_iter=0), dict(lse_form=3), dict(lse_form=-1)):
        p = api.pd_sinkhorn_default_params(1e-2, 8)
        for k, v in kw.items():
            setattr(p, k, v)
        with pytest.raises(api.PdError) as e:
            api.pd_sinkhorn_batch(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), hists_to_gpu(h),
                                  dev(masses(h).view(np.int32)), p)
        assert e.value.status == api.PD_ERR_INVALID


# --------------------------------------------------------------------------- tensor-core engine
@pytest.mark.parametrize("d,gamma,npts", [(32, 1e-2, 20), (64, 5e-3, 80), (100, 1e-3, 200), (128, 1e-3, 300)])
def test_bf16_refined_matches_oracle(ctx, d, gamma, npts):
    """PD_BF16: tcgen05 BF16 phase then exact FP32 refinement to tol; the cost
    must meet the FP32 bar against the converged oracle."""
    b, t, o = inputs.random_diagrams(6, nmin=npts // 2, nmax=npts, seed=d + 7)
    h, _ = oracle.rasterize(b, t, o, d)
    tol = 1e-7 if gamma >= 5e-3 else 1e-6
    ref = oracle.sinkhorn_pd_batch(d, gamma, h[0::2], h[1::2], 40000, tol)
    g = _solve(ctx, h[0::2], h[1::2], d, gamma, 40000, tol, precision=api.PD_BF16, refine_iters=1)
    assert np.all(g["status"] == api.PD_OK), g["status"]
    rel = np.abs(g["cost"] - ref["cost"]) / ref["cost"]
    assert rel.max() <= 5e-6, rel


def test_bf16_unrefined_within_bf16_bar(ctx):
    """Without refinement the BF16 phase alone must land within the 1e-3 BF16 bar."""
    d, gamma = 32, 1e-2
    b, t, o = inputs.random_diagrams(4, nmin=20, nmax=40, seed=2)
    h, _ = oracle.rasterize(b, t, o, d)
    ref = oracle.sinkhorn_pd_batch(d, gamma, h[0::2], h[1::2], 20000, 1e-6)
    g = _solve(ctx, h[0::2], h[1::2], d, gamma, 20000, 1e-6, precision=api.PD_BF16, refine_iters=0)
    rel = np.abs(g["cost"] - ref["cost"]) / ref["cost"]
    assert rel.max() <= 1e-3, rel


def test_plain_one_pair_per_launch_equals_batched_dense(ctx):
    """PD_FP32_PLAIN runs the dense FP32 arithmetic with one pair per launch;
    a pair's CTA does the same work whatever else is in the launch, so its
    results are bitwise those of the batched PD_FP32_DENSE engine, and within
    the FP32 bar of the oracle (k-means-shaped pairs, d = 64, gamma = 5e-3)."""
    d, gamma = 64, 5e-3
    b, t, o, _ = inputs.mode_diagrams(8, 10, 30, 300, sigma=0.03, seed=3)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    dense = _solve(ctx, hA, hB, d, gamma, 20000, 1e-6, precision=api.PD_FP32_DENSE)
    plain = _solve(ctx, hA, hB, d, gamma, 20000, 1e-6, precision=api.PD_FP32_PLAIN)
    for k in ("cost", "iters", "status", "err"):
        assert np.array_equal(plain[k], dense[k]), k
    ref = oracle.sinkhorn_pd_batch(d, gamma, hA, hB, 20000, 1e-6)
    ok = plain["status"] == api.PD_OK
    assert ok.all()
    assert np.all(np.abs(plain["cost"] - ref["cost"]) <= 2e-6 * ref["cost"])


def test_autotuner_choice_changes_speed_not_results(ctx, tmp_path):
    """pd_sinkhorn_tune times one launch per CTA width on the batch and keys its
    choice by (d, support bucket); solves that pick the tuned width give the
    same results bitwise as the built-in rule (fixed-order sums), and the table
    survives a save / load round trip; a malformed table is refused."""
    d, gamma, P = 64, 5e-3, 600
    b, t, o = inputs.random_diagrams(2 * P, nmin=20, nmax=200, seed=31)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = hists_to_gpu(h[0::2]), hists_to_gpu(h[1::2])
    mA, mB = dev(masses(h[0::2]).view(np.int32)), dev(masses(h[1::2]).view(np.int32))
    prm = api.pd_sinkhorn_default_params(gamma, d, max_iter=4000, tol=1e-6)
    ref = api.pd_sinkhorn_batch(ctx, hA, mA, hB, mB, prm, want_potentials=True)
    c2 = api.Context(0)
    try:
        th, ms = api.pd_sinkhorn_tune(c2, hA, mA, hB, mB, prm, trial_iters=48)
        assert th in (128, 256, 512) and set(ms) == {128, 256, 512} and all(v > 0 for v in ms.values())
        assert ms[th] == min(ms.values())
        path = str(tmp_path / "tune.txt")
        api.pd_tune_save(c2, path)
        c3 = api.Context(0)
        try:
            api.pd_tune_load(c3, path)
            for cx in (c2, c3):
                out = api.pd_sinkhorn_batch(cx, hA, mA, hB, mB, prm, want_potentials=True)
                for k in ("cost", "iters", "err", "status", "f", "g"):
                    assert torch.equal(out[k], ref[k]), k
            with open(path, "w") as fh:
                fh.write("64 3 333\n")
            with pytest.raises(api.PdError) as e:
                api.pd_tune_load(c3, path)
            assert e.value.status == api.PD_ERR_INVALID
        finally:
            c3.close()
    finally:
        c2.close()


def test_mixed_grid_sizes_in_one_launch_equal_separate_batches(ctx):
    """pd_sinkhorn_batch_groups runs pairs of d = 32, 64, 128 and 256 in one
    persistent launch; each pair's results are bitwise those of a
    pd_sinkhorn_batch of its own grid size (a pair's CTA does the same
    arithmetic whatever else is in the launch), and a sample agrees with the
    oracle."""
    gamma = 5e-3
    groups, refs, hs = [], [], []
    for k, (d, P) in enumerate(((32, 40), (64, 30), (128, 20), (256, 6))):
        b, t, o = inputs.random_diagrams(2 * P, nmin=10, nmax=150, seed=400 + d)
        h, _ = oracle.rasterize(b, t, o, d)
        hA, hB = hists_to_gpu(h[0::2]), hists_to_gpu(h[1::2])
        mA, mB = dev(masses(h[0::2]).view(np.int32)), dev(masses(h[1::2]).view(np.int32))
        groups.append({"d": d, "histA": hA, "massA": mA, "histB": hB, "massB": mB})
        prm = api.pd_sinkhorn_default_params(gamma, d, max_iter=3000, tol=1e-6)
        refs.append(api.pd_sinkhorn_batch(ctx, hA, mA, hB, mB, prm, want_potentials=True))
        hs.append((h[0::2], h[1::2]))
    prm = api.pd_sinkhorn_default_params(gamma, 0, max_iter=3000, tol=1e-6)
    ctx.profile_enable(True)
    outs = api.pd_sinkhorn_batch_groups(ctx, groups, prm, want_potentials=True)
    torch.cuda.synchronize()
    launches = ctx.profile_read().get("iter", (0.0, 0))[1]
    ctx.profile_enable(False)
    assert launches <= 3    # one launch for all grid sizes (plus at most the two drain hand-overs)
    for g, o, r, (hA, hB) in zip(groups, outs, refs, hs):
        for k in ("cost", "iters", "err", "status", "f", "g"):
            assert torch.equal(o[k], r[k]), (g["d"], k)
        ref = oracle.sinkhorn_pd(g["d"], gamma, hA[0], hB[0], 3000, 1e-6)
        assert abs(float(o["cost"][0]) - ref["cost"]) <= 5e-6 * ref["cost"]


def test_tensor_core_wait_timeout_path(ctx):
    """The tcgen05 kernel's bounded mbarrier wait: with the diagnostic set, the
    kernel issues no GEMM and waits with a spin limit of 0, so the wait gives up
    with no tensor-core work in flight; the kernel frees its tensor memory and
    the call reports PD_ERR_TIMEOUT.  The same context then solves normally."""
    d, gamma = 32, 1e-2
    b, t, o = inputs.random_diagrams(4, nmin=20, nmax=40, seed=2)
    h, _ = oracle.rasterize(b, t, o, d)
    with pytest.raises(api.PdError) as e:
        _solve(ctx, h[0::2], h[1::2], d, gamma, 500, 1e-6, precision=api.PD_BF16, refine_iters=1,
               prm={"diag_tc_timeout": 1})
    assert e.value.status == api.PD_ERR_TIMEOUT
    ref = oracle.sinkhorn_pd_batch(d, gamma, h[0::2], h[1::2], 20000, 1e-6)
    for prec in (api.PD_BF16, api.PD_FP32):
        g = _solve(ctx, h[0::2], h[1::2], d, gamma, 20000, 1e-6, precision=prec, refine_iters=1)
        assert np.all(g["status"] == api.PD_OK)
        assert np.all(np.abs(g["cost"] - ref["cost"]) <= 5e-6 * ref["cost"])


@pytest.mark.parametrize("engine", [api.PD_FP32_DENSE, api.PD_FP32_PLAIN])
def test_linear_domain_engines_flag_dropped_terms(ctx, engine):
    """At d = 128, gamma = 1e-3 the absorbed linear-domain representation can
    lose terms that matter; such pairs must come back PD_ERR_RANGE, never
    PD_OK with a wrong answer.  Every pair reported PD_OK has a plan whose
    marginals, evaluated by the oracle's definition from the returned
    potentials, are within the check's bound, and its cost is close to the
    converged FP64 oracle."""
    d, gamma, P = 128, 1e-3, 16
    b, t, o = inputs.random_diagrams(2 * P, nmin=50, nmax=500, seed=1)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    g = _solve(ctx, hA, hB, d, gamma, 20000, 1e-6, precision=engine, want_potentials=True)
    ref = oracle.sinkhorn_pd_batch(d, gamma, hA, hB, 20000, 1e-9)
    ok = g["status"] == api.PD_OK
    rel = np.abs(g["cost"] - ref["cost"]) / ref["cost"]
    print("status", g["status"].tolist(), "rel", np.round(rel, 8).tolist())
    assert set(g["status"].tolist()) <= {api.PD_OK, api.PD_NOT_CONVERGED, api.PD_ERR_RANGE}
    for p in np.nonzero(ok)[0]:
        a, bb = oracle.augment(hA[p], hB[p])
        sa, sb = np.nonzero(a > 0)[0], np.nonzero(bb > 0)[0]
        C = np.array([[oracle.cost(d, x, y) for y in sb] for x in sa])
        lp = (np.log(a[sa])[:, None] + np.log(bb[sb])[None, :]
              + (g["f"][p][sa][:, None] + g["g"][p][sb][None, :] - C) / gamma)
        plan = np.exp(lp)
        e = (np.abs(plan.sum(1) - a[sa]).sum() + np.abs(plan.sum(0) - bb[sb]).sum()) / a.sum()
        assert e <= 2e-5, (p, e)
        assert rel[p] <= 1e-4, (p, rel[p])


def test_split_bf16_reaches_tolerance_on_the_tensor_cores(ctx):
    """For d <= 64 the tensor-core kernel holds every operand as BF16 hi + lo
    (three MMAs per product), which carries the iteration to the 1e-6
    tolerance: on k-means-shaped pairs (d = 64, gamma = 5e-3) the refined solve
    takes about the iterations of the exact engine (the refinement adds a few),
    the tensor-core launches carry nearly all of them, and every cost is within
    the FP32 bar of the oracle."""
    d, gamma, P = 64, 5e-3, 48
    b, t, o, _ = inputs.mode_diagrams(2 * P, 10, 30, 300, sigma=0.03, seed=3)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    exact = _solve(ctx, hA, hB, d, gamma, 20000, 1e-6)
    ctx.profile_enable(True)
    bf = _solve(ctx, hA, hB, d, gamma, 20000, 1e-6, precision=api.PD_BF16, refine_iters=1)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    assert np.all(bf["status"] == api.PD_OK) and np.all(exact["status"] == api.PD_OK)
    assert np.all(bf["iters"] <= exact["iters"] * 1.05 + 8), np.max(bf["iters"] - exact["iters"])
    tc_ms, exact_ms = prof.get("tc", (0.0, 0))[0], prof.get("iter", (0.0, 0))[0]
    print("tensor-core ms", tc_ms, "exact-engine ms", exact_ms)
    ref = oracle.sinkhorn_pd_batch(d, gamma, hA[:6], hB[:6], 20000, 1e-6)
    assert np.all(np.abs(bf["cost"][:6] - ref["cost"]) <= 2e-6 * ref["cost"])


def test_marginals_without_potentials_write_every_entry(ctx):
    """Marginals requested without potentials: every entry is written (0 off
    the supports), even where the output buffers held other values before."""
    d, gamma, P = 64, 5e-3, 3
    b, t, o = inputs.random_diagrams(2 * P, nmin=20, nmax=80, seed=17)
    h, _ = oracle.rasterize(b, t, o, d)
    hA, hB = h[0::2], h[1::2]
    n = d * d + 1
    for eng in (api.PD_FP32, api.PD_FP32_DENSE):
        out = {"row_marg": torch.full((P, n), float("nan"), dtype=torch.float32, device="cuda"),
               "col_marg": torch.full((P, n), float("nan"), dtype=torch.float32, device="cuda")}
        p = api.pd_sinkhorn_default_params(gamma, d, max_iter=300, tol=0.0, precision=eng)
        g = api.pd_sinkhorn_batch(ctx, hists_to_gpu(hA), dev(masses(hA).view(np.int32)), hists_to_gpu(hB),
                                  dev(masses(hB).view(np.int32)), p, want_marginals=True, out=out)
        torch.cuda.synchronize()
        rm, cm = g["row_marg"].cpu().numpy(), g["col_marg"].cpu().numpy()
        assert np.all(np.isfinite(rm)) and np.all(np.isfinite(cm))
        for q in range(P):
            a, bb = oracle.augment(hA[q], hB[q])
            assert np.all(rm[q][a == 0] == 0) and np.all(cm[q][bb == 0] == 0)
            r = oracle.sinkhorn_pd(d, gamma, hA[q], hB[q], 300, 0.0)
            assert np.allclose(rm[q], r["rmarg"], rtol=5e-6, atol=1e-6)
            assert np.allclose(cm[q], r["cmarg"], rtol=5e-6, atol=1e-6)
