"""Pins for the FP64 oracle against what the paper and mathematics fix.

Every test here checks the oracle against something other than itself:
hand-worked cells, geometric definitions, closed forms of small transport
problems, brute-force optimal matchings, finite differences and invariants.
None needs a GPU.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1805_08331_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hist(d, cells):
    h = np.zeros((d, d), dtype=np.uint32)
    for (i, j) in cells:
        h[i, j] += 1
    return h


# --------------------------------------------------------------------------- rasteriser
def test_raster_golden_cells():
    """Sec. 3 'Discretization': hand-worked cells (golden fixture)."""
    with open(os.path.join(GOLDEN, "raster_cases.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        d = c["d"]
        b = np.array(c["birth"])
        t = np.array(c["death"])
        hist, mass = oracle.rasterize(b, t, np.array([0, len(b)]), d)
        assert mass[0] == len(b)
        assert np.array_equal(hist[0], _hist(d, c["cells"]))


def test_raster_exact_rational_recount():
    """Recount with exact rational floor; FP64 floor(x*d) may differ only where
    the rounded product lands on an integer (the reading both sides adopt)."""
    b, t, o = inputs.random_diagrams(5, nmin=200, nmax=200, seed=11)
    for d in (7, 32, 100, 128):
        hist, mass = oracle.rasterize(b, t, o, d)
        for k in range(5):
            ref = np.zeros((d, d), dtype=np.int64)
            n_round = 0
            for p in range(o[k], o[k + 1]):
                ie = min(math.floor(Fraction(b[p]) * d), d - 1)
                je = min(math.floor(Fraction(t[p]) * d), d - 1)
                ifp = min(math.floor(b[p] * d), d - 1)
                jfp = min(math.floor(t[p] * d), d - 1)
                if (ie, je) != (ifp, jfp):
                    n_round += 1
                    assert float(b[p] * d).is_integer() or float(t[p] * d).is_integer()
                ref[ifp, jfp] += 1
            assert n_round <= 2
            assert np.array_equal(hist[k].astype(np.int64), ref)
            assert mass[k] == o[k + 1] - o[k] == hist[k].sum()


def test_raster_rejects_bad_points():
    for bb, tt in ((0.5, 0.4), (-0.1, 0.2), (0.1, 1.5), (float("nan"), 0.5)):
        with pytest.raises(ValueError):
            oracle.rasterize(np.array([bb]), np.array([tt]), np.array([0, 1]), 8)


# --------------------------------------------------------------------------- cost
def test_cost_matches_geometry():
    """Prop. 1 block cost: grid-grid = squared Euclidean distance of the cell
    points; grid-Delta = squared distance to the orthogonal projection onto the
    diagonal; Delta-Delta = 0 (p = 2, physical units on [0,1]^2)."""
    rng = np.random.default_rng(3)
    for d in (5, 32, 100):
        D = d * d
        for _ in range(50):
            x, y = rng.integers(0, D, size=2)
            px = np.array([x // d, x % d]) / d
            py = np.array([y // d, y % d]) / d
            assert oracle.cost(d, x, y) == pytest.approx(np.linalg.norm(px - py) ** 2, rel=1e-13, abs=1e-16)
            e = np.array([1.0, 1.0]) / math.sqrt(2.0)
            proj = (px @ e) * e
            assert oracle.cost(d, x, D) == pytest.approx(np.linalg.norm(px - proj) ** 2, rel=1e-12, abs=1e-16)
            assert oracle.cost(d, D, y) == pytest.approx(np.linalg.norm(py - (py @ e) * e) ** 2, rel=1e-12, abs=1e-16)
        assert oracle.cost(d, D, D) == 0.0


# --------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("gamma", [1e-1, 1e-2, 1e-3])
def test_empty_diagram_closed_form(gamma):
    """D_B empty: b = (0, n_A), the only feasible plan sends every point to
    Delta, so <P,C> = sum_x a_x C_xDelta at any gamma (Prop. 1)."""
    d = 32
    b, t, o = inputs.random_diagrams(1, nmin=40, nmax=40, seed=5)
    hA, _ = oracle.rasterize(b, t, o, d)
    hB = np.zeros_like(hA[0])
    r = oracle.sinkhorn_pd(d, gamma, hA[0], hB, 50, 1e-15)
    ii, jj = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    expect = float((hA[0] * ((jj - ii) / d) ** 2 / 2.0).sum())
    assert r["cost"] == pytest.approx(expect, rel=1e-12)
    assert r["iters"] <= 3
    assert np.allclose(r["rmarg"][:-1], hA[0].ravel(), rtol=1e-12)


def _two_by_two(mx, my, Cxy, CxD, CyD, gamma):
    """Plan [[t, mx-t], [my-t, t]] of the 2x2 augmented problem; optimality of
    Eq. (SinkhornMinimizationProblem) gives t^2 = exp(-D/gamma)(mx-t)(my-t),
    D = Cxy - CxD - CyD (the Delta-Delta cost is 0)."""
    from scipy.optimize import brentq
    q = math.exp(-(Cxy - CxD - CyD) / gamma)
    # (1-q) t^2 + q(mx+my) t - q mx my: negative at 0, equal to min(mx,my)^2 at min(mx,my)
    poly = lambda tt: (1 - q) * tt * tt + q * (mx + my) * tt - q * mx * my
    tt = brentq(poly, 0.0, float(min(mx, my)), xtol=1e-15, rtol=1e-15)
    return tt * Cxy + (mx - tt) * CxD + (my - tt) * CyD


@pytest.mark.parametrize("mx,my,gamma", [(1, 1, 0.05), (3, 2, 0.05), (2, 5, 0.2), (1, 1, 0.02)])
def test_one_cell_vs_one_cell_closed_form(mx, my, gamma):
    d = 16
    hA = np.zeros((d, d), np.uint32)
    hB = np.zeros((d, d), np.uint32)
    hA[3, 9] = mx
    hB[5, 12] = my
    r = oracle.sinkhorn_pd(d, gamma, hA, hB, 200000, 1e-14)
    Cxy = ((3 - 5) ** 2 + (9 - 12) ** 2) / d**2
    CxD = (9 - 3) ** 2 / (2 * d**2)
    CyD = (12 - 5) ** 2 / (2 * d**2)
    assert r["cost"] == pytest.approx(_two_by_two(mx, my, Cxy, CxD, CyD, gamma), rel=1e-9)


# --------------------------------------------------------------------------- exact OT limit
def _snapped_points(b, t, d):
    i = np.minimum(np.floor(b * d), d - 1) / d
    j = np.minimum(np.floor(t * d), d - 1) / d
    return np.stack([i, j], 1)


def _diag_matching_sq(X, Y):
    """d_2^2 of Eq. (Wasserstein_Dgm) by the augmented assignment of the
    proof of Prop. 1: an (nX+nY) square cost, Delta row/column repeated,
    zeros in the Delta-Delta block."""
    from scipy.optimize import linear_sum_assignment
    nX, nY = len(X), len(Y)
    n = nX + nY
    M = np.zeros((n, n))
    dX = ((X[:, 1] - X[:, 0]) ** 2) / 2.0
    dY = ((Y[:, 1] - Y[:, 0]) ** 2) / 2.0
    M[:nX, :nY] = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    M[:nX, nY:] = dX[:, None]
    M[nX:, :nY] = dY[None, :]
    r, c = linear_sum_assignment(M)
    return float(M[r, c].sum()), M


def test_assignment_matches_permutations():
    """The scipy assignment used below equals the minimum over all permutations."""
    rng = np.random.default_rng(0)
    for _ in range(5):
        X = np.sort(rng.random((3, 2)), axis=1)
        Y = np.sort(rng.random((4, 2)), axis=1)
        v, M = _diag_matching_sq(X, Y)
        n = M.shape[0]
        best = min(sum(M[i, p[i]] for i in range(n)) for p in itertools.permutations(range(n)))
        assert v == pytest.approx(best, rel=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gamma_to_zero_matches_brute_force(seed):
    """Prop. 1 + Eq. (Altschuler bounds): 0 <= S^gamma - d_2^2(snapped) <=
    2 gamma n log n + err*||C||_inf, and S^gamma -> d_2^2 as gamma -> 0."""
    d = 16
    b, t, o = inputs.random_diagrams(2, nmin=6, nmax=9, seed=seed, log_uniform=False)
    hist, mass = oracle.rasterize(b, t, o, d)
    X = _snapped_points(b[o[0]:o[1]], t[o[0]:o[1]], d)
    Y = _snapped_points(b[o[1]:o[2]], t[o[1]:o[2]], d)
    L, _ = _diag_matching_sq(X, Y)
    n = int(mass.sum())
    prev = None
    for gamma in (1e-2, 3e-3, 1e-3, 3e-4):
        r = oracle.sinkhorn_pd(d, gamma, hist[0], hist[1], 200000, 1e-11)
        bound = 2 * gamma * n * math.log(n) + r["err"] * n * 2.0
        assert -r["err"] * n * 2.0 - 1e-12 <= r["cost"] - L <= bound
        if prev is not None:
            assert abs(r["cost"] - L) <= abs(prev - L) + 1e-9
        prev = r["cost"]
    assert abs(prev - L) <= 2e-3 * max(L, 1e-3) + 1e-5


def test_grid_refinement_bound():
    """Supplementary 'Error control due to discretization', with the l2 move of
    a snapped point bounded by sqrt(2)/d (the paper states 1/d per point, the
    l_inf move): |d_2(D_A,D_B) - L^(1/2)| <= sqrt(2)/d (sqrt nA + sqrt nB)."""
    b, t, o = inputs.random_diagrams(2, nmin=12, nmax=12, seed=9)
    X0 = np.stack([b[o[0]:o[1]], t[o[0]:o[1]]], 1)
    Y0 = np.stack([b[o[1]:o[2]], t[o[1]:o[2]]], 1)
    dtrue = math.sqrt(_diag_matching_sq(X0, Y0)[0])
    for d in (8, 16, 32, 64, 128, 256):
        hist, mass = oracle.rasterize(b, t, o, d)
        X = _snapped_points(X0[:, 0], X0[:, 1], d)
        Y = _snapped_points(Y0[:, 0], Y0[:, 1], d)
        Lg = math.sqrt(_diag_matching_sq(X, Y)[0])
        assert abs(dtrue - Lg) <= math.sqrt(2) / d * (math.sqrt(len(X)) + math.sqrt(len(Y))) + 1e-12


# --------------------------------------------------------------------------- invariants
def test_marginals_symmetry_positivity():
    d, gamma = 32, 1e-2
    b, t, o = inputs.random_diagrams(2, nmin=20, nmax=20, seed=0)
    hist, mass = oracle.rasterize(b, t, o, d)
    r = oracle.sinkhorn_pd(d, gamma, hist[0], hist[1], 20000, 1e-13)
    a, bb = oracle.augment(hist[0], hist[1])
    assert np.allclose(r["cmarg"], bb, rtol=1e-11, atol=1e-11)     # column side exact after v-update
    assert np.abs(r["rmarg"] - a).sum() / a.sum() < 1e-11
    assert r["cost"] > 0
    rs = oracle.sinkhorn_pd(d, gamma, hist[1], hist[0], 20000, 1e-13)
    assert rs["cost"] == pytest.approx(r["cost"], rel=1e-9)
    # dual potentials: P = a b exp((f+g-C)/gamma) reproduces the marginals
    sa = np.nonzero(a)[0]
    sb = np.nonzero(bb)[0]
    C = np.array([[oracle.cost(d, x, y) for y in sb] for x in sa])
    P = a[sa, None] * bb[None, sb] * np.exp((r["f"][sa, None] + r["g"][None, sb] - C) / gamma)
    assert np.allclose(P.sum(0), bb[sb], rtol=1e-10)
    assert float((P * C).sum()) == pytest.approx(r["cost"], rel=1e-12)


def test_self_distance_vanishes():
    """S^gamma(a, a) -> 0 as gamma -> 0 (d_2(D, D) = 0), within 2 gamma n log n."""
    d = 32
    b, t, o = inputs.random_diagrams(1, nmin=15, nmax=15, seed=4)
    h, m = oracle.rasterize(b, t, o, d)
    n = 2 * int(m[0])
    for gamma in (1e-2, 1e-3):
        r = oracle.sinkhorn_pd(d, gamma, h[0], h[0], 100000, 1e-12)
        assert 0 <= r["cost"] <= 2 * gamma * n * math.log(n)


def test_fixed_iteration_count_and_warm_start():
    """max_iter is honoured exactly, and a warm start from the converged g
    reproduces the converged cost within one iteration."""
    d, gamma = 32, 1e-2
    b, t, o = inputs.random_diagrams(2, nmin=20, nmax=20, seed=0)
    hist, _ = oracle.rasterize(b, t, o, d)
    r300 = oracle.sinkhorn_pd(d, gamma, hist[0], hist[1], 300, 0.0)
    assert r300["iters"] == 300
    rc = oracle.sinkhorn_pd(d, gamma, hist[0], hist[1], 100000, 1e-13)
    rw = oracle.sinkhorn_pd(d, gamma, hist[0], hist[1], 1, 0.0, g_init=rc["g"])
    assert rw["cost"] == pytest.approx(rc["cost"], rel=1e-10)


# --------------------------------------------------------------------------- barycenter
def _reg_value(d, gamma, a, bb, r):
    """Dual value of Eq. (SinkhornDual) at the converged potentials:
    L^gamma = <f + gamma log a, a> + <g + gamma log b, b> - gamma * sum(P),
    with sum(P) = total mass."""
    ma = a > 0
    mb = bb > 0
    return (float((a[ma] * (r["f"][ma] + gamma * np.log(a[ma]))).sum())
            + float((bb[mb] * (r["g"][mb] + gamma * np.log(bb[mb]))).sum()) - gamma * a.sum())


def test_barycenter_gradient_finite_differences():
    """Prop. (gradient of E^gamma): d/dz_x L^gamma(z + R a, a + R z) =
    gamma log u(x) + gamma log v(Delta), checked by central differences of the
    regularised value; then one outer step of the oracle's Alg. 2 equals
    z * exp(-lambda * mean gradient)."""
    d, gamma = 8, 5e-2
    b, t, o = inputs.random_diagrams(2, nmin=5, nmax=5, seed=21)
    hist, _ = oracle.rasterize(b, t, o, d)
    D = d * d
    z0 = np.zeros(D)
    ii, jj = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    up = (jj >= ii).ravel()
    z0[up] = 5.0 / up.sum() * (1 + 0.3 * np.sin(np.arange(up.sum())))

    def val(z, hi):
        a = np.concatenate([z, [float(hi.sum())]])
        bb = np.concatenate([hi.ravel().astype(float), [z.sum()]])
        r = oracle.sinkhorn_w(d, gamma, a, bb, 200000, 1e-14)
        return _reg_value(d, gamma, a, bb, r), r

    grads = []
    for hi in hist:
        _, r = val(z0, hi)
        g_an = gamma * np.log(np.where(z0 > 0, z0, 1)) + r["f"][:D] + gamma * math.log(z0.sum()) + r["g"][D]
        for x in np.nonzero(up)[0][::7]:
            h = 1e-5 * z0[x]
            zp = z0.copy(); zp[x] += h
            zm = z0.copy(); zm[x] -= h
            fd = (val(zp, hi)[0] - val(zm, hi)[0]) / (2 * h)
            assert fd == pytest.approx(g_an[x], rel=1e-5, abs=1e-7)
        grads.append(g_an)
    lam = 2.0
    z1, _ = oracle.barycenter(d, gamma, hist, lam, 1, 200000, 1e-14, z_init=z0.reshape(d, d))
    expect = np.where(up, z0 * np.exp(-lam * np.mean(grads, 0)), 0.0)
    assert np.allclose(z1.ravel(), expect, rtol=1e-8, atol=1e-14)


def test_barycenter_regularised_energy_decreases():
    """Alg. 2 is mirror descent on the convex energy E^gamma (supplementary
    'Convexity of E'): along the multiplicative updates the regularised energy
    sum_i L^gamma(z + R a_i, a_i + R z) decreases."""
    d, gamma, lam = 10, 1e-2, 2.0
    b, t, o = inputs.random_diagrams(3, nmin=5, nmax=7, seed=8, log_uniform=False)
    hist, _ = oracle.rasterize(b, t, o, d)
    D = d * d
    z = None
    vals = []
    for step in range(6):
        z, _ = oracle.barycenter(d, gamma, hist, lam, 1, 200000, 1e-12, z_init=z)
        zf = z.ravel()
        tot = 0.0
        for hi in hist:
            a = np.concatenate([zf, [float(hi.sum())]])
            bb = np.concatenate([hi.ravel().astype(float), [zf.sum()]])
            r = oracle.sinkhorn_w(d, gamma, a, bb, 200000, 1e-12)
            tot += _reg_value(d, gamma, a, bb, r)
        vals.append(tot)
    assert np.all(np.diff(vals) < 0), vals


def test_barycenter_identical_diagrams_concentrate():
    """N copies of one diagram D: the unregularised barycenter is D itself
    (energy 0).  As gamma decreases, Alg. 2's transport energy falls and the
    share of the barycenter's mass at or next to D's cells grows."""
    d = 16
    b, t, o = inputs.random_diagrams(1, nmin=6, nmax=6, seed=2)
    h, m = oracle.rasterize(b, t, o, d)
    hists = np.repeat(h, 3, axis=0)
    near = np.zeros((d, d), bool)
    for (i, j) in zip(*np.nonzero(h[0])):
        near[max(i - 1, 0):i + 2, max(j - 1, 0):j + 2] = True
    energies, shares = [], []
    for gamma in (1e-2, 3e-3, 1e-3):
        z, e = oracle.barycenter(d, gamma, hists, 5.0, 60, 20000, 1e-6)
        energies.append(e[-1])
        shares.append(z[near].sum() / z.sum())
    assert energies[0] > energies[1] > energies[2]
    assert shares[0] < shares[1] < shares[2]
    assert energies[-1] < 0.1 * energies[0]


# --------------------------------------------------------------------------- k-means
def test_kmeans_best_run_recovers_modes():
    """Sec. 5 k-means (Lloyd with Alg. 1 assignment and Alg. 2 centroids) is
    non-convex, so single runs depend on the seeding; over several seeds the
    run with the lowest objective is the generating partition (up to
    relabelling) of well-separated synthetic modes."""
    d, gamma = 16, 5e-3
    b, t, o, lab = inputs.mode_diagrams(12, 3, 40, 60, sigma=0.02, seed=5)
    hist, _ = oracle.rasterize(b, t, o, d)
    runs = []
    for seed in range(8):
        assign, cent, obj = oracle.kmeans(d, gamma, hist, 3, 5.0, 4, 3, 5000, 1e-4, seed)
        runs.append((obj[-1], assign))
    best = min(runs, key=lambda r: r[0])[1]
    pairs = set(zip(lab.tolist(), best.tolist()))
    assert len(pairs) == 3 and len({p[1] for p in pairs}) == 3


def test_kmeans_objective_non_increasing_over_rounds():
    """Lloyd's alternation: the assignment takes the minimum over centroids and
    the centroid update (Alg. 2 steps on each cluster) lowers each cluster's
    energy when the mirror-descent step is small enough, so on well-separated
    modes the objective sum_n min_c <P, C> does not rise from round to round (a
    sign error in the update or an argmax in the assignment makes it rise).
    With lambda = 0.3 the update is in that regime (lambda = 5, the paper's
    barycenter step, overshoots from centroids seeded on single diagrams and the
    objective can rise: measured 6.77 -> 9.11 on this data)."""
    d, gamma = 16, 5e-3
    b, t, o, lab = inputs.mode_diagrams(12, 3, 40, 60, sigma=0.02, seed=5)
    hist, _ = oracle.rasterize(b, t, o, d)
    for seed in (0, 3):
        _, _, obj = oracle.kmeans(d, gamma, hist, 3, 0.3, 5, 3, 5000, 1e-6, seed)
        assert np.all(np.diff(obj) <= 1e-9 * obj[:-1]), obj
        assert obj[-1] < 0.97 * obj[0]


def test_kmeans_tie_goes_to_lowest_index_and_empty_cluster_keeps_centroid():
    """Two identical diagrams and k = 2: seeding takes both, so the two
    centroids are equal and every assignment is a tie.  The reading of Sec. 5
    fixes ties to the lowest centroid index, so both diagrams join centroid 0;
    centroid 1 is then empty and keeps its value (the seeded histogram)
    exactly, while centroid 0 moves by its Alg. 2 steps."""
    d, gamma = 12, 1e-2
    b, t, o = inputs.random_diagrams(1, nmin=7, nmax=7, seed=4)
    h, _ = oracle.rasterize(b, t, o, d)
    hists = np.repeat(h, 2, axis=0)
    assign, cent, obj = oracle.kmeans(d, gamma, hists, 2, 2.0, 1, 2, 5000, 1e-9, 0)
    assert assign.tolist() == [0, 0]
    assert np.array_equal(cent[1], h[0].astype(np.float64))
    assert not np.allclose(cent[0], h[0].astype(np.float64))


def test_barycenter_energy_stop_rule():
    """The barycenter experiment's stop (Sec. 5, Fig. 5): after step t >= 1,
    stop when |E_t / E_{t-1} - 1| < tol.  From the energies of a fixed-length
    run, the stopped run must end at the first such t, with the energies and
    the measure of a fixed run of t + 1 steps; tol = 0 runs every step."""
    d, gamma, lam = 10, 1e-2, 2.0
    b, t, o = inputs.random_diagrams(3, nmin=5, nmax=7, seed=8, log_uniform=False)
    hist, _ = oracle.rasterize(b, t, o, d)
    T = 8
    z_all, e_all = oracle.barycenter(d, gamma, hist, lam, T, 20000, 1e-10)
    assert len(e_all) == T
    ratios = np.abs(e_all[1:] / e_all[:-1] - 1.0)
    tol = float(np.sort(ratios)[len(ratios) // 2]) * 1.0001   # stops somewhere inside the run
    t_stop = 1 + int(np.nonzero(ratios < tol)[0][0])
    z_s, e_s = oracle.barycenter(d, gamma, hist, lam, T, 20000, 1e-10, rel_energy_tol=tol)
    assert len(e_s) == t_stop + 1 < T
    z_ref, e_ref = oracle.barycenter(d, gamma, hist, lam, t_stop + 1, 20000, 1e-10)
    assert np.array_equal(e_s, e_ref) and np.array_equal(e_s, e_all[:t_stop + 1])
    assert np.array_equal(z_s, z_ref)
    z0, e0 = oracle.barycenter(d, gamma, hist, lam, T, 20000, 1e-10, rel_energy_tol=0.0)
    assert len(e0) == T and np.array_equal(z0, z_all)


# --------------------------------------------------------------------------- Prop. 3 rounding upper bound
@pytest.mark.parametrize("T", [2, 10, 60, None])
def test_round_bound_plan_is_feasible_and_closes(T):
    """The rounded plan R has the marginals (a, b) exactly at any iterate, and
    once the iterates converge the correction vanishes: <R, C> -> <P, C>."""
    d, gamma = 16, 1e-2
    b, t, o = inputs.random_diagrams(2, nmin=12, nmax=12, seed=7)
    h, _ = oracle.rasterize(b, t, o, d)
    a, bb = oracle.augment(h[0], h[1])
    r = oracle.sinkhorn_w(d, gamma, a, bb, T, 0.0) if T else oracle.sinkhorn_w(d, gamma, a, bb, 200000, 1e-13)
    rb = oracle.round_bound(d, gamma, a, bb, r["f"], r["g"])
    assert rb["row_dev"] <= 1e-12 * a.sum() and rb["col_dev"] <= 1e-12 * a.sum()
    assert rb["er"] >= -1e-12 and rb["ec"] >= -1e-12
    assert abs(rb["er"] - rb["ec"]) <= 1e-10 * a.sum()        # both sides lose the same mass
    if T is None:   # converged (marginal error 1e-13)
        assert rb["ec"] <= 1e-9 * a.sum()
        assert rb["upper"] == pytest.approx(r["cost"], rel=1e-9)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_round_bound_is_above_exact_transport(seed):
    """R is a feasible transport plan, so <R, C> >= the exact optimal cost,
    which for rasterised diagrams is d_2^2 of the snapped points (Prop. 1),
    computed here by assignment; at early iterates the plan P itself can be far
    below it (not feasible), the rounded one never is."""
    d = 16
    b, t, o = inputs.random_diagrams(2, nmin=6, nmax=9, seed=seed, log_uniform=False)
    h, _ = oracle.rasterize(b, t, o, d)
    X = _snapped_points(b[o[0]:o[1]], t[o[0]:o[1]], d)
    Y = _snapped_points(b[o[1]:o[2]], t[o[1]:o[2]], d)
    L, _ = _diag_matching_sq(X, Y)
    a, bb = oracle.augment(h[0], h[1])
    below = 0
    for gamma in (1e-2, 1e-3):
        for T in (1, 3, 20, 400):
            r = oracle.sinkhorn_w(d, gamma, a, bb, T, 0.0)
            rb = oracle.round_bound(d, gamma, a, bb, r["f"], r["g"])
            assert rb["upper"] >= L - 1e-12, (gamma, T, rb["upper"], L)
            below += r["cost"] < L - 1e-9
    assert below > 0   # the check has teeth: some unrounded plans undercut the optimum


# --------------------------------------------------------------------------- C-transform lower bound m_t
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ctransform_bound_below_exact_transport(seed):
    """Sec. 3 "Upper and Lower Bounds": m_t <= L_C(a, b) <= M_t at every
    iterate (weak duality below, feasibility of the rounded plan above), with
    L_C = d_2^2 of the snapped points from an assignment solver (Prop. 1), and
    both bounds close in on L_C as gamma -> 0 and the iterates converge."""
    d = 16
    b, t, o = inputs.random_diagrams(2, nmin=6, nmax=9, seed=seed, log_uniform=False)
    h, _ = oracle.rasterize(b, t, o, d)
    X = _snapped_points(b[o[0]:o[1]], t[o[0]:o[1]], d)
    Y = _snapped_points(b[o[1]:o[2]], t[o[1]:o[2]], d)
    L, _ = _diag_matching_sq(X, Y)
    a, bb = oracle.augment(h[0], h[1])
    for gamma in (1e-2, 1e-3, 2e-4):
        for T in (1, 5, 50, 2000):
            r = oracle.sinkhorn_w(d, gamma, a, bb, T, 0.0)
            m = oracle.ctransform_bound(d, gamma, a, bb, r["f"])
            M = oracle.round_bound(d, gamma, a, bb, r["f"], r["g"])["upper"]
            assert m <= L + 1e-12 <= M + 2e-12, (gamma, T, m, L, M)
    r = oracle.sinkhorn_w(d, 2e-4, a, bb, 400000, 1e-12)
    m = oracle.ctransform_bound(d, 2e-4, a, bb, r["f"])
    assert L - m <= 1e-3 * max(L, 1e-3)


def test_ctransform_bound_exact_on_a_single_point():
    """One point against the empty diagram: the only feasible plan sends the
    point to the diagonal, and with any alpha the transforms give exactly its
    cost (alpha^c(Delta) = cD - alpha, alpha^cc = cD - alpha^c = alpha)."""
    d = 16
    h = np.zeros((2, d, d), np.uint32)
    h[0, 3, 9] = 1
    a, bb = oracle.augment(h[0], h[1])
    f = np.random.default_rng(0).normal(size=d * d + 1)
    m = oracle.ctransform_bound(d, 1e-2, a, bb, f)
    assert m == pytest.approx((9 - 3) ** 2 / (2 * d * d), rel=1e-12)


# --------------------------------------------------------------------------- ground cost ||.||_p^p (NEXT-3)
@pytest.mark.parametrize("p", [1.0, 1.5, 3.0])
def test_cost_p_matches_geometry(p):
    """||.||_p^p between cell corners, and the diagonal cost ||x - pi(x)||_p^p
    with pi the orthogonal projection onto the diagonal."""
    d = 16
    for (i, j, k, l) in [(3, 9, 5, 12), (0, 15, 15, 15), (7, 7, 2, 11)]:
        x, y = i * d + j, k * d + l
        assert oracle.cost(d, x, y, p) == pytest.approx(abs(i - k) ** p / d ** p + abs(j - l) ** p / d ** p, rel=1e-14)
        s, t = i / d, j / d
        m = (s + t) / 2
        assert oracle.cost(d, x, d * d, p) == pytest.approx(abs(s - m) ** p + abs(t - m) ** p, rel=1e-12)
        assert oracle.cost(d, d * d, x, p) == oracle.cost(d, x, d * d, p)
    assert oracle.cost(d, d * d, d * d, p) == 0.0


@pytest.mark.parametrize("p", [1.0, 1.5])
def test_p_empty_diagram_and_two_cells_closed_forms(p):
    """Closed forms hold for any ground cost: against an empty diagram the plan
    is forced (S = sum_x a_x C(x, Delta)), and one cell against one cell is the
    2x2 problem of the p = 2 pin with the ||.||_p^p entries."""
    d, gamma = 16, 1e-2
    h = np.zeros((2, d, d), np.uint32)
    h[0, 3, 9] = 2
    h[0, 1, 4] = 1
    r = oracle.sinkhorn_pd(d, gamma, h[0], h[1], 50, 0.0, p=p)
    expect = 2 * oracle.cost(d, 3 * d + 9, d * d, p) + oracle.cost(d, 1 * d + 4, d * d, p)
    assert r["cost"] == pytest.approx(expect, rel=1e-12)
    h = np.zeros((2, d, d), np.uint32)
    h[0, 3, 9] = 1
    h[1, 5, 12] = 1
    gamma = 0.2     # well-conditioned 2x2 problem (|D|/gamma of order 1)
    r = oracle.sinkhorn_pd(d, gamma, h[0], h[1], 100000, 1e-14, p=p)
    Cxy = oracle.cost(d, 3 * d + 9, 5 * d + 12, p)
    CxD = oracle.cost(d, 3 * d + 9, d * d, p)
    CyD = oracle.cost(d, 5 * d + 12, d * d, p)
    assert r["cost"] == pytest.approx(_two_by_two(1, 1, Cxy, CxD, CyD, gamma), rel=1e-9)


def test_p1_gamma_to_zero_matches_assignment():
    """p = 1: as gamma -> 0 the cost tends to the optimal partial matching with
    ||.||_1 costs (point to point sum of |db| + |dt|, point to diagonal
    |t - s|, i.e. 2 |(t-s)/2|), by assignment on the augmented matrix."""
    from scipy.optimize import linear_sum_assignment
    d = 16
    b, t, o = inputs.random_diagrams(2, nmin=6, nmax=8, seed=4, log_uniform=False)
    h, _ = oracle.rasterize(b, t, o, d)
    X = _snapped_points(b[o[0]:o[1]], t[o[0]:o[1]], d)
    Y = _snapped_points(b[o[1]:o[2]], t[o[1]:o[2]], d)
    nX, nY = len(X), len(Y)
    M = np.zeros((nX + nY, nX + nY))
    M[:nX, :nY] = np.abs(X[:, None, :] - Y[None, :, :]).sum(-1)
    M[:nX, nY:] = np.abs(X[:, 1] - X[:, 0])[:, None]
    M[nX:, :nY] = np.abs(Y[:, 1] - Y[:, 0])[None, :]
    r_, c_ = linear_sum_assignment(M)
    L = M[r_, c_].sum()
    n = int(h.sum())
    for gamma in (1e-2, 1e-3, 2e-4):
        r = oracle.sinkhorn_pd(d, gamma, h[0], h[1], 400000, 1e-12, p=1.0)
        assert -1e-9 <= r["cost"] - L <= 2 * gamma * n * math.log(n) + 1e-9
    assert abs(r["cost"] - L) <= 5e-3 * max(L, 1e-3)


# --------------------------------------------------------------------------- entropic sharpening (NEXT-2)
def _entropy(w):
    w = np.asarray(w, dtype=np.float64).ravel()
    w = w[w > 0] / w.sum()
    return float(-(w * np.log(w)).sum())


def test_sharpen_hits_target_entropy_as_a_power():
    """Sharpening replaces z by |z| w^beta / sum w^beta (w = z/|z|): the result
    has the target entropy and the same mass and support, and it is a power of
    z (log z'_x - log z'_y = beta (log z_x - log z_y) for every pair of cells)."""
    d = 16
    rng = np.random.default_rng(0)
    z = np.zeros((d, d))
    iu = np.triu_indices(d)
    z[iu] = rng.random(len(iu[0])) + 0.05
    H = _entropy(z)
    H0 = H - 0.7
    zs, beta = oracle.sharpen(d, z, H0)
    assert beta > 1.0
    assert _entropy(zs) == pytest.approx(H0, abs=1e-10)
    assert zs.sum() == pytest.approx(z.sum(), rel=1e-12)
    assert np.array_equal(zs > 0, z > 0)
    lz, lzs = np.log(z[iu]), np.log(zs[iu])
    assert np.allclose(lzs - lzs[0], beta * (lz - lz[0]), atol=1e-9)
    # already below the target: unchanged
    z2, b2 = oracle.sharpen(d, z, H + 0.1)
    assert b2 == 1.0 and np.array_equal(z2, z)


def test_sharpen_large_beta_reaches_target():
    """A nearly uniform measure sharpened far below its entropy needs a large
    beta (here > 100): the result still has exactly the target entropy, i.e.
    the powers do not underflow on the way."""
    d = 32
    rng = np.random.default_rng(1)
    z = np.zeros((d, d))
    iu = np.triu_indices(d)
    z[iu] = 0.014 + 0.038 * rng.random(len(iu[0]))
    H0 = 2.97
    zs, beta = oracle.sharpen(d, z, H0)
    assert beta > 50
    assert _entropy(zs) == pytest.approx(H0, abs=1e-9)
    assert zs.sum() == pytest.approx(z.sum(), rel=1e-12)


def test_sharpened_barycenter_entropy_bounded_and_energy_close():
    """Alg. 2 with sharpening after every step: z's entropy never exceeds the
    largest input entropy, while the plain barycenter's does (smearing), and the
    sharpened barycenter is more concentrated (larger largest cell share)."""
    d, gamma = 16, 1e-2
    b, t, o, _ = inputs.mode_diagrams(4, 1, 20, 30, sigma=0.04, seed=3)
    h, _ = oracle.rasterize(b, t, o, d)
    H0 = max(_entropy(x) for x in h)
    z0, _ = oracle.barycenter(d, gamma, h, 2.0, 6, 300, 0.0)
    zs, _ = oracle.barycenter(d, gamma, h, 2.0, 6, 300, 0.0, sharpen=True)
    assert _entropy(z0) > H0
    assert _entropy(zs) <= H0 + 1e-9
    assert (zs / zs.sum()).max() > (z0 / z0.sum()).max()
