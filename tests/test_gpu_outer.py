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


def test_outer_loop_takes_the_separable_form_where_records_cost_occupancy(ctx):
    """Alg. 2 at d = 64: the barycenter side is dense (2080 cells), and with
    the pairwise records the largest pair's shared memory leaves one CTA per
    SM instead of two, so the automatic form runs the whole call separable:
    bit for bit lse_form = 1, and the oracle's barycenter (same fixed inner
    iterations).  At d = 32 the records cost no CTA per SM and the automatic
    forms stay (the result differs from form 1 in its rounding)."""
    d, gamma, lam, steps, T = 64, 5e-3, 5.0, 2, 150
    b, t, o = inputs.random_diagrams(4, nmin=200, nmax=300, exp_mean=0.2, seed=64, log_uniform=False)
    h, _ = oracle.rasterize(b, t, o, d)
    hist, mass = hists_to_gpu(h), dev(masses(h).view(np.int32))
    z0, e0 = api.pd_barycenter(ctx, hist, mass, api.pd_sinkhorn_default_params(gamma, d, max_iter=T, tol=0.0), lam,
                               steps)
    z1, e1 = api.pd_barycenter(ctx, hist, mass, api.pd_sinkhorn_default_params(gamma, d, max_iter=T, tol=0.0,
                                                                               lse_form=1), lam, steps)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1) and torch.equal(e0, e1)
    z_ref, e_ref = oracle.barycenter(d, gamma, h, lam, steps, T, 0.0)
    z, e = z0.cpu().numpy(), e0.cpu().numpy()
    assert np.allclose(e, e_ref, rtol=1e-6, atol=0)
    assert np.allclose(z, z_ref, rtol=1e-5, atol=1e-9 * z_ref.max())
    d = 32
    b, t, o = inputs.random_diagrams(4, nmin=10, nmax=60, seed=32)
    h, _ = oracle.rasterize(b, t, o, d)
    hist, mass = hists_to_gpu(h), dev(masses(h).view(np.int32))
    z0, _ = api.pd_barycenter(ctx, hist, mass, api.pd_sinkhorn_default_params(gamma, d, max_iter=T, tol=0.0), lam,
                              steps)
    z1, _ = api.pd_barycenter(ctx, hist, mass, api.pd_sinkhorn_default_params(gamma, d, max_iter=T, tol=0.0,
                                                                              lse_form=1), lam, steps)
    assert not torch.equal(z0, z1)


def test_barycenter_energy_stop_matches_oracle(ctx):
    """The barycenter experiment's stop |E_t/E_{t-1} - 1| < tol (Sec. 5):
    the GPU run stops at the same step as the oracle's, with the same energies
    and measure.  tol is placed halfway (geometrically) between two well
    separated ratios of a fixed-length oracle run, so the rounding of the two
    sides cannot move the stop."""
    d, gamma, lam, T = 16, 1e-2, 2.0, 200
    b, t, o = inputs.random_diagrams(4, nmin=8, nmax=25, seed=11, log_uniform=False)
    h, _ = oracle.rasterize(b, t, o, d)
    steps = 10
    _, e_all = oracle.barycenter(d, gamma, h, lam, steps, T, 0.0)
    ratios = np.abs(e_all[1:] / e_all[:-1] - 1.0)
    order = np.sort(ratios)
    gaps = order[1:] / np.maximum(order[:-1], 1e-300)
    q = int(np.argmax(gaps))                      # the widest gap between two ratios
    tol = float(np.sqrt(order[q] * order[q + 1]))
    # the two sides' energies agree to ~1e-6 relative, i.e. the ratios to a few
    # 1e-6 absolute: a 10 % gap keeps both sides on the same side of tol
    assert gaps[q] > 1.1 and order[q + 1] - order[q] > 1e-4
    z_ref, e_ref = oracle.barycenter(d, gamma, h, lam, steps, T, 0.0, rel_energy_tol=tol)
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=T, tol=0.0)
    z, e = api.pd_barycenter(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, lam, steps, rel_energy_tol=tol)
    torch.cuda.synchronize()
    assert len(e) == len(e_ref) < steps
    assert np.allclose(e.cpu().numpy(), e_ref, rtol=1e-6, atol=0)
    assert np.allclose(z.cpu().numpy(), z_ref, rtol=1e-5, atol=1e-9 * z_ref.max())


def test_caller_workspace_of_the_queried_size(ctx):
    """pd_workspace_query gives the bytes a call needs; a context given exactly
    that much caller-owned memory (pd_ctx_set_workspace) allocates nothing and
    returns the same results bitwise as a library-allocated context, and 256
    bytes less is refused with PD_ERR_OOM."""
    d, gamma = 32, 5e-3
    b, t, o = inputs.random_diagrams(6, nmin=20, nmax=60, seed=12)
    h, _ = oracle.rasterize(b, t, o, d)
    hist, mass = hists_to_gpu(h), dev(masses(h).view(np.int32))
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=400, tol=1e-6)
    ref = api.pd_sinkhorn_batch(ctx, hist[:3], mass[:3], hist[3:], mass[3:], p)
    zr, er = api.pd_barycenter(ctx, hist, mass, p, 2.0, 3)
    need_s = api.pd_workspace_query(api.PD_OP_SINKHORN, p, 3)
    need_b = api.pd_workspace_query(api.PD_OP_BARYCENTER, p, 6)
    assert need_s > 0 and need_b > need_s
    c2 = api.Context(0)
    try:
        for need, run in ((need_s, lambda: api.pd_sinkhorn_batch(c2, hist[:3], mass[:3], hist[3:], mass[3:], p)),
                          (need_b, lambda: api.pd_barycenter(c2, hist, mass, p, 2.0, 3))):
            buf = torch.empty(need, dtype=torch.uint8, device="cuda")
            api.pd_ctx_set_workspace(c2, buf, need)
            out = run()
            torch.cuda.synchronize()
            if isinstance(out, dict):
                assert np.array_equal(out["cost"].cpu().numpy(), ref["cost"].cpu().numpy())
                assert np.array_equal(out["iters"].cpu().numpy(), ref["iters"].cpu().numpy())
            else:
                assert np.array_equal(out[0].cpu().numpy(), zr.cpu().numpy())
                assert np.array_equal(out[1].cpu().numpy(), er.cpu().numpy())
            api.pd_ctx_set_workspace(c2, buf, need - 256)
            with pytest.raises(api.PdError) as ex:
                run()
            assert ex.value.status == api.PD_ERR_OOM
            api.pd_ctx_set_workspace(c2, None)
            del buf
    finally:
        c2.close()


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
    # the split step and the assignment: bad sizes and parameters are refused
    z = torch.zeros((1, 8, 8), dtype=torch.float64, device="cuda")
    gs = torch.zeros((1, 64), dtype=torch.float64, device="cuda")
    cnt = torch.ones(1, dtype=torch.float64, device="cuda")
    for gamma, lam in ((0.0, 1.0), (1e-2, 0.0), (1e-2, -1.0)):
        with pytest.raises(api.PdError) as e:
            api.pd_barycenter_apply(ctx, z, gs, cnt, gamma, lam)
        assert e.value.status == api.PD_ERR_INVALID
    with pytest.raises(api.PdError):
        api.pd_barycenter_grad(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, z, 0)     # k = 0
    a, obj, _ = api.pd_kmeans_assign(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, z[:1] + 1.0)
    torch.cuda.synchronize()
    assert a.cpu().tolist() == [0, 0] and np.isfinite(obj.item())


def test_sharded_step_one_shard_is_pd_barycenter_bitwise(ctx):
    """pd_barycenter_grad + pd_barycenter_apply with one shard: bitwise the
    z of pd_barycenter (same solves, same sums in the same order), from a
    given start and from the default start; energies to the rounding of the
    mean."""
    from paper_1805_08331_gb300 import sharded
    d, gamma, lam, steps = 32, 5e-3, 5.0, 4
    b, t, o = inputs.random_diagrams(6, nmin=10, nmax=60, seed=11)
    h, _ = oracle.rasterize(b, t, o, d)
    hist, mass = hists_to_gpu(h), dev(masses(h).view(np.int32))
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=3000, tol=1e-6)
    for z_init in (None, torch.from_numpy(np.triu(np.full((d, d), 0.05))).cuda()):
        z_ref, e_ref = api.pd_barycenter(ctx, hist, mass, p, lam, steps, z_init=z_init)
        z, e = sharded.barycenter_sharded(ctx, hist, mass, p, lam, steps, z_init=z_init)
        torch.cuda.synchronize()
        assert torch.equal(z, z_ref)
        assert np.allclose(e.cpu().numpy(), e_ref.cpu().numpy(), rtol=1e-13, atol=0)


def test_sharded_step_two_shards_match_one_gpu(ctx):
    """The exchange of the sharded step emulated on one GPU: the diagrams in two
    shards, each with its own pd_barycenter_grad and warm potentials, the two
    sums added (the all-reduce), one pd_barycenter_apply.  Each pair's solve is
    the same in either batch (at d = 32 no call switches to the separable form
    for occupancy), so z only differs from pd_barycenter by the rounding of
    adding two partial sums."""
    d, gamma, lam, steps = 32, 5e-3, 5.0, 4
    b, t, o = inputs.random_diagrams(7, nmin=10, nmax=60, seed=12)
    h, _ = oracle.rasterize(b, t, o, d)
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=3000, tol=1e-6)
    z0 = torch.from_numpy(np.triu(np.full((d, d), 0.05))).cuda()
    z_ref, e_ref = api.pd_barycenter(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, lam, steps, z_init=z0)
    shards = [h[:3], h[3:]]
    hs = [(hists_to_gpu(x), dev(masses(x).view(np.int32))) for x in shards]
    gw = [torch.empty((len(x), d * d + 1), dtype=torch.float64, device="cuda") for x in shards]
    z = z0.clone()
    e = []
    for step in range(steps):
        parts = [api.pd_barycenter_grad(ctx, hh, mm, p, z, 1, None, g, step > 0) for (hh, mm), g in zip(hs, gw)]
        gsum = parts[0][0] + parts[1][0]
        count = parts[0][1] + parts[1][1]
        csum = parts[0][2] + parts[1][2]
        assert count.item() == len(h)
        api.pd_barycenter_apply(ctx, z, gsum, count, gamma, lam)
        e.append((csum / count).item())
    torch.cuda.synchronize()
    assert torch.allclose(z, z_ref, rtol=1e-9, atol=1e-12 * z_ref.max().item())
    assert np.allclose(e, e_ref.cpu().numpy(), rtol=1e-9, atol=0)


def test_sharded_step_k_measures_with_owner(ctx):
    """k = 2 measures, owner per diagram: the per-measure sums equal the
    one-measure sums over each measure's own diagrams."""
    d, gamma = 16, 1e-2
    b, t, o = inputs.random_diagrams(5, nmin=8, nmax=30, seed=13)
    h, _ = oracle.rasterize(b, t, o, d)
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=2000, tol=1e-6)
    z = torch.from_numpy(np.stack([np.triu(np.full((d, d), 0.1)), np.triu(np.full((d, d), 0.2))])).cuda()
    owner = torch.tensor([1, 0, 1, 1, 0], dtype=torch.int32, device="cuda")
    gsum, count, csum = api.pd_barycenter_grad(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, z, 2, owner)
    assert count.cpu().tolist() == [2.0, 3.0]
    for c in range(2):
        idx = [n for n in range(5) if owner[n].item() == c]
        hc = h[idx]
        g1, n1, s1 = api.pd_barycenter_grad(ctx, hists_to_gpu(hc), dev(masses(hc).view(np.int32)), p, z[c], 1)
        assert n1.item() == len(idx)
        assert torch.equal(gsum[c], g1[0]) and torch.equal(csum[c], s1[0])
    with pytest.raises(api.PdError):
        api.pd_barycenter_grad(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)),
                               api.pd_sinkhorn_default_params(gamma, d, bary_sharpen=1), z, 2, owner)
    for bad in (2, -1):                                    # owner outside [0, k): refused, nothing solved
        ob = owner.clone()
        ob[3] = bad
        with pytest.raises(api.PdError) as e:
            api.pd_barycenter_grad(ctx, hists_to_gpu(h), dev(masses(h).view(np.int32)), p, z, 2, ob)
        assert e.value.status == api.PD_ERR_INVALID


def test_kmeans_assign_matches_pd_kmeans_costs(ctx):
    """pd_kmeans_assign against the seeded centroids: argmin of the costs it
    returns (lowest index on ties), objective = sum of the minima, and the
    costs equal those of pd_sinkhorn_batch-style solves of the same pairs
    through pd_kmeans' first assignment (same objective)."""
    d, gamma = 16, 5e-3
    b, t, o, _ = inputs.mode_diagrams(12, 3, 40, 60, sigma=0.02, seed=5)
    h, _ = oracle.rasterize(b, t, o, d)
    hist, mass = hists_to_gpu(h), dev(masses(h).view(np.int32))
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=300, tol=0.0)
    _, c0, _ = api.pd_kmeans(ctx, hist, mass, 3, p, 5.0, 0, 2, seed=2)        # seeding only
    a, obj, cost = api.pd_kmeans_assign(ctx, hist, mass, p, c0, want_cost=True)
    _, _, obj_k = api.pd_kmeans(ctx, hist, mass, 3, p, 5.0, 1, 0, seed=2)     # one round, no update
    torch.cuda.synchronize()
    cost = cost.cpu().numpy()
    assert np.array_equal(a.cpu().numpy(), np.argmin(cost, axis=1))
    assert np.isclose(obj.item(), cost.min(axis=1).sum(), rtol=1e-14)
    assert obj.item() == obj_k.item()


@pytest.mark.parametrize("shards", [1, 2])
def test_kmeans_sharded_matches_pd_kmeans(ctx, shards):
    """kmeans_sharded from pd_kmeans' seeding: one shard gives bitwise the
    assignments, centroids and objectives of pd_kmeans; two shards emulated on
    one GPU (assign and grad per shard, sums added, one apply) the same
    assignments and centroids to the rounding of the added partial sums."""
    from paper_1805_08331_gb300 import sharded
    d, gamma, k, lam, rounds, steps = 16, 5e-3, 3, 5.0, 3, 2
    b, t, o, _ = inputs.mode_diagrams(12, 3, 40, 60, sigma=0.02, seed=5)
    h, _ = oracle.rasterize(b, t, o, d)
    hist, mass = hists_to_gpu(h), dev(masses(h).view(np.int32))
    p = api.pd_sinkhorn_default_params(gamma, d, max_iter=2000, tol=1e-6)
    _, c0, _ = api.pd_kmeans(ctx, hist, mass, k, p, lam, 0, steps, seed=3)
    a_ref, c_ref, obj_ref = api.pd_kmeans(ctx, hist, mass, k, p, lam, rounds, steps, seed=3)
    if shards == 1:
        a, c, obj = sharded.kmeans_sharded(ctx, hist, mass, p, c0, lam, rounds, steps)
        torch.cuda.synchronize()
        assert torch.equal(a, a_ref) and torch.equal(c, c_ref) and torch.equal(obj, obj_ref)
        return
    parts = [(hists_to_gpu(x), dev(masses(x).view(np.int32))) for x in (h[:5], h[5:])]
    gw = [torch.empty((hh.shape[0], d * d + 1), dtype=torch.float64, device="cuda") for hh, _ in parts]
    z = c0.clone()
    objs = []
    for rd in range(rounds):
        asg = [api.pd_kmeans_assign(ctx, hh, mm, p, z) for hh, mm in parts]
        objs.append(sum(x[1].item() for x in asg))
        for st in range(steps):
            g = [api.pd_barycenter_grad(ctx, hh, mm, p, z, k, x[0], gg, st > 0)
                 for (hh, mm), x, gg in zip(parts, asg, gw)]
            api.pd_barycenter_apply(ctx, z, g[0][0] + g[1][0], g[0][1] + g[1][1], gamma, lam)
    torch.cuda.synchronize()
    assert torch.equal(torch.cat([asg[0][0], asg[1][0]]), a_ref)
    assert torch.allclose(z, c_ref, rtol=1e-9, atol=1e-12 * c_ref.max().item())
    assert np.allclose(objs, obj_ref.cpu().numpy(), rtol=1e-12, atol=0)
