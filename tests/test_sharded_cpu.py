"""The sharded barycenter's exchange on CPU: two gloo ranks each hold half of
the diagrams and run `barycenter_sharded` with stand-in ops (the library's
ops need a GPU); both must end with the same measure and energies, equal to a
one-process run over all the diagrams up to the rounding of adding the
per-rank partial sums (the stand-in gradient is a per-diagram sum, like the
real one)."""
import os
import socket
import sys
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
D_GRID, N_ALL, STEPS = 6, 10, 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _data():
    rng = np.random.default_rng(5)
    hist = rng.integers(0, 4, size=(N_ALL, D_GRID, D_GRID)).astype(np.int32)
    return hist, hist.reshape(N_ALL, -1).sum(1).astype(np.int32)


def _ops():
    import torch

    def grad(ctx, hist, mass, params, z, k, owner, g_warm, warm):
        # per-diagram terms summed over the shard: a_n(x) + |a_n| z(x) / 64
        h = hist.reshape(hist.shape[0], -1).to(torch.float64)
        gsum = (h + mass.to(torch.float64)[:, None] * z.reshape(1, -1) / 64).sum(0, keepdim=True)
        count = torch.tensor([float(hist.shape[0])], dtype=torch.float64)
        csum = mass.to(torch.float64).sum().reshape(1)
        return gsum, count, csum

    def apply(ctx, z, gsum, count, gamma, lam):
        z.mul_(torch.exp(-lam * (gsum.reshape(z.shape) / count[0]) / 64))
        return z

    def init(ctx, hist, mass, params, lam, outer_iters):
        per = mass.to(torch.float64).mean() / (D_GRID * (D_GRID + 1) / 2)
        z = torch.triu(torch.ones(D_GRID, D_GRID, dtype=torch.float64)) * per
        return z, torch.empty(0, dtype=torch.float64)

    return {"grad": grad, "apply": apply, "init": init}


def _run(hist, mass, z_init):
    import torch
    sys.path.insert(0, ROOT)
    from paper_1805_08331_gb300 import sharded
    params = SimpleNamespace(d=D_GRID, gamma=1e-2)
    zi = None if z_init is None else torch.from_numpy(z_init)
    z, e = sharded.barycenter_sharded(None, torch.from_numpy(hist), torch.from_numpy(mass), params, 0.5, STEPS,
                                      z_init=zi, ops=_ops())
    return z.numpy().copy(), e.numpy().copy()


def _rank_main(rank, port, z_init, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        hist, mass = _data()
        lo, hi = (0, 4) if rank == 0 else (4, N_ALL)     # unequal shards
        out.put((rank, *_run(hist[lo:hi], mass[lo:hi], z_init)))
    finally:
        dist.destroy_process_group()


def _two_ranks(z_init):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, z_init, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_sharded_barycenter_two_gloo_ranks_equal_one_process():
    hist, mass = _data()
    z_init = np.triu(np.full((D_GRID, D_GRID), 2.0))
    (_, z0, e0), (_, z1, e1) = _two_ranks(z_init)
    assert np.array_equal(z0, z1) and np.array_equal(e0, e1)       # the same measure on every rank
    z, e = _run(hist, mass, z_init)                                # one process, all diagrams
    assert np.allclose(z0, z, rtol=1e-13, atol=0) and np.allclose(e0, e, rtol=1e-13, atol=0)
    assert not np.allclose(z, z_init, rtol=1e-3)


def test_sharded_barycenter_default_start_uses_all_ranks_mass():
    hist, mass = _data()
    (_, z0, e0), (_, z1, e1) = _two_ranks(None)
    assert np.array_equal(z0, z1)
    z, e = _run(hist, mass, None)
    assert np.allclose(z0, z, rtol=1e-13, atol=0) and np.allclose(e0, e, rtol=1e-13, atol=0)


K_CENT, ROUNDS, BSTEPS = 3, 3, 2


def _km_ops():
    import torch

    def assign(ctx, hist, mass, params, z):
        # stand-in cost: | |a_n| - 2 |z_c| |, ties to the lowest c
        zm = z.reshape(z.shape[0], -1).sum(1)
        cost = (mass.to(torch.float64)[:, None] - 2 * zm[None, :]).abs()
        a = torch.argmin(cost, dim=1).to(torch.int32)
        return a, cost.min(dim=1).values.sum().reshape(1), cost

    def grad(ctx, hist, mass, params, z, k, owner, g_warm, warm):
        h = hist.reshape(hist.shape[0], -1).to(torch.float64)
        zf = z.reshape(k, -1)
        gsum = torch.zeros((k, zf.shape[1]), dtype=torch.float64)
        count = torch.zeros(k, dtype=torch.float64)
        csum = torch.zeros(k, dtype=torch.float64)
        for n in range(h.shape[0]):
            c = int(owner[n])
            gsum[c] += h[n] + float(mass[n]) * zf[c] / 64
            count[c] += 1
            csum[c] += float(mass[n])
        return gsum, count, csum

    def apply(ctx, z, gsum, count, gamma, lam):
        zf = z.reshape(count.shape[0], -1)
        for c in range(count.shape[0]):
            if count[c] > 0:
                zf[c].mul_(torch.exp(-lam * (gsum[c] / count[c]) / 6400))   # small steps: clusters stay apart
        return z

    return {"assign": assign, "grad": grad, "apply": apply}


def _km_run(hist, mass):
    import torch
    sys.path.insert(0, ROOT)
    from paper_1805_08331_gb300 import sharded
    params = SimpleNamespace(d=D_GRID, gamma=1e-2)
    c0 = torch.from_numpy(np.stack([np.triu(np.full((D_GRID, D_GRID), v)) for v in (1.143, 1.262, 1.381)]))
    a, z, obj = sharded.kmeans_sharded(None, torch.from_numpy(hist), torch.from_numpy(mass), params, c0, 0.5,
                                       ROUNDS, BSTEPS, ops=_km_ops())
    return a.numpy().copy(), z.numpy().copy(), obj.numpy().copy()


def _km_rank_main(rank, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        hist, mass = _data()
        lo, hi = (0, 4) if rank == 0 else (4, N_ALL)
        out.put((rank, *_km_run(hist[lo:hi], mass[lo:hi])))
    finally:
        dist.destroy_process_group()


def test_sharded_kmeans_two_gloo_ranks_equal_one_process():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_km_rank_main, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    (_, a0, z0, o0), (_, a1, z1, o1) = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert np.array_equal(z0, z1) and np.array_equal(o0, o1)       # the same centroids on every rank
    hist, mass = _data()
    a, z, o = _km_run(hist, mass)                                  # one process, all diagrams
    assert np.array_equal(np.concatenate([a0, a1]), a)
    assert len(set(a.tolist())) > 1                                # several clusters in use
    assert np.allclose(z0, z, rtol=1e-13, atol=0) and np.allclose(o0, o, rtol=1e-13, atol=0)
