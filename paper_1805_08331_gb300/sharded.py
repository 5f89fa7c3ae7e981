"""Alg. 2 (smoothed barycenter) and the k-means of Sec. 5 over diagrams sharded
across processes, one GPU each.

The gradient of the smoothed energy (gradient proposition of Sec. 4) is a sum
over the diagrams, so a step splits at one exchange: every rank solves the
pairs (z + R a_n, a_n + R z) of its own diagrams and sums their gradient terms
(``pd_barycenter_grad``), the per-rank sums are added by one all-reduce of
d*d + 2 doubles, and every rank applies the same multiplicative update
(``pd_barycenter_apply``), so z stays identical on all ranks.  With one rank
the result is bitwise that of ``pd_barycenter``.  k-means adds a local
assignment per round (``pd_kmeans_assign``) and runs the same split step for
all k centroids at once, owner = assignment.  The arithmetic runs in the
library's kernels; this module only moves the sums between the ranks.
"""
from __future__ import annotations

from . import api


def _world(group):
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return None, 1
    return dist, dist.get_world_size(group)


def _default_ops():
    return {"grad": api.pd_barycenter_grad, "apply": api.pd_barycenter_apply, "init": api.pd_barycenter}


def barycenter_sharded(ctx, hist, mass, params, lam, outer_iters, z_init=None, group=None, ops=None):
    """Alg. 2 on this rank's diagrams (hist, mass: int32 CUDA tensors of uint32
    counts, [N_r, d, d] and [N_r]); the barycenter is that of the diagrams of
    all ranks of ``group`` (torch.distributed, NCCL for CUDA tensors; no
    process group: one rank).  z_init: float64 [d, d] or None (the uniform
    measure above the diagonal with the mean mass of all ranks' diagrams).
    Returns (z [d, d] float64, energy [outer_iters] float64), the same on every
    rank."""
    import torch
    ops = ops or _default_ops()
    dist, ws = _world(group)
    d = params.d
    n_local = int(hist.shape[0])

    def allreduce(t):
        if ws > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t

    if z_init is None:
        # each rank's uniform start carries its own mean mass; weighting by the
        # diagram counts and adding gives the mean over all diagrams
        z, _ = ops["init"](ctx, hist, mass, params, lam, 0)
        if ws > 1:
            nt = allreduce(torch.tensor([float(n_local)], dtype=torch.float64, device=z.device))
            z = allreduce(z * n_local) / nt
    else:
        z = z_init.to(torch.float64).clone()
    z = z.reshape(d, d).contiguous()
    g_warm = torch.empty((n_local, d * d + 1), dtype=torch.float64, device=z.device)
    energy = torch.empty(outer_iters, dtype=torch.float64, device=z.device)
    for t in range(outer_iters):
        gsum, count, csum = ops["grad"](ctx, hist, mass, params, z, 1, None, g_warm, t > 0)
        if ws > 1:
            buf = allreduce(torch.cat([gsum.reshape(-1), count, csum]))
            gsum, count, csum = buf[:d * d].reshape(1, d * d), buf[d * d:d * d + 1], buf[d * d + 1:]
        ops["apply"](ctx, z, gsum, count, params.gamma, lam)
        energy[t] = csum[0] / count[0]
    return z, energy


def kmeans_sharded(ctx, hist, mass, params, centroids_init, lam, rounds, bary_steps, group=None, ops=None):
    """k-means rounds (Sec. 5) over diagrams sharded across the ranks of
    ``group``: each rank assigns its own diagrams (``pd_kmeans_assign``), the
    objective is summed across ranks, and each of the ``bary_steps`` Alg. 2
    steps of the centroid update adds the per-rank, per-centroid sums
    (``pd_barycenter_grad`` with owner = assignment; k*d*d + 2k doubles) before
    ``pd_barycenter_apply``.  centroids_init: float64 [k, d, d], the same on
    every rank (pd_kmeans with rounds = 0 gives its seeding).  With one rank the
    result is bitwise that of pd_kmeans from the same centroids.  Returns
    (assign [N_r] of the last round, centroids [k, d, d], objective [rounds])."""
    import torch
    ops = ops or {"assign": api.pd_kmeans_assign, "grad": api.pd_barycenter_grad, "apply": api.pd_barycenter_apply}
    dist, ws = _world(group)
    d = params.d
    z = centroids_init.to(torch.float64).clone().contiguous()
    k = int(z.shape[0])
    n_local = int(hist.shape[0])

    def allreduce(t):
        if ws > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t

    g_warm = torch.empty((n_local, d * d + 1), dtype=torch.float64, device=z.device)
    objective = torch.empty(rounds, dtype=torch.float64, device=z.device)
    assign = None
    for rd in range(rounds):
        assign, obj, _ = ops["assign"](ctx, hist, mass, params, z)
        objective[rd] = allreduce(obj.clone())[0]
        for st in range(bary_steps):
            gsum, count, csum = ops["grad"](ctx, hist, mass, params, z, k, assign, g_warm, st > 0)
            if ws > 1:
                buf = allreduce(torch.cat([gsum.reshape(-1), count, csum]))
                gsum, count = buf[:k * d * d].reshape(k, d * d), buf[k * d * d:k * d * d + k]
            ops["apply"](ctx, z, gsum, count, params.gamma, lam)
    return assign, z, objective
