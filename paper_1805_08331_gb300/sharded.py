"""Alg. 2 (smoothed barycenter) over diagrams sharded across processes, one GPU
each.

The gradient of the smoothed energy (gradient proposition of Sec. 4) is a sum
over the diagrams, so a step splits at one exchange: every rank solves the
pairs (z + R a_n, a_n + R z) of its own diagrams and sums their gradient terms
(``pd_barycenter_grad``), the per-rank sums are added by one all-reduce of
d*d + 2 doubles, and every rank applies the same multiplicative update
(``pd_barycenter_apply``), so z stays identical on all ranks.  With one rank
the result is bitwise that of ``pd_barycenter``.  The arithmetic runs in the
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
