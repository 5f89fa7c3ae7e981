"""The bench's N > 1 path on CPU: world-size-2 gloo ranks check the
reductions the driver relies on (max of the per-rank times, sum of the
per-rank units), that each rank draws its own workload (weak scaling, no
data-path collective), and that only rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, out):
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench.dist_env()
        mx = bench.max_over_ranks(1.5 + rank, ws)
        sm = bench.sum_over_ranks(10.0 * (rank + 1), ws)
        bench.barrier(ws)

        class A:
            pairs, seed = 3, 1
        b, t, o = bench.workload(A, rank)
        out.put((rank, got_ws, got_rank, mx, sm, float(np.sum(b)), int(o[-1])))
    finally:
        dist.destroy_process_group()


def _reference_rank1(port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    import bench
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    out.put(bench.run_reference(bench.parse()))


def test_bench_reductions_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, k0, mx0, sm0, sb0, n0), (r1, ws1, k1, mx1, sm1, sb1, n1) = res
    assert (ws0, ws1, k0, k1) == (2, 2, 0, 1)
    assert mx0 == mx1 == 2.5          # max of the per-rank times
    assert sm0 == sm1 == 30.0         # sum of the per-rank units
    assert sb0 != sb1                 # each rank solves its own pairs


def test_reference_arm_runs_on_rank0_only():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_reference_rank1, args=(0, q))
    p.start()
    rc = q.get(timeout=120)
    p.join(timeout=60)
    assert p.exitcode == 0 and rc == 0
