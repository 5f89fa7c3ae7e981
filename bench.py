"""Benchmark: batched Sinkhorn grid-cell updates/s on persistence-diagram pairs.

Workload (default): 2048 pairs of synthetic diagrams, point counts log-uniform
in [50, 500], birth ~ U[0,1), death = min(1, birth + Exp(mean 0.2)); grid
d = 128 (the metric's grid); gamma = 1e-3 (log-stabilised); every pair runs
until its relative marginal L1 error is <= 1e-6 (max 20000 iterations).

One step = rasterise all diagrams + solve all pairs (Alg. 1) + transport cost
(Prop. 2), inputs resident on the GPU.  value = sum over pairs of
iterations * 2 (d^2 + 1) cell updates / time.  e2e repeats the step through
the public API with the points in pinned host memory (H2D of the points and
D2H of the costs inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp32|bf16] [--pairs P] [--d D]

Under torchrun each rank solves its own batch (weak scaling, no data-path
collective); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1805_08331_gb300 import inputs  # noqa: E402

METRIC = "batched Sinkhorn grid-cell updates/s at d=128, fixed error vs FP64"
UNIT = "cell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "fp32_dense", "bf16"])
    ap.add_argument("--pairs", type=int, default=2048)
    ap.add_argument("--d", type=int, default=128)
    ap.add_argument("--gamma", type=float, default=1e-3)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=16, help="pairs in the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--parity-sample", type=int, default=4, help="pairs checked against the oracle")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving (p50/p99) leg")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="offered queries/s (Poisson)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="length of the query stream (60 s: the serving workload's length)")
    ap.add_argument("--serve-centroids", type=int, default=25, help="resident centroids per grid size")
    ap.add_argument("--serve-gamma", type=float, default=5e-3)
    ap.add_argument("--serve-tol", type=float, default=1e-4)
    ap.add_argument("--serve-nmax", type=int, default=5000, help="largest diagram of the stream (points)")
    ap.add_argument("--serve-inner", type=int, default=64, help="iterations per serving scheduling round")
    ap.add_argument("--no-compare", action="store_true", help="skip the engine comparison leg")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuning pass before the warm-up")
    ap.add_argument("--compare-only", action="store_true",
                    help="run only the engine comparison leg (print its JSON; for profiling)")
    ap.add_argument("--cta-threads", type=int, default=0, help="fix the iteration kernel's CTA width (0: automatic)")
    ap.add_argument("--lse-form", type=int, default=0,
                    help="log-sum-exp form of the iteration kernel: 0 automatic per half-step, 1 separable, "
                         "2 pairwise over the supports")
    ap.add_argument("--eps-stages", type=int, default=0,
                    help="gamma-continuation stages before the target gamma (0: plain Sinkhorn, Alg. 1)")
    ap.add_argument("--compare-pairs", type=int, default=2048, help="pairs of the engine comparison workload")
    ap.add_argument("--compare-plain-sample", type=int, default=24,
                    help="pairs timed with the one-pair-per-launch FP32 engine")
    return ap.parse_args()


def workload(args, rank):
    """Points of 2*pairs diagrams (pair p = diagrams 2p, 2p+1)."""
    b, t, o = inputs.random_diagrams(2 * args.pairs, nmin=50, nmax=500, exp_mean=0.2,
                                     seed=args.seed + 1000 * rank)
    return b, t, o


def config_dict(args, precision):
    return {"workload": f"{args.pairs} PD pairs, 50-500 points (log-uniform), birth~U[0,1), "
                        f"death=min(1,birth+Exp(0.2)); d={args.d}; gamma={args.gamma:g} log-stabilised; "
                        f"stop at relative marginal L1 error {args.tol:g}",
            "pairs_per_gpu": args.pairs, "d": args.d, "gamma": args.gamma, "tol": args.tol,
            "precision": precision, "eps_stages": args.eps_stages, "lse_form": args.lse_form,
            "l2": "flushed (512 MiB write) before every timed step"}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, n in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- peaks
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            m = json.load(fh)
        return m, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


FP32_LANES_PER_SM = 128
MUFU_PER_SM = 16


def num_sms():
    """SM count of the current device (152 on a GB300)."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def fp32_peak_tflops(sm_mhz):
    """CUDA-core FP32 FMA peak: SMs x 128 lanes x 2 flop x clock."""
    return num_sms() * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# DRAM bytes (read + write) of the base-2 iteration kernel per pair and
# launch, from one ncu capture of the current kernel (paired pairwise records;
# 512 pairs of this workload, one launch: 54.40 MB read + 0.32 MB written).  The kernel keeps every pair's state on chip; these bytes are the
# launch's load and store of the potentials, weights and support lists,
# whatever the number of iterations.
LSE2_DRAM_BYTES_PER_PAIR_LAUNCH = (54.397696e6 + 0.320768e6) / 512


def mufu_peak_gexp(sm_mhz):
    """Special-function-unit ex2 peak: SMs x 16 ex2/clk x clock, in 1e9/s."""
    return num_sms() * MUFU_PER_SM * sm_mhz * 1e6 / 1e9


PW_RATIO = 5   # the iteration kernel's form rule (pairwise while <= 5x the separable terms)


def lse_terms_per_iteration(hist, pairs, d, form=0, p2=True):
    """Log-sum-exp terms (one exponential each) of one iteration of the
    log-domain engine for every pair, in the form each half-step takes:
    separable = stage 1 nnz(in) x |columns of out| + stage 2 nnz(out) x |rows
    of in|; pairwise (p = 2) = nnz(in) x nnz(out); plus the Delta terms.
    Returns (terms of the forms taken, terms of the separable form)."""
    nz = hist.reshape(hist.shape[0], d, d) > 0
    nnz = nz.reshape(nz.shape[0], -1).sum(1).astype(np.float64)
    rows = nz.any(2).sum(1)
    cols = nz.any(1).sum(1)
    a, b = pairs[:, 0], pairs[:, 1]
    taken = np.zeros(len(a))
    sep_all = np.zeros(len(a))
    for o, i in ((a, b), (b, a)):   # u-update (out A, in B), v-update (out B, in A)
        sep = nnz[i] * cols[o] + rows[i] * nnz[o]
        direct = nnz[i] * nnz[o]
        pw = np.full(len(a), p2 and form == 2) | ((form == 0) & p2 & (direct <= PW_RATIO * sep))
        delta = nnz[o] + nnz[i] + 1
        taken += np.where(pw, direct, sep) + delta
        sep_all += sep + delta
    return taken, sep_all


# --------------------------------------------------------------------------- distributed helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- CPU baseline (oracle)
def cpu_baseline(args, b, t, o, n_pairs):
    import oracle
    d = args.d
    hist, _ = oracle.rasterize(b[:o[2 * n_pairs]], t[:o[2 * n_pairs]], o[:2 * n_pairs + 1], d)
    t0 = time.perf_counter()
    r = oracle.sinkhorn_pd_batch(d, args.gamma, hist[0::2], hist[1::2], args.max_iter, args.tol)
    dt = time.perf_counter() - t0
    cells = float(np.sum(r["iters"])) * 2 * (d * d + 1)
    return {"value": cells / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {n_pairs} pairs of the workload solved to tol by the FP64 oracle "
                      f"(OpenMP over pairs), {dt:.1f} s"}, r


def parity_sample(args, b, t, o, outs, status):
    """Costs of a sample of the timed step's pairs against the FP64 oracle run
    with the same max_iter and tol: the first few pairs, the first two pairs
    that stopped at max_iter (if any) and the largest pair (most points)."""
    import oracle
    P = args.pairs
    npts = np.diff(o)
    size = npts[0::2] + npts[1::2]
    sel = list(range(min(args.parity_sample, P)))
    sel += [int(p) for p in np.nonzero(status == 6)[0][:2] if int(p) not in sel]
    big = int(np.argmax(size))
    if big not in sel:
        sel.append(big)
    hist, _ = oracle.rasterize(b, t, o, args.d)
    hA = np.stack([hist[2 * p] for p in sel])
    hB = np.stack([hist[2 * p + 1] for p in sel])
    t0 = time.perf_counter()
    ref = oracle.sinkhorn_pd_batch(args.d, args.gamma, hA, hB, args.max_iter, args.tol)
    dt = time.perf_counter() - t0
    c_gpu = outs["cost"].cpu().numpy()[sel]
    rel = np.abs(c_gpu - ref["cost"]) / ref["cost"]
    return {"pairs_checked": len(sel), "pairs": sel, "status": [int(status[p]) for p in sel],
            "points": [int(size[p]) for p in sel], "rel_cost_err_vs_fp64": [float(x) for x in rel],
            "max_rel_cost_err_vs_fp64": float(rel.max()), "oracle_s": dt}


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    import oracle
    b, t, o = workload(args, 0)
    n = max(1, min(args.cpu_sample // 2, args.pairs))
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; warm-up steps are not repeated on the CPU
    times, cells = [], 0.0
    for s in range(args.steps):
        lo = (s * n) % max(1, args.pairs - n + 1)
        sel = slice(2 * lo, 2 * (lo + n))
        hist, _ = oracle.rasterize(b, t, o, args.d)
        hA, hB = hist[sel][0::2], hist[sel][1::2]
        t0 = time.perf_counter()
        r = oracle.sinkhorn_pd_batch(args.d, args.gamma, hA, hB, args.max_iter, args.tol)
        times.append(time.perf_counter() - t0)
        cells += float(np.sum(r["iters"])) * 2 * (args.d * args.d + 1)
    total = sum(times)
    val = cells / total
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, "fp64 oracle"), "impl": "reference",
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"each step: {n} pairs of the workload solved to tol (OpenMP over pairs)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1805_08331_gb300 import api
    api.load(build_if_missing=True)
    ctx = api.Context(local)
    precision = {"auto": api.PD_FP32, "fp32": api.PD_FP32, "fp32_dense": api.PD_FP32_DENSE,
                 "bf16": api.PD_BF16}[args.precision]
    pname = {api.PD_FP32: "fp32", api.PD_FP32_DENSE: "fp32", api.PD_BF16: "bf16"}[precision]
    b, t, o = workload(args, rank)
    d, P = args.d, args.pairs
    params = api.pd_sinkhorn_default_params(args.gamma, d, max_iter=args.max_iter, tol=args.tol,
                                            precision=precision, cta_threads=args.cta_threads,
                                            eps_stages=args.eps_stages, lse_form=args.lse_form)
    db, dt_, do = torch.from_numpy(b).cuda(), torch.from_numpy(t).cuda(), torch.from_numpy(o).cuda()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    # pair p = (diagram 2p, diagram 2p+1), both read from the one rasterised batch
    pairs = torch.arange(2 * P, dtype=torch.int32, device="cuda").view(P, 2).contiguous()

    def step():
        hist, mass = api.pd_rasterize(ctx, db, dt_, do, d)
        return api.pd_sinkhorn_batch(ctx, hist, mass, hist, mass, params, pairs=pairs)

    tuning = None
    if precision == api.PD_FP32 and not args.no_tune and args.cta_threads == 0:
        # autotuner: one trial launch per CTA width on this batch; the choice
        # goes into ctx's table and the timed steps use it
        hist_t, mass_t = api.pd_rasterize(ctx, db, dt_, do, d)
        th, trial = api.pd_sinkhorn_tune(ctx, hist_t, mass_t, hist_t, mass_t, params, pairs=pairs,
                                         trial_iters=args.max_iter)
        tuning = {"chosen_cta_threads": th, "trial_ms": {str(k): v for k, v in trial.items()},
                  "trial": "one launch per width: the full solve of the batch, cold-started"}
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    hist0, _ = api.pd_rasterize(ctx, db, dt_, do, d)
    terms, terms_sep = lse_terms_per_iteration(hist0.cpu().numpy(), pairs.cpu().numpy(), d, args.lse_form)
    barrier(ws)
    clocks = ClockSampler(local)
    clocks.start()
    ctx.profile_enable(True)
    ev = []
    cells = 0.0
    cells_all = 0.0
    iters_in_iter_kernel = 0
    pair_launches = 0.0
    lse_terms = 0.0
    lse_terms_sep = 0.0
    outs = None
    torch.cuda.synchronize()
    barrier(ws)
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = step()
        e1.record(stream)
        ev.append((e0, e1))
        it = outs["iters"].cpu().numpy()
        ok = outs["status"].cpu().numpy() == api.PD_OK
        # only results within the stated error count: pairs that stopped at
        # max_iter above tol are reported beside the value, not in it
        cells += float(it[ok].sum()) * 2 * (d * d + 1)
        cells_all += float(it.sum()) * 2 * (d * d + 1)
        iters_in_iter_kernel += int(np.maximum(it - 1, 0).sum())
        lse_terms += float((it * terms).sum())
        lse_terms_sep += float((it * terms_sep).sum())
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    step_ms = [a.elapsed_time(bq) for a, bq in ev]
    # the flush is excluded: each step is bracketed by its own events
    my_ms = float(np.sum(step_ms))
    tot_ms = max_over_ranks(my_ms, ws)
    all_cells = sum_over_ranks(cells, ws)
    value = all_cells / (tot_ms / 1e3)
    value_all_pairs = sum_over_ranks(cells_all, ws) / (tot_ms / 1e3)
    status = outs["status"].cpu().numpy()
    errs = outs["err"].cpu().numpy()

    # ---- e2e through the public API with host buffers (pinned)
    hb, ht, ho = (torch.from_numpy(x).pin_memory() for x in (b, t, o))
    h2d = int(hb.numel() * 8 + ht.numel() * 8 + ho.numel() * 8)
    d2h = int(P * 8)
    e2e_cells, e2e_s = 0.0, 0.0
    cost_host = torch.empty(P, dtype=torch.float64).pin_memory()
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xb, xt, xo = hb.cuda(non_blocking=True), ht.cuda(non_blocking=True), ho.cuda(non_blocking=True)
        hist, mass = api.pd_rasterize(ctx, xb, xt, xo, d)
        out = api.pd_sinkhorn_batch(ctx, hist, mass, hist, mass, params, pairs=pairs)
        cost_host.copy_(out["cost"], non_blocking=True)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
        ok = out["status"] == api.PD_OK
        e2e_cells += float(out["iters"][ok].sum().item()) * 2 * (d * d + 1)
    e2e_s = max_over_ranks(e2e_s, ws)
    e2e_val = sum_over_ranks(e2e_cells, ws) / e2e_s

    # ---- roofline of the dominant kernel (the iteration kernel)
    pk, pk_kind = peaks()
    iter_ms, iter_launches = prof.get("iter", (0.0, 0))
    flops = iters_in_iter_kernel * 8.0 * d ** 3          # two d^3-MAC GEMMs per half-step
    if precision == api.PD_BF16:
        peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
        bound, unit, kname = "tensor", "TFLOP/s", "sk_iter (tcgen05 BF16 separable GEMMs)"
        achieved = flops / (iter_ms / 1e3) / 1e12 if iter_ms > 0 else 0.0
        src = f"{pk_kind} bf16_tflops_sustained"
    elif precision == api.PD_FP32_DENSE:
        peak = fp32_peak_tflops(pk.get("sm_max_mhz", 2070.0))
        bound, unit, kname = "alu", "TFLOP/s", "sk_iter_fp32_kernel (CUDA-core FP32 separable GEMMs)"
        achieved = flops / (iter_ms / 1e3) / 1e12 if iter_ms > 0 else 0.0
        src = f"{pk_kind} sm_max_mhz x {num_sms()} SMs x 128 FP32 lanes x 2"
    else:
        peak = mufu_peak_gexp(pk.get("sm_max_mhz", 2070.0))
        bound, unit, kname = "alu", "Gexp/s", "sk_lse2_kernel (on-chip base-2 log-domain Sinkhorn)"
        achieved = lse_terms / (iter_ms / 1e3) / 1e9 if iter_ms > 0 else 0.0
        src = (f"{pk_kind} sm_max_mhz x {num_sms()} SMs x 16 MUFU ex2/clk (one exponential per log-sum-exp "
               f"term of the form each half-step takes)")
    traffic = None
    if precision == api.PD_FP32 and iter_launches:
        # pair loads: the first launch of a step loads every pair; the
        # drain-time hand-overs reload at most 2 x 152 pairs (512-thread CTAs)
        # and then at most 152 (1024-thread CTAs)
        per_step = iter_launches / max(args.steps, 1)
        nsm = num_sms()
        pair_launches = args.steps * (P + (2 * nsm if per_step >= 2 else 0) + (nsm if per_step >= 3 else 0))
        traffic = LSE2_DRAM_BYTES_PER_PAIR_LAUNCH * pair_launches / iter_launches
    # the metric's own tensor-unit roofline: one cell update of the dense
    # separable form = two d x d x d GEMMs per half-step over 2 (d^2 + 1) cells,
    # 4d flop per cell, against the sustained BF16 tensor peak
    tpk = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    tensor_unit = {"flop_per_cell": 4 * d, "peak_tflops": tpk,
                   "peak_source": f"{pk_kind} bf16_tflops_sustained",
                   "achieved_tflops": value / ws * 4 * d / 1e12,
                   "frac": value / ws * 4 * d / (tpk * 1e12)}
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak if peak else None, "traffic": traffic, "kernel": kname, "peak_source": src,
            "launches": iter_launches, "kernel_ms": iter_ms,
            "share_of_step": iter_ms / my_ms if my_ms else None, "tensor_unit": tensor_unit}
    if precision == api.PD_FP32:
        roof["terms"] = {"taken": lse_terms, "separable": lse_terms_sep, "lse_form": args.lse_form,
                         "separable_equivalent_gexp_per_s": lse_terms_sep / (iter_ms / 1e3) / 1e9 if iter_ms else None,
                         "note": "terms of all timed steps; achieved counts the terms the kernel evaluates "
                                 "(pairwise n_in x n_out where the form rule takes it)"}
    launches = int(sum(n for _, n in prof.values()))

    # ---- parity sample and CPU baseline (rank 0 only)
    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        n = max(1, min(args.cpu_sample, P))
        cpu, _ = cpu_baseline(args, b, t, o, n)
        parity = parity_sample(args, b, t, o, outs, status)
    serving = None
    if rank == 0 and not args.no_serve:
        serving = serve_leg(args, ctx)
    compare = None
    if rank == 0 and not args.no_compare:
        compare = compare_leg(args, ctx)
    if tuning is not None and rank == 0:
        # the same step on a context without a tuning table (built-in rule)
        c0 = api.Context(local)
        hist0, mass0 = api.pd_rasterize(c0, db, dt_, do, d)
        api.pd_sinkhorn_batch(c0, hist0, mass0, hist0, mass0, params, pairs=pairs)
        tms = []
        for _ in range(2):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hist0, mass0 = api.pd_rasterize(c0, db, dt_, do, d)
            api.pd_sinkhorn_batch(c0, hist0, mass0, hist0, mass0, params, pairs=pairs)
            e1.record(stream)
            torch.cuda.synchronize()
            tms.append(e0.elapsed_time(e1))
        c0.close()
        tuning["untuned_ms_per_step"] = float(np.mean(tms))
        tuning["tuned_ms_per_step"] = my_ms / args.steps
    ctx.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": pname, "data": "synthetic",
                "config": config_dict(args, pname), "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clk, "parity": parity,
                "status_counts": {str(int(s)): int((status == s).sum()) for s in np.unique(status)},
                "value_counts": "pairs with status PD_OK (relative marginal error <= tol) only",
                "excluded": {"pairs": int((status != api.PD_OK).sum()),
                             "iterations_per_step": int(outs["iters"].cpu().numpy()[status != api.PD_OK].sum()),
                             "value_with_them": value_all_pairs},
                "max_err": float(errs.max()), "max_err_counted": float(errs[status == api.PD_OK].max()) if
                (status == api.PD_OK).any() else None, "tuning": tuning, "serving": serving,
                "precision_comparison": compare}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------- engine comparison leg
def compare_leg(args, ctx):
    """The batched BF16 tensor-core engine (refined by the exact FP32 engine)
    against the plain FP32 form (one pair per launch) and the batched FP32
    engines, at equal stated accuracy (every engine stops at relative marginal
    error 1e-6; costs of a sample checked against the FP64 oracle), on
    k-means-shaped diagrams: d = 64, gamma = 5e-3, diagrams of 10 modes
    (30-300 points, sigma 0.03), where the linear domain holds."""
    import torch
    import oracle
    from paper_1805_08331_gb300 import api
    d, gamma, tol, P = 64, 5e-3, 1e-6, args.compare_pairs
    b, t, o, _ = inputs.mode_diagrams(2 * P, 10, 30, 300, sigma=0.03, seed=3)
    db_, dt_, do_ = (torch.from_numpy(x).cuda() for x in (b, t, o))
    hist, mass = api.pd_rasterize(ctx, db_, dt_, do_, d)
    pairs = torch.arange(2 * P, dtype=torch.int32, device="cuda").view(P, 2).contiguous()
    ns = 4
    href, _ = oracle.rasterize(b[:o[2 * ns]], t[:o[2 * ns]], o[:2 * ns + 1], d)
    ref = oracle.sinkhorn_pd_batch(d, gamma, href[0::2], href[1::2], 20000, tol)["cost"]
    cells_per_iter = 2 * (d * d + 1)

    def run(precision, npairs, reps, **kw):
        prm = api.pd_sinkhorn_default_params(gamma, d, max_iter=20000, tol=tol, precision=precision, **kw)
        out = None
        times = []
        for k in range(reps + 1):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = api.pd_sinkhorn_batch(ctx, hist, mass, hist, mass, prm, pairs=pairs[:npairs])
            e1.record()
            torch.cuda.synchronize()
            if k > 0 or reps == 0:
                times.append(e0.elapsed_time(e1))
        ms = float(np.mean(times))
        it = out["iters"].cpu().numpy()
        st = out["status"].cpu().numpy()
        m = min(ns, npairs)
        c = out["cost"].cpu().numpy()[:m]
        ok = st == api.PD_OK
        return {"pairs": npairs, "ms": ms, "cell_updates_per_s": float(it[ok].sum()) * cells_per_iter / (ms / 1e3),
                "iterations": int(it.sum()), "status_counts": {str(int(x)): int((st == x).sum()) for x in np.unique(st)},
                "max_rel_cost_err_vs_fp64_sample": float(np.max(np.abs(c - ref[:m]) / ref[:m]))}

    def by_class(precision, **kw):
        """Kernel time per launch class of one profiled solve (the library's CUDA-event profiler)."""
        prm = api.pd_sinkhorn_default_params(gamma, d, max_iter=20000, tol=tol, precision=precision, **kw)
        torch.cuda.synchronize()
        ctx.profile_enable(True)
        t0 = time.perf_counter()
        api.pd_sinkhorn_batch(ctx, hist, mass, hist, mass, prm, pairs=pairs)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) * 1e3
        prof = ctx.profile_read()
        ctx.profile_enable(False)
        return {"wall_ms": wall, "kernel_ms": {k: round(v[0], 3) for k, v in prof.items()},
                "launches": {k: int(v[1]) for k, v in prof.items()}}

    res = {"workload": f"{P} pairs of 10-mode diagrams (30-300 points, sigma 0.03), d={d}, gamma={gamma:g}, "
                       f"stop at relative marginal error {tol:g}; oracle sample: pairs 0-{ns - 1}",
           "bf16_tensor_core_refined": run(api.PD_BF16, P, 2, refine_iters=1),
           "fp32_plain_one_pair_per_launch": run(api.PD_FP32_PLAIN, min(args.compare_plain_sample, P), 0),
           "fp32_dense_batched": run(api.PD_FP32_DENSE, P, 1),
           "fp32_log_domain_batched": run(api.PD_FP32, P, 2)}
    res["bf16_tensor_core_refined"]["breakdown"] = by_class(api.PD_BF16, refine_iters=1)
    res["fp32_log_domain_batched"]["breakdown"] = by_class(api.PD_FP32)
    # tensor-core kernel alone: fixed 256 BF16 iterations, no stop, profiled
    pk, pk_kind = peaks()
    nfix = 256
    prm = api.pd_sinkhorn_default_params(gamma, d, max_iter=nfix, tol=0.0, precision=api.PD_BF16)
    api.pd_sinkhorn_batch(ctx, hist, mass, hist, mass, prm, pairs=pairs)
    torch.cuda.synchronize()
    ctx.profile_enable(True)
    out = api.pd_sinkhorn_batch(ctx, hist, mass, hist, mass, prm, pairs=pairs)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    tc_ms, tc_n = prof.get("tc", (0.0, 0))
    tc_iters = float(np.minimum(out["iters"].cpu().numpy(), nfix).sum())
    # d <= 64: two pairs share each 128 x 128 x 64 MMA GEMM (four per iteration)
    executed = tc_iters * 4 * (2.0 * 128 * 128 * 64) / 2
    algorithmic = tc_iters * 8.0 * d ** 3
    peak = pk.get("bf16_tflops", 1900.0)
    res["tensor_core_kernel"] = {
        "kernel": "sk_iter_bf16x2_kernel (tcgen05 kind::f16, BF16 operands by TMA, FP32 accumulation in TMEM, "
                  "two pairs per CTA)",
        "launches": int(tc_n), "ms": tc_ms, "pair_iterations": tc_iters,
        "executed_tflops": executed / (tc_ms / 1e3) / 1e12 if tc_ms else None,
        "algorithmic_tflops": algorithmic / (tc_ms / 1e3) / 1e12 if tc_ms else None,
        "peak_tflops": peak, "peak_source": f"{pk_kind} bf16_tflops (burst)",
        "executed_frac": executed / (tc_ms / 1e3) / 1e12 / peak if tc_ms else None,
        "note": "executed = four 128x128x64 MMA GEMMs per iteration shared by two pairs (each pair's product is a "
                "diagonal 64x64 block); algorithmic = 8 x d^3 flop per pair-iteration"}
    bf = res["bf16_tensor_core_refined"]["cell_updates_per_s"]
    for k in ("fp32_plain_one_pair_per_launch", "fp32_dense_batched", "fp32_log_domain_batched"):
        v = res[k]["cell_updates_per_s"]
        res["bf16_over_" + k] = bf / v if v > 0 else None
    return res


# --------------------------------------------------------------------------- serving leg
def serve_leg(args, ctx):
    """Poisson stream of distance / nearest-centroid queries through pd_serve:
    mixed grid sizes {32, 64, 128, 256}, log-uniform 10..5000 points, half of
    them nearest-centroid queries against resident centroids.  Returns the
    latency percentiles and the throughput of the completed queries."""
    import torch
    from paper_1805_08331_gb300 import api
    grids = api.SERVE_D
    k = args.serve_centroids
    # resident centroids: per mode, the mean of 8 rasterised diagrams of that mode
    cents = {}
    for d in grids:
        b, t, o, _ = inputs.mode_diagrams(8 * k, n_modes=k, nmin=30, nmax=300, sigma=0.03,
                                          seed=100 + d, labels=np.repeat(np.arange(k), 8))
        db_, dt_, do_ = (torch.from_numpy(x).cuda() for x in (b, t, o))
        h, _ = api.pd_rasterize(ctx, db_, dt_, do_, d)
        cents[d] = h.view(k, 8, d * d).to(torch.float64).mean(1).contiguous()
    tarr, kind, grid, counts = inputs.poisson_queries(args.serve_rate, args.serve_seconds, grids=grids,
                                                      nmin=10, nmax=args.serve_nmax, seed=args.seed + 77)
    nq = len(tarr)
    rng = np.random.default_rng(args.seed + 78)
    qa = inputs.random_diagrams(nq, counts=counts, seed=args.seed + 79)
    qb = inputs.random_diagrams(nq, counts=inputs.log_uniform_counts(rng, nq, 10, args.serve_nmax), seed=args.seed + 80)

    def pts(q, i):
        b, t, o = q
        return b[o[i]:o[i + 1]], t[o[i]:o[i + 1]]

    cfg = api.serve_default_config(gamma=args.serve_gamma, tol=args.serve_tol, max_iter=5000, inner_iters=args.serve_inner,
                                   max_hbm_bytes=48 << 30, warm_start=1)
    sv = api.Server(ctx, cfg)
    for d in grids:
        sv.load_centroids(d, cents[d])
    tickets = [None] * nq
    results = [None] * nq
    submitted = threading.Event()

    def collector():
        for i in range(nq):
            while tickets[i] is None and not submitted.is_set():
                time.sleep(0.0002)
            if tickets[i] is not None:
                results[i] = sv.wait(tickets[i], 600000)

    th = threading.Thread(target=collector)
    th.start()
    t0 = time.perf_counter()
    refused = 0
    for i in range(nq):
        dt = tarr[i] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ba, da = pts(qa, i)
        try:
            if kind[i] == 0:
                bb, dbb = pts(qb, i)
                tickets[i] = sv.submit_distance(int(grid[i]), ba, da, bb, dbb)
            else:
                tickets[i] = sv.submit_nearest(int(grid[i]), ba, da)
        except api.PdError:
            refused += 1
    submitted.set()
    th.join()
    wall = time.perf_counter() - t0
    sv.close()
    done = [r for r in results if r is not None]
    lat = np.array([r["latency_ms"] for r in done])
    dgrid = np.array([int(grid[i]) for i in range(nq) if results[i] is not None])
    per_d = {}
    # points of a query's diagrams (the larger of A and, for a distance, B)
    npts = np.array([max(counts[i], (qb[2][i + 1] - qb[2][i]) if kind[i] == 0 else 0)
                     for i in range(nq) if results[i] is not None])
    for d in grids:
        ld = lat[dgrid == d]
        if len(ld):
            per_d[str(d)] = {"queries": int(len(ld)), "p50_ms": float(np.percentile(ld, 50)),
                             "p99_ms": float(np.percentile(ld, 99))}
            small = lat[(dgrid == d) & (npts <= 1000)]
            big = lat[(dgrid == d) & (npts > 1000)]
            if len(small):
                per_d[str(d)]["p99_ms_up_to_1000_points"] = float(np.percentile(small, 99))
            if len(big):
                per_d[str(d)]["p99_ms_over_1000_points"] = float(np.percentile(big, 99))
                per_d[str(d)]["queries_over_1000_points"] = int(len(big))
    st = np.array([r["status"] for r in done])
    it = np.array([r["iters"] for r in done])
    return {"p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "throughput_qps": len(done) / wall, "offered_qps": args.serve_rate, "stream_s": args.serve_seconds,
            "wall_s": wall, "queries": int(nq), "completed": len(done), "refused": refused,
            "status_counts": {str(int(x)): int((st == x).sum()) for x in np.unique(st)},
            "mean_iters": float(it.mean()) if len(it) else None, "per_d": per_d,
            "workload": f"Poisson {args.serve_rate:g} q/s for {args.serve_seconds:g} s; half distance, half "
                        f"nearest of {k} resident centroids per d (mean histograms of mode diagrams); "
                        f"d uniform on {{32,64,128,256}}; 10-{args.serve_nmax} points log-uniform; gamma={args.serve_gamma:g}, "
                        f"tol={args.serve_tol:g}; warm-started centroid potentials"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.compare_only:
        import torch
        from paper_1805_08331_gb300 import api
        api.load(build_if_missing=True)
        ctx = api.Context(0)
        print(json.dumps({"precision_comparison": compare_leg(args, ctx)}), flush=True)
        ctx.close()
        torch.cuda.synchronize()
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
