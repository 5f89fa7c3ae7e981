"""Thin Python binding of the C ABI in ``include/pd_ot.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libpdot.so``.  Tensors are PyTorch CUDA tensors (PyTorch is
used for device memory and streams); their data pointers and the current
stream are passed straight through.  If the library is missing, loading it
raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PD_OK, PD_ERR_INVALID, PD_ERR_OOM, PD_ERR_CUDA, PD_ERR_TIMEOUT, PD_ERR_QUEUE_FULL = 0, 1, 2, 3, 4, 5
PD_NOT_CONVERGED, PD_PENDING, PD_ERR_RANGE = 6, 7, 8
PD_FP32, PD_BF16, PD_FP32_DENSE, PD_FP32_PLAIN = 0, 1, 2, 3
STATUS_NAMES = {0: "PD_OK", 1: "PD_ERR_INVALID", 2: "PD_ERR_OOM", 3: "PD_ERR_CUDA", 4: "PD_ERR_TIMEOUT",
                5: "PD_ERR_QUEUE_FULL", 6: "PD_NOT_CONVERGED", 7: "PD_PENDING", 8: "PD_ERR_RANGE"}

# Every symbol the header declares (checked by the ABI test).
EXPORTED = ["pd_abi_version", "pd_ctx_create", "pd_ctx_destroy", "pd_last_error", "pd_rasterize",
            "pd_sinkhorn_default_params", "pd_sinkhorn_batch", "pd_profile_enable", "pd_profile_read",
            "pd_sinkhorn_batch_noalloc", "pd_barycenter", "pd_kmeans", "pd_serve_default_config",
            "pd_serve_create", "pd_serve_load_centroids", "pd_serve_submit", "pd_serve_poll", "pd_serve_wait",
            "pd_serve_inject_failure", "pd_serve_destroy", "pd_sinkhorn_bounds", "pd_barycenter_grad",
            "pd_barycenter_apply", "pd_kmeans_assign", "pd_workspace_query", "pd_ctx_set_workspace",
            "pd_sinkhorn_tune", "pd_tune_save", "pd_tune_load", "pd_sinkhorn_batch_groups"]
PD_OP_SINKHORN, PD_OP_BOUNDS, PD_OP_BARYCENTER, PD_OP_BARY_GRAD, PD_OP_KMEANS_ASSIGN, PD_OP_KMEANS = 0, 1, 2, 3, 4, 5
PD_Q_DISTANCE, PD_Q_NEAREST = 0, 1
SERVE_D = (32, 64, 128, 256)
PD_K_RASTER, PD_K_SETUP, PD_K_LOGSTEP, PD_K_ABSORB, PD_K_ITER, PD_K_FINALIZE, PD_K_TC, PD_K_COUNT = (
    0, 1, 2, 3, 4, 5, 6, 16)
KERNEL_NAMES = {0: "raster", 1: "setup", 2: "logstep", 3: "absorb", 4: "iter", 5: "finalize", 6: "tc"}


class PdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SinkhornParams(ctypes.Structure):
    """Mirror of pd_sinkhorn_params."""
    _fields_ = [("gamma", ctypes.c_double), ("d", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("tol", ctypes.c_double), ("precision", ctypes.c_int), ("refine_iters", ctypes.c_int),
                ("absorb_tau", ctypes.c_double), ("absorb_every", ctypes.c_int), ("rel_log_thresh", ctypes.c_double),
                ("eps_stages", ctypes.c_int), ("p", ctypes.c_double), ("bary_sharpen", ctypes.c_int),
                ("cta_threads", ctypes.c_int), ("kernel_tier", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("diag_tc_timeout", ctypes.c_int), ("lse_form", ctypes.c_int)]


class SinkhornGroup(ctypes.Structure):
    """Mirror of pd_sinkhorn_group."""
    _fields_ = [("d", ctypes.c_int), ("P", ctypes.c_int), ("histA", ctypes.c_void_p), ("massA", ctypes.c_void_p),
                ("histB", ctypes.c_void_p), ("massB", ctypes.c_void_p), ("pairs", ctypes.c_void_p),
                ("g_init", ctypes.c_void_p), ("cost", ctypes.c_void_p), ("row_marg", ctypes.c_void_p),
                ("col_marg", ctypes.c_void_p), ("f", ctypes.c_void_p), ("g", ctypes.c_void_p),
                ("iters", ctypes.c_void_p), ("err", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class ServeConfig(ctypes.Structure):
    """Mirror of pd_serve_config."""
    _fields_ = [("gamma", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("inner_iters", ctypes.c_int), ("slots", ctypes.c_int * 4), ("max_hbm_bytes", ctypes.c_size_t),
                ("queue_capacity", ctypes.c_int), ("warm_start", ctypes.c_int)]


class Query(ctypes.Structure):
    """Mirror of pd_query."""
    _fields_ = [("kind", ctypes.c_int), ("d", ctypes.c_int),
                ("birth_a_host", ctypes.c_void_p), ("death_a_host", ctypes.c_void_p), ("n_a", ctypes.c_int),
                ("birth_b_host", ctypes.c_void_p), ("death_b_host", ctypes.c_void_p), ("n_b", ctypes.c_int)]


class Result(ctypes.Structure):
    """Mirror of pd_result."""
    _fields_ = [("status", ctypes.c_int), ("cost", ctypes.c_double), ("centroid", ctypes.c_int),
                ("iters", ctypes.c_int), ("latency_ms", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libpdot.so (optionally building it first).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise PdError(PD_ERR_CUDA, f"CUDA library not built: {path} (run __graft_entry__.build())")
            _build.build()
        lib = ctypes.CDLL(path)
        lib.pd_abi_version.restype = ctypes.c_int
        lib.pd_ctx_create.argtypes = [ctypes.c_int, ctypes.POINTER(_vp)]
        lib.pd_ctx_destroy.argtypes = [_vp]
        lib.pd_ctx_destroy.restype = None
        lib.pd_last_error.argtypes = [_vp]
        lib.pd_last_error.restype = ctypes.c_char_p
        lib.pd_rasterize.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
        lib.pd_sinkhorn_default_params.argtypes = [ctypes.POINTER(SinkhornParams), ctypes.c_double, ctypes.c_int]
        lib.pd_sinkhorn_default_params.restype = None
        lib.pd_sinkhorn_batch.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(SinkhornParams),
                                          _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        lib.pd_sinkhorn_batch_noalloc.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int,
                                                  ctypes.POINTER(SinkhornParams), _vp, _vp, _vp, _vp, _vp, _vp,
                                                  _vp, _vp, _vp, _vp]
        lib.pd_sinkhorn_bounds.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int,
                                           ctypes.POINTER(SinkhornParams), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        lib.pd_barycenter.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(SinkhornParams), ctypes.c_double,
                                      ctypes.c_int, ctypes.c_double, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int), _vp]
        lib.pd_workspace_query.argtypes = [ctypes.c_int, ctypes.POINTER(SinkhornParams), ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_size_t)]
        lib.pd_ctx_set_workspace.argtypes = [_vp, _vp, ctypes.c_size_t]
        lib.pd_sinkhorn_tune.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(SinkhornParams),
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                         _vp]
        lib.pd_tune_save.argtypes = [_vp, ctypes.c_char_p]
        lib.pd_sinkhorn_batch_groups.argtypes = [_vp, ctypes.c_int, _vp, ctypes.POINTER(SinkhornParams), _vp]
        lib.pd_tune_load.argtypes = [_vp, ctypes.c_char_p]
        lib.pd_kmeans.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(SinkhornParams),
                                  ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _vp, _vp, _vp, _vp]
        lib.pd_barycenter_grad.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(SinkhornParams),
                                           _vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp]
        lib.pd_barycenter_apply.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_double,
                                            ctypes.c_double, _vp]
        lib.pd_kmeans_assign.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(SinkhornParams),
                                         _vp, _vp, _vp, _vp, _vp]
        lib.pd_serve_default_config.argtypes = [ctypes.POINTER(ServeConfig)]
        lib.pd_serve_default_config.restype = None
        lib.pd_serve_create.argtypes = [_vp, ctypes.POINTER(ServeConfig), ctypes.POINTER(_vp)]
        lib.pd_serve_load_centroids.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int]
        lib.pd_serve_submit.argtypes = [_vp, ctypes.POINTER(Query), ctypes.POINTER(ctypes.c_uint64)]
        lib.pd_serve_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(Result)]
        lib.pd_serve_wait.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(Result), ctypes.c_double]
        lib.pd_serve_inject_failure.argtypes = [_vp]
        lib.pd_serve_destroy.argtypes = [_vp]
        lib.pd_serve_destroy.restype = None
        lib.pd_profile_enable.argtypes = [_vp, ctypes.c_int]
        lib.pd_profile_read.argtypes = [_vp, _vp, _vp]
        _lib = lib
        return lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """Owns a pd_ctx (library workspace) bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = _vp()
        st = self.lib.pd_ctx_create(int(device), ctypes.byref(h))
        if st != PD_OK:
            raise PdError(st, "pd_ctx_create failed")
        self.handle = h
        self.device = device

    def last_error(self) -> str:
        return self.lib.pd_last_error(self.handle).decode()

    def check(self, st):
        if st != PD_OK:
            raise PdError(st, self.last_error())

    def profile_enable(self, on: bool = True):
        self.check(self.lib.pd_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self):
        """{kernel class name: (total ms, launches)} of the recorded launches."""
        ms = (ctypes.c_double * PD_K_COUNT)()
        n = (ctypes.c_int64 * PD_K_COUNT)()
        self.check(self.lib.pd_profile_read(self.handle, ctypes.cast(ms, _vp), ctypes.cast(n, _vp)))
        return {KERNEL_NAMES.get(k, str(k)): (ms[k], n[k]) for k in range(PD_K_COUNT) if n[k] > 0}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.pd_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pd_sinkhorn_default_params(gamma: float, d: int, **kw) -> SinkhornParams:
    p = SinkhornParams()
    load().pd_sinkhorn_default_params(ctypes.byref(p), float(gamma), int(d))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def pd_rasterize(ctx: Context, birth, death, offsets, d: int, hist=None, mass=None, stream=None):
    """Rasterise B diagrams given as CUDA tensors (float64 birth/death, int64
    offsets [B+1]).  Returns (hist uint32 [B,d,d] as int32 storage, mass)."""
    import torch
    B = offsets.numel() - 1
    dev = offsets.device
    if hist is None:
        hist = torch.empty((B, d, d), dtype=torch.int32, device=dev)
    if mass is None:
        mass = torch.empty((B,), dtype=torch.int32, device=dev)
    ctx.check(ctx.lib.pd_rasterize(ctx.handle, _ptr(birth), _ptr(death), _ptr(offsets), int(B), int(d),
                                   _ptr(hist), _ptr(mass), _stream(stream)))
    return hist, mass


def pd_sinkhorn_batch(ctx: Context, histA, massA, histB, massB, params: SinkhornParams, pairs=None, g_init=None,
                      want_marginals=False, want_potentials=False, stream=None, out=None):
    """Alg. 1 over P pairs.  Histograms are int32 CUDA tensors holding uint32
    counts.  Returns a dict of CUDA tensors (cost, iters, err, status and, if
    requested, row_marg, col_marg, f, g)."""
    import torch
    dev = histA.device
    P = pairs.shape[0] if pairs is not None else histA.shape[0]
    n = params.d * params.d + 1
    o = dict(out or {})
    o.setdefault("cost", torch.empty(P, dtype=torch.float64, device=dev))
    o.setdefault("iters", torch.empty(P, dtype=torch.int32, device=dev))
    o.setdefault("err", torch.empty(P, dtype=torch.float32, device=dev))
    o.setdefault("status", torch.empty(P, dtype=torch.int32, device=dev))
    if want_marginals:
        o.setdefault("row_marg", torch.empty((P, n), dtype=torch.float32, device=dev))
        o.setdefault("col_marg", torch.empty((P, n), dtype=torch.float32, device=dev))
    if want_potentials:
        o.setdefault("f", torch.empty((P, n), dtype=torch.float64, device=dev))
        o.setdefault("g", torch.empty((P, n), dtype=torch.float64, device=dev))
    ctx.check(ctx.lib.pd_sinkhorn_batch(
        ctx.handle, _ptr(histA), _ptr(massA), _ptr(histB), _ptr(massB), _ptr(pairs), int(P), ctypes.byref(params),
        _ptr(g_init), _ptr(o["cost"]), _ptr(o.get("row_marg")), _ptr(o.get("col_marg")), _ptr(o.get("f")),
        _ptr(o.get("g")), _ptr(o["iters"]), _ptr(o["err"]), _ptr(o["status"]), _stream(stream)))
    return o


def pd_sinkhorn_batch_groups(ctx: Context, groups, params: SinkhornParams, want_marginals=False,
                             want_potentials=False, stream=None):
    """Pairs of several grid sizes in one persistent launch.  groups: list of
    dicts with d, histA, massA, histB, massB and optional pairs, g_init (CUDA
    tensors as for pd_sinkhorn_batch).  Returns one output dict per group."""
    import torch
    arr = (SinkhornGroup * len(groups))()
    outs = []
    for k, gd in enumerate(groups):
        d, hA = int(gd["d"]), gd["histA"]
        pairs = gd.get("pairs")
        P = pairs.shape[0] if pairs is not None else hA.shape[0]
        n = d * d + 1
        dev = hA.device
        o = {"cost": torch.empty(P, dtype=torch.float64, device=dev),
             "iters": torch.empty(P, dtype=torch.int32, device=dev),
             "err": torch.empty(P, dtype=torch.float32, device=dev),
             "status": torch.empty(P, dtype=torch.int32, device=dev)}
        if want_marginals:
            o["row_marg"] = torch.empty((P, n), dtype=torch.float32, device=dev)
            o["col_marg"] = torch.empty((P, n), dtype=torch.float32, device=dev)
        if want_potentials:
            o["f"] = torch.empty((P, n), dtype=torch.float64, device=dev)
            o["g"] = torch.empty((P, n), dtype=torch.float64, device=dev)
        val = lambda t: None if t is None else t.data_ptr()   # noqa: E731
        arr[k] = SinkhornGroup(d, int(P), val(hA), val(gd["massA"]), val(gd["histB"]), val(gd["massB"]), val(pairs),
                               val(gd.get("g_init")), val(o["cost"]), val(o.get("row_marg")), val(o.get("col_marg")),
                               val(o.get("f")), val(o.get("g")), val(o["iters"]), val(o["err"]), val(o["status"]))
        outs.append(o)
    ctx.check(ctx.lib.pd_sinkhorn_batch_groups(ctx.handle, len(groups), ctypes.cast(arr, _vp), ctypes.byref(params),
                                               _stream(stream)))
    return outs


def pd_sinkhorn_bounds(ctx: Context, histA, massA, histB, massB, params: SinkhornParams, pairs=None,
                       g_init=None, stream=None):
    """pd_sinkhorn_bounds (Sec. 3 bounds): dict with cost, lower (m_t), upper
    (M_t, the rounded plan's cost, Prop. 3), iters, err, status."""
    import torch
    P = pairs.shape[0] if pairs is not None else histA.shape[0]
    dev = histA.device
    o = {"cost": torch.empty(P, dtype=torch.float64, device=dev),
         "lower": torch.empty(P, dtype=torch.float64, device=dev),
         "upper": torch.empty(P, dtype=torch.float64, device=dev),
         "iters": torch.empty(P, dtype=torch.int32, device=dev),
         "err": torch.empty(P, dtype=torch.float32, device=dev),
         "status": torch.empty(P, dtype=torch.int32, device=dev)}
    ctx.check(ctx.lib.pd_sinkhorn_bounds(
        ctx.handle, _ptr(histA), _ptr(massA), _ptr(histB), _ptr(massB), _ptr(pairs), int(P), ctypes.byref(params),
        _ptr(g_init), _ptr(o["cost"]), _ptr(o["lower"]), _ptr(o["upper"]), _ptr(o["iters"]), _ptr(o["err"]),
        _ptr(o["status"]), _stream(stream)))
    return o


def pd_barycenter(ctx: Context, hist, mass, params: SinkhornParams, lam: float, outer_iters: int, z_init=None,
                  stream=None, rel_energy_tol: float = 0.0):
    """Alg. 2 on N histograms (int32 CUDA tensors holding uint32 counts), at
    most outer_iters steps; with rel_energy_tol > 0 it stops after the first
    step t >= 1 with |E_t/E_{t-1} - 1| < rel_energy_tol.
    Returns (z [d,d] float64 CUDA tensor, energy [steps run] float64)."""
    import torch
    d = params.d
    z = torch.empty((d, d), dtype=torch.float64, device=hist.device)
    e = torch.empty(max(outer_iters, 1), dtype=torch.float64, device=hist.device)
    steps = ctypes.c_int(0)
    ctx.check(ctx.lib.pd_barycenter(ctx.handle, _ptr(hist), _ptr(mass), int(hist.shape[0]), ctypes.byref(params),
                                    float(lam), int(outer_iters), float(rel_energy_tol), _ptr(z_init), _ptr(z),
                                    _ptr(e), ctypes.byref(steps), _stream(stream)))
    return z, e[:steps.value]


def pd_sinkhorn_tune(ctx: Context, histA, massA, histB, massB, params: SinkhornParams, pairs=None,
                     trial_iters: int = 64, stream=None):
    """Autotune the iteration kernel's CTA width on this batch (see
    include/pd_ot.h); the choice goes into ctx's tuning table.  Returns
    (threads, {width: trial ms})."""
    P = pairs.shape[0] if pairs is not None else histA.shape[0]
    th = ctypes.c_int(0)
    ms = (ctypes.c_double * 4)()
    ctx.check(ctx.lib.pd_sinkhorn_tune(ctx.handle, _ptr(histA), _ptr(massA), _ptr(histB), _ptr(massB), _ptr(pairs),
                                       int(P), ctypes.byref(params), int(trial_iters), ctypes.byref(th), ms,
                                       _stream(stream)))
    return th.value, {w: ms[k] for k, w in enumerate((128, 256, 512, 1024)) if ms[k] == ms[k]}


def pd_tune_save(ctx: Context, path: str):
    ctx.check(ctx.lib.pd_tune_save(ctx.handle, os.fsencode(path)))


def pd_tune_load(ctx: Context, path: str):
    ctx.check(ctx.lib.pd_tune_load(ctx.handle, os.fsencode(path)))


def pd_workspace_query(op: int, params: SinkhornParams, n: int, k: int = 0) -> int:
    """Device workspace bytes a context holds for one call of `op` (PD_OP_*)."""
    out = ctypes.c_size_t(0)
    st = load().pd_workspace_query(int(op), ctypes.byref(params), int(n), int(k), ctypes.byref(out))
    if st != PD_OK:
        raise PdError(st, "pd_workspace_query failed")
    return int(out.value)


def pd_ctx_set_workspace(ctx: Context, ws=None, nbytes: int = 0):
    """Give the context a caller-owned device buffer (a CUDA tensor, 256-byte
    aligned) as its workspace; None returns to library-allocated workspace."""
    ctx.check(ctx.lib.pd_ctx_set_workspace(ctx.handle, _ptr(ws), int(nbytes) if ws is not None else 0))


def pd_barycenter_grad(ctx: Context, hist, mass, params: SinkhornParams, z, k: int = 1, owner=None, g_warm=None,
                       warm: bool = False, stream=None):
    """Per-shard half of an Alg. 2 step (see include/pd_ot.h).  z: float64
    CUDA tensor [k, d, d] (or [d, d] for k = 1); owner: int32 [N] or None;
    g_warm: float64 [N, d*d+1] or None (written; read when warm).  Returns
    (gsum [k, d*d], count [k], cost_sum [k]) float64 CUDA tensors."""
    import torch
    d, N = params.d, int(hist.shape[0])
    gsum = torch.empty((k, d * d), dtype=torch.float64, device=hist.device)
    count = torch.empty(k, dtype=torch.float64, device=hist.device)
    csum = torch.empty(k, dtype=torch.float64, device=hist.device)
    ctx.check(ctx.lib.pd_barycenter_grad(ctx.handle, _ptr(hist), _ptr(mass), N, int(k), ctypes.byref(params), _ptr(z),
                                         _ptr(owner), _ptr(g_warm), 1 if warm else 0, _ptr(gsum), _ptr(count),
                                         _ptr(csum), _stream(stream)))
    return gsum, count, csum


def pd_barycenter_apply(ctx: Context, z, gsum, count, gamma: float, lam: float, stream=None):
    """Second half of the step: z (float64 [k, d, d] or [d, d], updated in
    place) from the summed gsum [k, d*d] and count [k]."""
    k = int(count.shape[0])
    d = int(z.shape[-1])
    ctx.check(ctx.lib.pd_barycenter_apply(ctx.handle, _ptr(z), k, d, _ptr(gsum), _ptr(count), float(gamma),
                                          float(lam), _stream(stream)))
    return z


def pd_kmeans_assign(ctx: Context, hist, mass, params: SinkhornParams, centroids, want_cost=False, stream=None):
    """Assignment of N histograms to the k centroids (float64 CUDA tensor
    [k, d, d]).  Returns (assign [N] int32, objective [1] float64, cost [N, k]
    float64 or None) as CUDA tensors."""
    import torch
    N, k = int(hist.shape[0]), int(centroids.shape[0])
    assign = torch.empty(N, dtype=torch.int32, device=hist.device)
    obj = torch.empty(1, dtype=torch.float64, device=hist.device)
    cost = torch.empty((N, k), dtype=torch.float64, device=hist.device) if want_cost else None
    ctx.check(ctx.lib.pd_kmeans_assign(ctx.handle, _ptr(hist), _ptr(mass), N, k, ctypes.byref(params),
                                       _ptr(centroids), _ptr(assign), _ptr(cost), _ptr(obj), _stream(stream)))
    return assign, obj, cost


def pd_kmeans(ctx: Context, hist, mass, k: int, params: SinkhornParams, lam: float, rounds: int, bary_steps: int,
              seed: int = 0, stream=None):
    """k-means on N histograms.  Returns (assign [N] int32, centroids [k,d,d]
    float64, objective [rounds] float64) as CUDA tensors."""
    import torch
    d, N = params.d, int(hist.shape[0])
    assign = torch.empty(N, dtype=torch.int32, device=hist.device)
    cent = torch.empty((k, d, d), dtype=torch.float64, device=hist.device)
    obj = torch.empty(max(rounds, 1), dtype=torch.float64, device=hist.device)
    ctx.check(ctx.lib.pd_kmeans(ctx.handle, _ptr(hist), _ptr(mass), N, int(k), ctypes.byref(params), float(lam),
                                int(rounds), int(bary_steps), ctypes.c_uint64(seed), _ptr(assign), _ptr(cent),
                                _ptr(obj), _stream(stream)))
    return assign, cent, obj[:rounds]


def pd_sinkhorn_batch_noalloc(histA, massA, histB, massB, params: SinkhornParams, pairs=None, g_init=None,
                              out=None, stream=None):
    """The allocation-free solve (see include/pd_ot.h): same arguments as
    pd_sinkhorn_batch but no context; output tensors must be supplied in `out`
    (cost, iters, err, status; optional row_marg, col_marg, f, g) by callers
    that cannot allocate.  Raises PdError on a non-PD_OK status."""
    lib = load()
    P = pairs.shape[0] if pairs is not None else histA.shape[0]
    o = dict(out)
    st = lib.pd_sinkhorn_batch_noalloc(
        _ptr(histA), _ptr(massA), _ptr(histB), _ptr(massB), _ptr(pairs), int(P), ctypes.byref(params),
        _ptr(g_init), _ptr(o["cost"]), _ptr(o.get("row_marg")), _ptr(o.get("col_marg")), _ptr(o.get("f")),
        _ptr(o.get("g")), _ptr(o["iters"]), _ptr(o["err"]), _ptr(o["status"]), _stream(stream))
    if st != PD_OK:
        raise PdError(st, "pd_sinkhorn_batch_noalloc failed")
    return o


# --------------------------------------------------------------------------- serving
def serve_default_config(**overrides) -> ServeConfig:
    """pd_serve_default_config, then the given fields (slots as a 4-sequence)."""
    cfg = ServeConfig()
    load().pd_serve_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "slots":
            for i, x in enumerate(v):
                cfg.slots[i] = int(x)
        else:
            setattr(cfg, k, v)
    return cfg


class Server:
    """pd_server: continuous-batching request loop (pd_serve_* in the C ABI)."""

    def __init__(self, ctx: Context, cfg: ServeConfig | None = None, **overrides):
        self.lib = ctx.lib
        self.ctx = ctx
        cfg = cfg if cfg is not None else serve_default_config(**overrides)
        h = _vp()
        st = self.lib.pd_serve_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h))
        if st != PD_OK:
            raise PdError(st, "pd_serve_create failed")
        self.handle = h

    def load_centroids(self, d: int, z):
        """z: CUDA float64 tensor [k, d*d] (or [k, d, d]) of centroid weights."""
        import torch
        z = z.reshape(z.shape[0], d * d).to(torch.float64).contiguous()
        st = self.lib.pd_serve_load_centroids(self.handle, int(d), _ptr(z), int(z.shape[0]))
        torch.cuda.synchronize()
        if st != PD_OK:
            raise PdError(st, "pd_serve_load_centroids failed")

    def _submit(self, kind, d, ba, da, bb=None, db=None) -> int:
        import numpy as np
        ba = np.ascontiguousarray(ba, dtype=np.float64)
        da = np.ascontiguousarray(da, dtype=np.float64)
        q = Query(kind, int(d), ba.ctypes.data, da.ctypes.data, int(ba.size), None, None, 0)
        if bb is not None:
            bb = np.ascontiguousarray(bb, dtype=np.float64)
            db = np.ascontiguousarray(db, dtype=np.float64)
            q.birth_b_host, q.death_b_host, q.n_b = bb.ctypes.data, db.ctypes.data, int(bb.size)
        t = ctypes.c_uint64()
        st = self.lib.pd_serve_submit(self.handle, ctypes.byref(q), ctypes.byref(t))
        if st != PD_OK:
            raise PdError(st, "pd_serve_submit failed")
        return t.value

    def submit_distance(self, d, birth_a, death_a, birth_b, death_b) -> int:
        return self._submit(PD_Q_DISTANCE, d, birth_a, death_a, birth_b, death_b)

    def submit_nearest(self, d, birth, death) -> int:
        return self._submit(PD_Q_NEAREST, d, birth, death)

    @staticmethod
    def _as_dict(r: Result):
        return {"status": r.status, "cost": r.cost, "centroid": r.centroid, "iters": r.iters,
                "latency_ms": r.latency_ms}

    def poll(self, ticket: int):
        """None while pending, else the result dict (the ticket is released)."""
        r = Result()
        st = self.lib.pd_serve_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(r))
        if st == PD_PENDING:
            return None
        if st == PD_ERR_INVALID and r.status == 0 and r.latency_ms == 0:
            raise PdError(st, f"unknown ticket {ticket}")
        return self._as_dict(r)

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        r = Result()
        st = self.lib.pd_serve_wait(self.handle, ctypes.c_uint64(ticket), ctypes.byref(r), float(timeout_ms))
        if st == PD_PENDING:
            return None
        if st == PD_ERR_INVALID and r.status == 0 and r.latency_ms == 0:
            raise PdError(st, f"unknown ticket {ticket}")
        return self._as_dict(r)

    def inject_failure(self):
        st = self.lib.pd_serve_inject_failure(self.handle)
        if st != PD_OK:
            raise PdError(st, "pd_serve_inject_failure failed")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.pd_serve_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
