"""ctypes wrapper of the FP64 C oracle (``pd_oracle.c``).  TEST INFRASTRUCTURE.

Every function here only marshals arguments; the arithmetic is in the C file,
each C function citing the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libpd_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile pd_oracle.c into a shared library next to it (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.or_rasterize.argtypes = [_dp, _dp, _i64p, ctypes.c_int, ctypes.c_int, _u32p, _u32p]
            lib.or_cost.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.or_cost.restype = ctypes.c_double
            lib.or_sinkhorn_w.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int,
                                          ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp,
                                          ctypes.POINTER(ctypes.c_int), _dp]
            lib.or_sinkhorn_pd_batch.argtypes = [ctypes.c_int, ctypes.c_double, _u32p, _u32p,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                 _dp, _dp, _dp, _dp, _dp, ctypes.POINTER(ctypes.c_int), _dp]
            lib.or_sinkhorn_pd_batchp.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _u32p, _u32p,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                  _dp, _dp, _dp, _dp, _dp, ctypes.POINTER(ctypes.c_int), _dp]
            lib.or_sinkhorn_wp.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, ctypes.c_int,
                                           ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp,
                                           ctypes.POINTER(ctypes.c_int), _dp]
            lib.or_cost_p.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int]
            lib.or_cost_p.restype = ctypes.c_double
            lib.or_barycenter.argtypes = [ctypes.c_int, ctypes.c_double, _u32p, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          _dp, _dp, _dp]
            lib.or_barycenter_s.argtypes = [ctypes.c_int, ctypes.c_double, _u32p, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            _dp, _dp, _dp, ctypes.c_int]
            lib.or_barycenter_e.argtypes = [ctypes.c_int, ctypes.c_double, _u32p, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            _dp, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_int)]
            lib.or_sharpen.argtypes = [ctypes.c_int, _dp, ctypes.c_double]
            lib.or_sharpen.restype = ctypes.c_double
            lib.or_kmeans.argtypes = [ctypes.c_int, ctypes.c_double, _u32p, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_uint64, _i32p, _dp, _dp]
            lib.or_round_bound.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                           _dp, _dp]
            lib.or_ctransform_bound.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp]
            lib.or_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(t)


def num_threads() -> int:
    return int(_load().or_num_threads())


def rasterize(birth, death, offsets, d):
    """Rasterise B diagrams (CSR: points offsets[b]..offsets[b+1]) on a d x d grid.
    Returns (hist uint32 [B,d,d], mass uint32 [B])."""
    birth = np.ascontiguousarray(birth, dtype=np.float64)
    death = np.ascontiguousarray(death, dtype=np.float64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    B = len(offsets) - 1
    hist = np.zeros((B, d, d), dtype=np.uint32)
    mass = np.zeros(B, dtype=np.uint32)
    rc = _load().or_rasterize(_ptr(birth, _dp), _ptr(death, _dp), _ptr(offsets, _i64p), B, d,
                              _ptr(hist, _u32p), _ptr(mass, _u32p))
    if rc != 0:
        raise ValueError("or_rasterize: invalid point (need finite 0 <= birth <= death <= 1)")
    return hist, mass


def cost(d, x, y, p=2.0):
    """Entry C_xy of the augmented cost (index d*d is the Delta bin), ground cost ||.||_p^p."""
    if p == 2.0:
        return float(_load().or_cost(d, int(x), int(y)))
    return float(_load().or_cost_p(d, float(p), int(x), int(y)))


def augment(hA, hB):
    """Prop. 1 augmentation of two histograms: a = (hA, |B|), b = (hB, |A|)."""
    hA = np.asarray(hA, dtype=np.float64).ravel()
    hB = np.asarray(hB, dtype=np.float64).ravel()
    return np.concatenate([hA, [hB.sum()]]), np.concatenate([hB, [hA.sum()]])


def sinkhorn_w(d, gamma, a, b, max_iter, tol, g_init=None, p=2.0):
    """Log-domain FP64 Sinkhorn on the explicit augmented cost (weights a, b of
    length d*d+1; ground cost ||.||_p^p).  Returns a dict with cost, f, g,
    rmarg, cmarg, iters, err."""
    n = d * d + 1
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    assert a.shape == (n,) and b.shape == (n,)
    gi = None if g_init is None else np.ascontiguousarray(g_init, dtype=np.float64)
    c = ctypes.c_double()
    it = ctypes.c_int()
    er = ctypes.c_double()
    f = np.empty(n)
    g = np.empty(n)
    rm = np.empty(n)
    cm = np.empty(n)
    rc = _load().or_sinkhorn_wp(d, float(p), gamma, _ptr(a, _dp), _ptr(b, _dp), int(max_iter), float(tol),
                               _ptr(gi, _dp), ctypes.byref(c), _ptr(f, _dp), _ptr(g, _dp),
                               _ptr(rm, _dp), _ptr(cm, _dp), ctypes.byref(it), ctypes.byref(er))
    if rc != 0:
        raise ValueError("or_sinkhorn_w: invalid weights (negative or unequal total mass)")
    return dict(cost=c.value, f=f, g=g, rmarg=rm, cmarg=cm, iters=it.value, err=er.value)


def round_bound(d, gamma, a, b, f, g):
    """Rounded plan of P(f, g) onto Pi(a, b) and its cost <R, C> (Prop. 3's
    upper bound), on the dense matrices.  a, b, f, g: length d*d+1."""
    n = d * d + 1
    arr = [np.ascontiguousarray(x, dtype=np.float64) for x in (a, b, f, g)]
    assert all(x.shape == (n,) for x in arr)
    out = [ctypes.c_double() for _ in range(5)]
    rc = _load().or_round_bound(d, gamma, *[_ptr(x, _dp) for x in arr], *[ctypes.byref(o) for o in out])
    if rc != 0:
        raise ValueError("or_round_bound: d > 64")
    return dict(upper=out[0].value, row_dev=out[1].value, col_dev=out[2].value, er=out[3].value, ec=out[4].value)


def ctransform_bound(d, gamma, a, b, f):
    """Lower bound m_t = <alpha^cc, a> + <alpha^c, b> with alpha = f + gamma log a."""
    n = d * d + 1
    arr = [np.ascontiguousarray(x, dtype=np.float64) for x in (a, b, f)]
    assert all(x.shape == (n,) for x in arr)
    out = ctypes.c_double()
    _load().or_ctransform_bound(d, gamma, *[_ptr(x, _dp) for x in arr], ctypes.byref(out))
    return out.value


def sinkhorn_pd(d, gamma, hA, hB, max_iter, tol, g_init=None, p=2.0):
    """Alg. 1 for one pair of d x d histograms (Prop. 1 augmentation)."""
    a, b = augment(hA, hB)
    return sinkhorn_w(d, gamma, a, b, max_iter, tol, g_init, p=p)


def sinkhorn_pd_batch(d, gamma, hA, hB, max_iter, tol, want_potentials=False, want_marginals=False, p=2.0):
    """Alg. 1 over P pairs (OpenMP over pairs).  hA, hB: uint32 [P,d,d]."""
    hA = np.ascontiguousarray(hA, dtype=np.uint32)
    hB = np.ascontiguousarray(hB, dtype=np.uint32)
    P = hA.shape[0]
    n = d * d + 1
    cost_ = np.empty(P)
    it = np.empty(P, dtype=np.int32)
    er = np.empty(P)
    f = np.empty((P, n)) if want_potentials else None
    g = np.empty((P, n)) if want_potentials else None
    rm = np.empty((P, n)) if want_marginals else None
    cm = np.empty((P, n)) if want_marginals else None
    rc = _load().or_sinkhorn_pd_batchp(d, float(p), gamma, _ptr(hA, _u32p), _ptr(hB, _u32p), P, int(max_iter),
                                      float(tol), _ptr(cost_, _dp), _ptr(f, _dp), _ptr(g, _dp),
                                      _ptr(rm, _dp), _ptr(cm, _dp),
                                      it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(er, _dp))
    if rc != 0:
        raise ValueError("or_sinkhorn_pd_batch failed")
    return dict(cost=cost_, iters=it, err=er, f=f, g=g, rmarg=rm, cmarg=cm)


def sharpen(d, z, H0):
    """Entropic sharpening of z (d x d) to entropy H0; returns (z', beta)."""
    z = np.ascontiguousarray(z, dtype=np.float64).ravel().copy()
    beta = _load().or_sharpen(d, _ptr(z, _dp), float(H0))
    return z.reshape(d, d), beta


def barycenter(d, gamma, hists, lam, outer_iters, max_iter, tol, z_init=None, sharpen=False,
               rel_energy_tol=0.0):
    """Alg. 2 (optionally with entropic sharpening after every step, and with
    the stop |E_t/E_{t-1} - 1| < rel_energy_tol after step t >= 1).
    hists: uint32 [N,d,d].  Returns (z [d,d], energy [steps run])."""
    hists = np.ascontiguousarray(hists, dtype=np.uint32)
    N = hists.shape[0]
    zi = None if z_init is None else np.ascontiguousarray(z_init, dtype=np.float64).ravel()
    z = np.empty(d * d)
    e = np.empty(max(outer_iters, 1))
    steps = ctypes.c_int(0)
    rc = _load().or_barycenter_e(d, gamma, _ptr(hists, _u32p), N, float(lam), int(outer_iters),
                                 int(max_iter), float(tol), _ptr(zi, _dp), _ptr(z, _dp), _ptr(e, _dp),
                                 1 if sharpen else 0, float(rel_energy_tol), ctypes.byref(steps))
    if rc != 0:
        raise ValueError("or_barycenter failed")
    return z.reshape(d, d), e[:steps.value]


def kmeans(d, gamma, hists, k, lam, rounds, bary_steps, max_iter, tol, seed):
    """k-means on diagrams.  Returns (assign [N], centroids [k,d,d], objective [rounds])."""
    hists = np.ascontiguousarray(hists, dtype=np.uint32)
    N = hists.shape[0]
    assign = np.empty(N, dtype=np.int32)
    cent = np.empty((k, d, d))
    obj = np.empty(rounds)
    rc = _load().or_kmeans(d, gamma, _ptr(hists, _u32p), N, k, float(lam), int(rounds),
                           int(bary_steps), int(max_iter), float(tol), ctypes.c_uint64(seed),
                           _ptr(assign, _i32p), _ptr(cent, _dp), _ptr(obj, _dp))
    if rc != 0:
        raise ValueError("or_kmeans failed")
    return assign, cent, obj
