"""Seeded synthetic persistence diagrams.

This module only draws random points; it holds none of the method's arithmetic
(no rasterisation, no cost, no transport).  Both the CUDA path and the oracle
are fed from it.  Diagrams are returned in CSR form: float64 ``birth``,
``death`` and int64 ``offsets`` (diagram b owns points offsets[b]..offsets[b+1]).

Workload shapes follow the paper's experiments (random diagrams with n..2n
points, Sec. 5 "A large scale approximation"; clustered diagrams standing in
for the 3D-shape diagrams of the k-means experiment, which are not available):

* ``random_diagrams``: birth ~ U[0,1), death = min(1, birth + Exp(mean)).
* ``mode_diagrams``: each mode is a few cluster centres in the upper triangle;
  a diagram of that mode scatters points around its centres with an isotropic
  Gaussian, resampling points until 0 <= birth < death <= 1.
"""
from __future__ import annotations

import math

import numpy as np


def _csr(points):
    counts = np.array([len(p[0]) for p in points], dtype=np.int64)
    offsets = np.zeros(len(points) + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    birth = np.concatenate([p[0] for p in points]) if points else np.zeros(0)
    death = np.concatenate([p[1] for p in points]) if points else np.zeros(0)
    return np.ascontiguousarray(birth, dtype=np.float64), np.ascontiguousarray(death, dtype=np.float64), offsets


def log_uniform_counts(rng, B, nmin, nmax):
    """floor(exp(U[ln nmin, ln nmax])) per diagram."""
    return np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=B))).astype(np.int64)


def random_diagrams(B, counts=None, nmin=20, nmax=20, exp_mean=0.2, seed=0, log_uniform=True):
    """B diagrams with birth ~ U[0,1), death = min(1, birth + Exp(exp_mean)).

    ``counts`` (array of B ints) overrides the point counts; otherwise counts are
    log-uniform in [nmin, nmax] (or uniform integers if ``log_uniform`` is False).
    """
    rng = np.random.default_rng(seed)
    if counts is None:
        if nmin == nmax:
            counts = np.full(B, nmin, dtype=np.int64)
        elif log_uniform:
            counts = log_uniform_counts(rng, B, nmin, nmax)
        else:
            counts = rng.integers(nmin, nmax + 1, size=B)
    pts = []
    for n in counts:
        s = rng.random(int(n))
        t = np.minimum(1.0, s + rng.exponential(exp_mean, int(n)))
        pts.append((s, t))
    return _csr(pts)


def mode_centres(n_modes, centres_per_mode=3, min_pers=0.15, seed=0):
    """Cluster centres (birth, death) per mode, death - birth >= min_pers."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_modes):
        cs = []
        while len(cs) < centres_per_mode:
            s, t = rng.random(2)
            s, t = min(s, t), max(s, t)
            if t - s >= min_pers and t <= 0.95 and s >= 0.05:
                cs.append((s, t))
        out.append(np.array(cs))
    return out


def mode_diagrams(N, n_modes, nmin, nmax, sigma=0.03, centres_per_mode=3, seed=0, labels=None):
    """N diagrams drawn from n_modes modes; returns (birth, death, offsets, labels).

    Point count ~ U{nmin..nmax}; each point picks one of its mode's centres
    uniformly and adds N(0, sigma^2 I), resampled until 0 <= birth < death <= 1.
    """
    rng = np.random.default_rng(seed)
    centres = mode_centres(n_modes, centres_per_mode, seed=seed + 7919)
    if labels is None:
        labels = np.arange(N) % n_modes
        rng.shuffle(labels)
    pts = []
    for lab in labels:
        n = int(rng.integers(nmin, nmax + 1))
        cs = centres[lab]
        s_all, t_all = [], []
        while len(s_all) < n:
            m = n - len(s_all)
            pick = rng.integers(0, len(cs), size=m)
            s = cs[pick, 0] + sigma * rng.standard_normal(m)
            t = cs[pick, 1] + sigma * rng.standard_normal(m)
            ok = (s >= 0) & (s < t) & (t <= 1)
            s_all.extend(s[ok].tolist())
            t_all.extend(t[ok].tolist())
        pts.append((np.array(s_all[:n]), np.array(t_all[:n])))
    b, t, o = _csr(pts)
    return b, t, o, np.asarray(labels, dtype=np.int32)


def poisson_queries(rate_hz, duration_s, grids=(32, 64, 128, 256), nmin=10, nmax=5000,
                    dist_fraction=0.5, seed=0):
    """Serving stream: arrival times (Poisson, ``rate_hz``), kind (0 = distance,
    1 = nearest centroid), grid size, and point counts (log-uniform)."""
    rng = np.random.default_rng(seed)
    n = rng.poisson(rate_hz * duration_s)
    t = np.sort(rng.uniform(0, duration_s, size=n))
    kind = (rng.random(n) >= dist_fraction).astype(np.int32)
    grid = rng.choice(np.asarray(grids, dtype=np.int32), size=n)
    counts = log_uniform_counts(rng, n, nmin, nmax)
    return t, kind, grid, counts
