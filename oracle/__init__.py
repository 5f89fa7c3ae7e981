"""FP64 CPU oracle for entropic OT between persistence diagrams.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package; the CUDA
library (``paper_1805_08331_gb300``) never does, and this package imports
nothing from it.  The arithmetic lives in ``pd_oracle.c`` (plain C, FP64);
this module builds it with gcc and marshals numpy arrays through ctypes.
"""
from .oracle import (build, rasterize, cost, sinkhorn_w, sinkhorn_pd, sinkhorn_pd_batch,
                     barycenter, kmeans, num_threads, augment, round_bound, ctransform_bound, sharpen)

__all__ = ["build", "rasterize", "cost", "sinkhorn_w", "sinkhorn_pd", "sinkhorn_pd_batch",
           "barycenter", "kmeans", "num_threads", "augment", "round_bound", "ctransform_bound", "sharpen"]
