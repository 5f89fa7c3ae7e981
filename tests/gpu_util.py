"""Helpers shared by the GPU tests (marshalling only)."""
import numpy as np
import torch

from paper_1805_08331_gb300 import api


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def raster_gpu(ctx, b, t, o, d):
    hist, mass = api.pd_rasterize(ctx, dev(b), dev(t), dev(o), d)
    torch.cuda.synchronize()
    return hist, mass


def hists_to_gpu(h):
    return dev(np.asarray(h, dtype=np.uint32).view(np.int32))


def masses(h):
    return np.asarray(h, dtype=np.int64).reshape(h.shape[0], -1).sum(1).astype(np.uint32)
