"""The allocation-free solve, pd_sinkhorn_batch_noalloc, for callers that may
not allocate device memory (applications whose pool allocator owns the device
memory, latency-critical threads that cannot take an allocation's device-wide
synchronisation).  Called through the C ABI with caller-owned buffers, it must give the
same results as pd_sinkhorn_batch on two calls in a row (the second call reuses
the static workspace the first one left behind), and refuse batches that do not
fit its fixed workspace.  Collected last so that a failure here does not stop a
-x run before the other tests."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1805_08331_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _problem(ctx, seed, d, P):
    b, t, o = inputs.random_diagrams(2 * P, nmin=30, nmax=200, seed=seed)
    hist, mass = api.pd_rasterize(ctx, torch.from_numpy(b).cuda(), torch.from_numpy(t).cuda(),
                                  torch.from_numpy(o).cuda(), d)
    pairs = torch.arange(2 * P, dtype=torch.int32, device="cuda").view(P, 2).contiguous()
    return hist, mass, pairs


def _outputs(P, n):
    return {"cost": torch.empty(P, dtype=torch.float64, device="cuda"),
            "iters": torch.empty(P, dtype=torch.int32, device="cuda"),
            "err": torch.empty(P, dtype=torch.float32, device="cuda"),
            "status": torch.empty(P, dtype=torch.int32, device="cuda"),
            "row_marg": torch.empty((P, n), dtype=torch.float32, device="cuda"),
            "f": torch.empty((P, n), dtype=torch.float64, device="cuda")}


def test_noalloc_matches_pd_sinkhorn_batch_on_two_calls():
    lib = api.load(build_if_missing=True)
    ctx = api.Context(0)
    try:
        for seed, d, P, gamma, every in ((3, 64, 6, 5e-3, 0), (4, 128, 4, 1e-3, 16)):
            hist, mass, pairs = _problem(ctx, seed, d, P)
            prm = api.pd_sinkhorn_default_params(gamma, d, max_iter=3000, tol=1e-6)
            prm.absorb_every = every   # a non-default parameter reaches both entry points alike
            ref = api.pd_sinkhorn_batch(ctx, hist, mass, hist, mass, prm, pairs=pairs, want_marginals=True,
                                        want_potentials=True)
            out = _outputs(P, d * d + 1)
            st = lib.pd_sinkhorn_batch_noalloc(
                ctypes.c_void_p(hist.data_ptr()), ctypes.c_void_p(mass.data_ptr()), ctypes.c_void_p(hist.data_ptr()),
                ctypes.c_void_p(mass.data_ptr()), ctypes.c_void_p(pairs.data_ptr()), P, ctypes.byref(prm), None,
                ctypes.c_void_p(out["cost"].data_ptr()), ctypes.c_void_p(out["row_marg"].data_ptr()), None,
                ctypes.c_void_p(out["f"].data_ptr()), None, ctypes.c_void_p(out["iters"].data_ptr()),
                ctypes.c_void_p(out["err"].data_ptr()), ctypes.c_void_p(out["status"].data_ptr()),
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert st == api.PD_OK
            torch.cuda.synchronize()
            c_ref, c = ref["cost"].cpu().numpy(), out["cost"].cpu().numpy()
            assert np.all(np.abs(c - c_ref) <= 1e-6 * np.abs(c_ref))
            assert np.array_equal(out["iters"].cpu().numpy(), ref["iters"].cpu().numpy())
            assert np.array_equal(out["status"].cpu().numpy(), ref["status"].cpu().numpy())
            assert np.allclose(out["row_marg"].cpu().numpy(), ref["row_marg"].cpu().numpy(), rtol=1e-6, atol=1e-7)
            fr, fo = ref["f"].cpu().numpy(), out["f"].cpu().numpy()
            fin = np.isfinite(fr)
            assert np.array_equal(fin, np.isfinite(fo)) and np.allclose(fo[fin], fr[fin], rtol=0, atol=1e-9)
    finally:
        ctx.close()


def test_noalloc_rejects_batches_beyond_its_workspace():
    ctx = api.Context(0)
    try:
        hist, mass, pairs = _problem(ctx, 5, 128, 64)
        prm = api.pd_sinkhorn_default_params(1e-3, 128, max_iter=10, tol=0.0)
        with pytest.raises(api.PdError) as e:
            api.pd_sinkhorn_batch_noalloc(hist, mass, hist, mass, prm, pairs=pairs, out=_outputs(64, 128 * 128 + 1))
        assert e.value.status == api.PD_ERR_INVALID
        # the gamma-continuation is not run by this entry point: refused, not ignored
        prm.eps_stages = 2
        with pytest.raises(api.PdError) as e:
            api.pd_sinkhorn_batch_noalloc(hist[:2], mass[:2], hist[:2], mass[:2], prm, pairs=pairs[:1],
                                          out=_outputs(1, 128 * 128 + 1))
        assert e.value.status == api.PD_ERR_INVALID
    finally:
        ctx.close()
