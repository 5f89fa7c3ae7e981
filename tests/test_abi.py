"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/pd_ot.h declares (no GPU needed: nothing is computed)."""
import ctypes
import os
import re

import pytest

from paper_1805_08331_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pd_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_the_binding_names():
    assert _declared() == set(api.EXPORTED)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_abi_version_and_params_defaults():
    lib = api.load()
    assert lib.pd_abi_version() == 3
    p = api.pd_sinkhorn_default_params(1e-3, 100)
    assert p.gamma == 1e-3 and p.d == 100 and p.max_iter == 20000 and p.tol == 1e-6
    assert p.precision == api.PD_FP32 and p.absorb_every == 64


def test_invalid_arguments_rejected_without_gpu():
    lib = api.load()
    # no context: every call reports PD_ERR_INVALID instead of crashing
    assert lib.pd_rasterize(None, None, None, None, 1, 8, None, None, None) == api.PD_ERR_INVALID
    p = api.pd_sinkhorn_default_params(1e-2, 8)
    assert lib.pd_sinkhorn_batch(None, None, None, None, None, None, 1, ctypes.byref(p),
                                 None, None, None, None, None, None, None, None, None, None) == api.PD_ERR_INVALID
    h = ctypes.c_void_p()
    st = lib.pd_ctx_create(-1, ctypes.byref(h))
    assert st == api.PD_ERR_INVALID


def test_workspace_query_host_arithmetic():
    """pd_workspace_query is host arithmetic (no GPU): linear in the number of
    pairs, the outer operations need more than their inner solves, and bad
    arguments are refused."""
    from paper_1805_08331_gb300 import api
    api.load(build_if_missing=True)
    p = api.pd_sinkhorn_default_params(1e-3, 128)
    s1 = api.pd_workspace_query(api.PD_OP_SINKHORN, p, 100)
    s2 = api.pd_workspace_query(api.PD_OP_SINKHORN, p, 200)
    assert s1 > 0 and abs((s2 - s1) - s1) <= 64 * 256   # grows by the per-pair part
    assert api.pd_workspace_query(api.PD_OP_SINKHORN, p, 0) == 0
    assert api.pd_workspace_query(api.PD_OP_BARYCENTER, p, 100) > s1
    assert api.pd_workspace_query(api.PD_OP_KMEANS, p, 100, 10) >= api.pd_workspace_query(api.PD_OP_SINKHORN, p, 1000)
    for op, n, k in ((99, 10, 1), (api.PD_OP_KMEANS, 10, 11), (api.PD_OP_BARYCENTER, 0, 0)):
        with pytest.raises(api.PdError):
            api.pd_workspace_query(op, p, n, k)
