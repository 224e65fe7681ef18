"""The C ABI on the CPU: the library builds, loads and exports every symbol
include/sng.h declares (no compute without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sng.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sng_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_boundary():
    names = _declared()
    for want in ("sng_build_graph", "sng_cluster", "sng_cluster_batched", "sng_graph_free",
                 "sng_strerror"):
        assert want in names


def test_library_exports_every_declared_symbol():
    import paper_2006_06743_gb300 as sng
    sng.build()
    lib = ctypes.CDLL(sng.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(sng.SIGNATURES)


def test_binding_loads_and_reports_without_gpu():
    import paper_2006_06743_gb300 as sng
    sng.build()
    L = sng.lib()
    assert L.sng_strerror(0) == b"ok"
    assert L.sng_strerror(-1) == b"invalid argument"
    assert sng.launch_count() >= 0


def test_invalid_params_rejected_on_host():
    """Validation happens before any CUDA call, so it works without a GPU."""
    import paper_2006_06743_gb300 as sng
    sng.build()
    p = sng.Params(eps=-1.0, min_pts=3, s=0.1).to_c(100, 3, 3, sng.SNG_F32)
    st = sng.sng_stats()
    rc = sng.lib().sng_cluster(ctypes.c_void_p(256), ctypes.byref(p), ctypes.c_void_p(256), None,
                               ctypes.byref(st), None)
    assert rc == sng.SNG_EINVAL
    assert "eps" in sng.last_error()
