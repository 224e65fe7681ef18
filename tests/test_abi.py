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


def _mapping(sng, d, ld, dtype, addr, **kw):
    master = 8192 if dtype == sng.SNG_BF16 else 0
    p = sng.Params(eps=0.5, min_pts=3, m=100, **kw).to_c(1000, d, ld, dtype, master)
    out = (ctypes.c_int32 * 7)()
    rc = sng.lib().sng_gather_mapping(ctypes.c_void_p(addr), ctypes.byref(p), out)
    return rc, list(out)


def test_default_mapping_is_compiled_for_every_shape():
    """The mapping rule must land on a compiled kernel for every row width the
    library accepts, for both element types and every row alignment (no GPU:
    the query only inspects the arguments)."""
    import paper_2006_06743_gb300 as sng
    sng.build()
    checked = 0
    for dtype, dmax, esize in ((sng.SNG_F32, 1024, 4), (sng.SNG_BF16, 2048, 2)):
        for d in list(range(1, 130)) + [255, 256, 257, 500, 512, 1000, 1024, 2000, 2048]:
            for pad in (0, 1, 3, 8):
                ld = d + pad
                for addr in (4096, 4096 + 2 * esize):
                    rc, m = _mapping(sng, d, ld, dtype, addr)
                    if rc != 0:
                        # only rows too wide for the compiled shapes may be refused
                        assert "wider" in sng.last_error(), (dtype, d, ld, addr, sng.last_error())
                        assert d > 256, (dtype, d, ld, addr)
                        continue
                    assert m[6] == 1, (dtype, d, ld, addr, m)
                    checked += 1
        # aligned rows up to the documented maximum always work
        rc, m = _mapping(sng, dmax, dmax, dtype, 4096)
        assert rc == 0 and m[6] == 1
    assert checked > 1500


def test_autotuner_candidates_are_compiled():
    import paper_2006_06743_gb300 as sng
    sng.build()
    for d, dtype in ((64, sng.SNG_F32), (128, sng.SNG_F32), (128, sng.SNG_BF16), (32, sng.SNG_F32),
                     (3, sng.SNG_F32)):
        ld = ((d + 3) // 4) * 4 if dtype == sng.SNG_F32 else ((d + 7) // 8) * 8
        g0 = 1
        n_ok = 0
        for g in (1, 2, 4, 8, 16, 32):
            for u in (1, 2, 4, 8):
                rc, m = _mapping(sng, d, ld, dtype, 4096, map_group=g, map_unroll=u)
                if rc == 0 and m[6] == 1:
                    n_ok += 1
        assert n_ok >= 4
