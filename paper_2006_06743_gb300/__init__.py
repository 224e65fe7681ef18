"""GB300 (sm_103a) SNG-DBSCAN: Python binding of libsng.so.

SNG-DBSCAN (Jiang, Jang & Lacki, NeurIPS 2020, Algorithm 1) clusters points
from a subsampled eps-neighbourhood graph: every point draws ceil(s n) random
partners, keeps the partners within eps, and DBSCAN's core / component / border
steps run on that sparse graph.  All of it runs in this package's CUDA kernels
behind the C ABI of ``include/sng.h``; this module only marshals arguments
(ctypes over plain pointers) and uses PyTorch for device memory and streams.
There is no CPU fallback: if the compiled library is missing, every call
raises.

Raw entry points carry the C names (``sng_cluster``, ``sng_build_graph``,
``sng_cluster_batched`` ...).  ``cluster`` / ``build_graph`` / ``ari`` are the
tensor-level conveniences most callers want.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsng.so")

SNG_OK, SNG_EINVAL, SNG_ENOMEM, SNG_ECUDA, SNG_ETIMEOUT, SNG_EINTERNAL = 0, -1, -2, -3, -4, -5
SNG_F32, SNG_BF16 = 0, 1
SNG_DEG_UNDIRECTED_MULTI, SNG_DEG_OUT, SNG_DEG_SIMPLE = 0, 1, 2
SNG_METRIC_L2, SNG_METRIC_DOT, SNG_METRIC_COSINE = 0, 1, 2
SNG_METRIC_L1, SNG_METRIC_LINF = 3, 4
SNG_SAMPLE_HASH, SNG_SAMPLE_ALL = 0, 1
SNG_FLAG_TIMING = 1
SNG_FLAG_PREFETCH = 2
SNG_FLAG_NO_SYNC = 4
SNG_FLAG_WARP_ROWS = 8
SNG_FLAG_TILED = 16
SNG_FLAG_SCREEN16 = 32
SNG_FLAG_SCREEN_MMA = 64
SNG_FLAG_TCGEN05 = 128
SNG_FLAG_SCREEN8 = 256

PHASES = ("gather", "scan", "fill", "core_union", "labels", "finalize", "total", "gate")


class SngError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class sng_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("ld", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("degree_mode", ctypes.c_int32),
                ("sample_mode", ctypes.c_int32), ("min_pts", ctypes.c_int32),
                ("eps", ctypes.c_float), ("band_rel", ctypes.c_float), ("s", ctypes.c_double),
                ("m_override", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("x_f32_master", ctypes.c_void_p), ("flags", ctypes.c_uint32),
                ("map_group", ctypes.c_int32), ("map_unroll", ctypes.c_int32),
                ("map_block", ctypes.c_int32), ("map_tile", ctypes.c_int32),
                ("map_passes", ctypes.c_int32), ("metric", ctypes.c_int32),
                ("row_begin", ctypes.c_int64), ("row_end", ctypes.c_int64),
                ("counters_out", ctypes.c_void_p)]


class sng_mi_terms(ctypes.Structure):
    _fields_ = [("ami", ctypes.c_double), ("mi", ctypes.c_double), ("emi", ctypes.c_double),
                ("h_a", ctypes.c_double), ("h_b", ctypes.c_double),
                ("clusters_a", ctypes.c_int64), ("clusters_b", ctypes.c_int64)]


AMI_AVERAGES = {"min": 0, "geometric": 1, "arithmetic": 2, "max": 3}


class sng_stats(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_int64), ("kept_edges", ctypes.c_int64),
                ("band_pairs", ctypes.c_int64), ("band_points", ctypes.c_int64),
                ("cores", ctypes.c_int64), ("clusters", ctypes.c_int64),
                ("noise", ctypes.c_int64), ("recheck_pairs", ctypes.c_int64),
                ("surrogate_core", ctypes.c_int64), ("surrogate_noise", ctypes.c_int64),
                ("ms", ctypes.c_float * 8), ("map_vec", ctypes.c_int32),
                ("map_group", ctypes.c_int32), ("map_nch", ctypes.c_int32),
                ("map_unroll", ctypes.c_int32), ("map_tiles", ctypes.c_int32),
                ("map_tex", ctypes.c_int32), ("map_screen", ctypes.c_int32),
                ("screen_pairs", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "ms"}
        d["ms"] = {PHASES[i]: float(self.ms[i]) for i in range(len(PHASES))}
        return d


class sng_mlp_config(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("hidden", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("adam_eps", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("sequential", ctypes.c_int32), ("fp32_activations", ctypes.c_int32)]


class sng_gate(ctypes.Structure):
    _fields_ = [("p_noise", ctypes.c_float), ("p_core", ctypes.c_float),
                ("core_draw_frac", ctypes.c_float), ("noise_draw_frac", ctypes.c_float),
                ("reweight", ctypes.c_int32), ("by_degree", ctypes.c_int32)]


class sng_graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("num_edges", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("deg", ctypes.c_void_p),
                ("core", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes); every symbol include/sng.h declares
_P = ctypes.c_void_p
SIGNATURES = {
    "sng_build_graph": (ctypes.c_int32, [_P, ctypes.POINTER(sng_params),
                                         ctypes.POINTER(sng_graph), ctypes.POINTER(sng_stats), _P]),
    "sng_graph_free": (None, [ctypes.POINTER(sng_graph)]),
    "sng_cluster": (ctypes.c_int32, [_P, ctypes.POINTER(sng_params), _P, _P,
                                     ctypes.POINTER(sng_stats), _P]),
    "sng_cluster_host": (ctypes.c_int32, [_P, ctypes.POINTER(sng_params), _P, _P,
                                          ctypes.POINTER(sng_stats), _P]),
    "sng_cluster_edges": (ctypes.c_int32, [ctypes.c_int64, _P, _P, ctypes.c_int64, _P,
                                           ctypes.POINTER(sng_params), _P, _P,
                                           ctypes.POINTER(sng_stats), _P]),
    "sng_cluster_batched": (ctypes.c_int32, [_P, _P, ctypes.c_int32, ctypes.POINTER(sng_params),
                                             _P, _P, ctypes.POINTER(sng_stats), _P]),
    "sng_batch_plan_create": (ctypes.c_int32, [_P, ctypes.c_int32, ctypes.POINTER(sng_params),
                                               _P, ctypes.POINTER(ctypes.c_void_p)]),
    "sng_batch_run": (ctypes.c_int32, [_P, _P, _P, ctypes.POINTER(sng_stats), _P]),
    "sng_batch_plan_destroy": (None, [_P]),
    "sng_sample_partners": (ctypes.c_int32, [ctypes.c_int64, ctypes.c_uint64, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _P, _P]),
    "sng_ari": (ctypes.c_int32, [_P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), _P]),
    "sng_ami": (ctypes.c_int32, [_P, _P, ctypes.c_int64, ctypes.c_int32,
                                 ctypes.POINTER(sng_mi_terms), _P]),
    "sng_mlp_param_count": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int32]),
    "sng_mlp_standardize": (ctypes.c_int32, [_P, ctypes.c_int64, ctypes.c_int32, _P, _P]),
    "sng_mlp_loss_grad": (ctypes.c_int32, [_P, _P, ctypes.c_int64, ctypes.POINTER(sng_mlp_config),
                                           _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "sng_mlp_train": (ctypes.c_int32, [_P, _P, ctypes.c_int64, ctypes.POINTER(sng_mlp_config),
                                       _P, _P, _P, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "sng_mlp_predict": (ctypes.c_int32, [_P, ctypes.c_int64, ctypes.POINTER(sng_mlp_config), _P,
                                         _P, _P]),
    "sng_cluster_surrogate": (ctypes.c_int32, [_P, ctypes.POINTER(sng_params),
                                               ctypes.POINTER(sng_mlp_config), _P,
                                               ctypes.POINTER(sng_gate), _P, _P,
                                               ctypes.POINTER(sng_stats), _P]),
    "sng_cluster_noalloc": (ctypes.c_int32, [_P, ctypes.POINTER(sng_params), _P,
                                             ctypes.POINTER(sng_stats), _P]),
    "sng_gather_mapping": (ctypes.c_int32, [_P, ctypes.POINTER(sng_params), _P]),
    "sng_measure_random_rows": (ctypes.c_int32, [ctypes.c_int64, ctypes.c_int32,
                                                 ctypes.c_int64, ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_double), _P]),
    "sng_measure_l2_read": (ctypes.c_int32, [ctypes.c_int64, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_double), _P]),
    "sng_launch_count": (ctypes.c_int64, []),
    "sng_last_error": (ctypes.c_char_p, []),
    "sng_strerror": (ctypes.c_char_p, [ctypes.c_int32]),
}


def lib():
    """Load libsng.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def _check(status: int):
    if status != SNG_OK:
        msg = lib().sng_last_error().decode(errors="replace")
        raise SngError(status, msg or lib().sng_strerror(status).decode())


def last_error() -> str:
    return lib().sng_last_error().decode(errors="replace")


def launch_count() -> int:
    return int(lib().sng_launch_count())


# ------------------------------------------------------------------ params

@dataclass
class Params:
    """Python mirror of ``sng_params`` (see include/sng.h)."""
    eps: float
    min_pts: int
    s: float = 0.0
    m: int = 0                  # > 0 overrides ceil(s n)
    seed: int = 0
    degree_mode: int = SNG_DEG_UNDIRECTED_MULTI
    sample_mode: int = SNG_SAMPLE_HASH
    band_rel: float = 0.0
    flags: int = 0
    map_group: int = 0
    map_unroll: int = 0
    map_block: int = 0
    map_tile: int = 0
    map_passes: int = 0
    row_begin: int = 0
    row_end: int = 0
    metric: int = 0             # SNG_METRIC_*: 0 Euclidean ball, 1 inner product, 2 cosine,
                                # 3 Manhattan, 4 Chebyshev distance

    def to_c(self, n: int, d: int, ld: int, dtype: int, master_ptr: int = 0) -> sng_params:
        p = sng_params()
        p.n, p.d, p.ld, p.dtype = n, d, ld, dtype
        p.degree_mode, p.sample_mode, p.min_pts = self.degree_mode, self.sample_mode, self.min_pts
        p.eps, p.band_rel, p.s, p.m_override = self.eps, self.band_rel, self.s, self.m
        p.seed = self.seed & (2**64 - 1)
        p.x_f32_master = master_ptr or None
        p.flags = self.flags
        p.map_group, p.map_unroll, p.map_block = self.map_group, self.map_unroll, self.map_block
        p.map_tile = self.map_tile
        p.map_passes = self.map_passes
        p.row_begin, p.row_end = self.row_begin, self.row_end
        p.metric = self.metric
        return p

    def draws(self, n: int) -> int:
        if self.sample_mode == SNG_SAMPLE_ALL:
            return n - 1
        if self.m > 0:
            return self.m
        return int(math.ceil(self.s * n))


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _rows(x, dtype: int):
    """(n, d, ld) of a 2-D CUDA tensor whose rows may be padded (stride >= d)."""
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("x must be a CUDA tensor")
    if x.dim() != 2 or x.stride(1) != 1:
        raise ValueError("x must be 2-D with unit stride in the last dimension")
    want = torch.float32 if dtype == SNG_F32 else torch.bfloat16
    if x.dtype != want:
        raise TypeError(f"x must be {want} for this dtype")
    return x.shape[0], x.shape[1], x.stride(0)


# -------------------------------------------------------------- calls

def sng_cluster(x_ptr: int, params: sng_params, labels_ptr: int, core_ptr: int = 0,
                stream: int = 0) -> dict:
    st = sng_stats()
    _check(lib().sng_cluster(x_ptr, ctypes.byref(params), labels_ptr, core_ptr or None,
                             ctypes.byref(st), stream or None))
    return st.as_dict()


def cluster(x, params: Params, x_master=None, want_core: bool = False, stream=None):
    """Algorithm 1 on the rows of ``x`` (CUDA float32, or bfloat16 with the
    float32 ``x_master`` for the FP64 recheck).  Returns ``(labels, stats)``
    or ``(labels, core, stats)``; labels are int32 on the device, -1 = noise,
    else the smallest core index of the cluster."""
    import torch
    dtype = SNG_BF16 if x.dtype == torch.bfloat16 else SNG_F32
    n, d, ld = _rows(x, dtype)
    mp = 0
    if dtype == SNG_BF16:
        if x_master is None or x_master.dtype != torch.float32 or x_master.stride(0) != ld:
            raise ValueError("bf16 input needs a float32 x_master with the same row stride")
        mp = x_master.data_ptr()
    labels = torch.empty(n, dtype=torch.int32, device=x.device)
    core = torch.empty(n, dtype=torch.uint8, device=x.device) if want_core else None
    st = sng_cluster(x.data_ptr(), params.to_c(n, d, ld, dtype, mp), labels.data_ptr(),
                     core.data_ptr() if core is not None else 0, _stream_ptr(stream))
    return (labels, core, st) if want_core else (labels, st)


def cluster_host(x, params: Params, x_master=None, want_core: bool = False, stream=None):
    """Algorithm 1 on HOST points (a C-contiguous float32 numpy array or CPU
    tensor, ideally pinned; bfloat16 CPU tensor with a float32 ``x_master``):
    the library copies them to the device, clusters, and copies the labels
    back.  Returns ``(labels, stats)`` or ``(labels, core, stats)`` as numpy
    arrays."""
    import numpy as np
    import torch
    t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))
    if t.is_cuda or t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("cluster_host takes a 2-D host array with unit column stride")
    dtype = SNG_BF16 if t.dtype == torch.bfloat16 else SNG_F32
    if dtype == SNG_F32 and t.dtype != torch.float32:
        raise ValueError("points must be float32 or bfloat16")
    n, d, ld = t.shape[0], t.shape[1], t.stride(0)
    mp = 0
    if dtype == SNG_BF16:
        if x_master is None or x_master.dtype != torch.float32 or x_master.stride(0) != ld:
            raise ValueError("bf16 input needs a float32 host x_master with the same row stride")
        mp = x_master.data_ptr()
    labels = np.empty(n, dtype=np.int32)
    core = np.empty(n, dtype=np.uint8) if want_core else None
    st = sng_stats()
    _check(lib().sng_cluster_host(t.data_ptr(), ctypes.byref(params.to_c(n, d, ld, dtype, mp)),
                                  labels.ctypes.data,
                                  core.ctypes.data if core is not None else None,
                                  ctypes.byref(st), _stream_ptr(stream)))
    return (labels, core, st.as_dict()) if want_core else (labels, st.as_dict())


def cluster_async(x, params: Params, labels, counters=None, core=None, stream=None):
    """Algorithm 1 without any host synchronisation inside the call
    (SNG_FLAG_NO_SYNC), so the call can be captured in a CUDA graph: labels
    (int32, n) and core (uint8, n, optional) are caller-owned CUDA tensors
    written when the stream reaches them; ``counters`` (int64 CUDA tensor of
    9, optional) receives [0] 0, [1] band pairs, [2] rechecks, [3] band
    points, [4] cores, [5] clusters, [6] noise, [7] kept draws and [8] the
    device status bits.  FP32 points only."""
    import torch
    dtype = SNG_BF16 if x.dtype == torch.bfloat16 else SNG_F32
    if dtype != SNG_F32:
        raise ValueError("cluster_async takes float32 points")
    n, d, ld = _rows(x, dtype)
    c = params.to_c(n, d, ld, dtype, 0)
    c.flags = (c.flags | SNG_FLAG_NO_SYNC) & ~SNG_FLAG_TIMING
    c.counters_out = counters.data_ptr() if counters is not None else None
    _check(lib().sng_cluster(x.data_ptr(), ctypes.byref(c), labels.data_ptr(),
                             core.data_ptr() if core is not None else None, None,
                             _stream_ptr(stream)))
    return labels


def sng_build_graph(x_ptr: int, params: sng_params, stream: int = 0):
    g = sng_graph()
    st = sng_stats()
    _check(lib().sng_build_graph(x_ptr, ctypes.byref(params), ctypes.byref(g), ctypes.byref(st),
                                 stream or None))
    return g, st.as_dict()


def build_graph(x, params: Params, x_master=None, stream=None) -> dict:
    """Algorithm 1, step 2 (+ degrees and core mask): CSR graph copied into
    torch tensors (row_ptr int64, col int32, deg int32, core uint8)."""
    import torch
    dtype = SNG_BF16 if x.dtype == torch.bfloat16 else SNG_F32
    n, d, ld = _rows(x, dtype)
    mp = x_master.data_ptr() if dtype == SNG_BF16 else 0
    g, st = sng_build_graph(x.data_ptr(), params.to_c(n, d, ld, dtype, mp), _stream_ptr(stream))
    try:
        dev = x.device
        out = {}
        for name, count, tdt, ts in (("row_ptr", n + 1, torch.int64, "<i8"),
                                     ("col", int(g.num_edges), torch.int32, "<i4"),
                                     ("deg", n, torch.int32, "<i4"), ("core", n, torch.uint8, "|u1")):
            out[name] = _copy_out(getattr(g, name) or 0, count, ts, tdt, dev)
        torch.cuda.synchronize(dev)
    finally:
        lib().sng_graph_free(ctypes.byref(g))
    out["stats"] = st
    out["m"] = int(g.m)
    return out


class _DeviceArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _copy_out(ptr: int, count: int, typestr: str, dtype, device):
    import torch
    if count == 0 or not ptr:
        return torch.empty(count, dtype=dtype, device=device)
    return torch.as_tensor(_DeviceArray(ptr, count, typestr), device=device).clone()


def cluster_edges(n: int, src, col, deg, params: Params, want_core: bool = False, stream=None):
    """Algorithm 1, steps 3-5 on a given graph: kept draws src[e] -> col[e]
    (int32 CUDA tensors) and degrees deg (int32, n; None with the simple-graph
    degree, which is computed from the edges).  Returns (labels[, core],
    stats)."""
    import torch
    dev = src.device
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    core = torch.empty(n, dtype=torch.uint8, device=dev) if want_core else None
    st = sng_stats()
    E = int(src.numel())
    _check(lib().sng_cluster_edges(n, src.data_ptr() if E else None,
                                   col.data_ptr() if E else None, E,
                                   deg.data_ptr() if deg is not None else None,
                                   ctypes.byref(params.to_c(n, 1, 1, SNG_F32)), labels.data_ptr(),
                                   core.data_ptr() if core is not None else None,
                                   ctypes.byref(st), _stream_ptr(stream)))
    d = st.as_dict()
    return (labels, core, d) if want_core else (labels, d)


def sample_partners(n: int, seed: int, i0: int, rows: int, m: int, sample_all: bool = False,
                    stream=None):
    """Partner draws of rows i0..i0+rows-1 as an int32 (rows, m) CUDA tensor."""
    import torch
    out = torch.empty((rows, m), dtype=torch.int32, device="cuda")
    _check(lib().sng_sample_partners(n, seed & (2**64 - 1), i0, rows, m, int(sample_all),
                                     out.data_ptr(), _stream_ptr(stream)))
    return out


def ami(a, b, average: str = "arithmetic", stream=None) -> dict:
    """Adjusted mutual information of two int32 CUDA label tensors (values in
    [-1, n)) with its terms: ami, mi, emi, h_a, h_b, clusters_a, clusters_b."""
    t = sng_mi_terms()
    _check(lib().sng_ami(a.data_ptr(), b.data_ptr(), a.numel(), AMI_AVERAGES[average],
                         ctypes.byref(t), _stream_ptr(stream)))
    return {k: getattr(t, k) for k, _ in t._fields_}


def measure_l2_read(bytes_: int = 48 << 20, passes: int = 200, stream=None) -> float:
    """GB/s the SMs read from an L2-resident buffer (the library's own probe
    kernel; see sng_measure_l2_read)."""
    v = ctypes.c_double()
    _check(lib().sng_measure_l2_read(int(bytes_), int(passes), ctypes.byref(v),
                                     _stream_ptr(stream)))
    return float(v.value)


def measure_random_rows(n_rows: int, row_bytes: int = 128, fetches: int = 1 << 30,
                        blocks_per_sm: int = 0, stream=None) -> float:
    """Rows per second the SMs fetch at random from a buffer of n_rows rows
    (the library's own probe kernel; see sng_measure_random_rows)."""
    v = ctypes.c_double()
    _check(lib().sng_measure_random_rows(int(n_rows), int(row_bytes), int(fetches),
                                         int(blocks_per_sm), ctypes.byref(v),
                                         _stream_ptr(stream)))
    return float(v.value)


def ari(a, b, stream=None) -> float:
    """Adjusted Rand index of two int32 CUDA label tensors (values in [-1, n))."""
    v = ctypes.c_double()
    _check(lib().sng_ari(a.data_ptr(), b.data_ptr(), a.numel(), ctypes.byref(v),
                         _stream_ptr(stream)))
    return float(v.value)
