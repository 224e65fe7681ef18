"""FP64 CPU oracle for SNG-DBSCAN -- test infrastructure, not part of the product.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The CUDA library never calls it,
and it imports nothing from ``paper_2006_06743_gb300``: the two sides share no
kernels, headers, helpers or constants.  Seeded inputs come from
``paper_2006_06743_gb300.datagen`` (random inputs only, none of the method's
arithmetic), which tests hand to both sides.

Contents
  * ``sng_oracle.c`` (built here with gcc, FP64, ``-ffp-contract=off``):
    Algorithm 1 of Jiang, Jang & Lacki (NeurIPS 2020), Section 3 -- partner
    draws, the sampled eps-graph, degrees, core mask, core components (BFS and
    union-find), border labels -- plus textbook brute-force DBSCAN.
  * ``ari``: the adjusted Rand index of Hubert & Arabie (1985), the score the
    paper's Section 5 evaluates clusterings with.
  * ``ami``: the adjusted mutual information of Vinh, Epps & Bailey (2010),
    the paper's second score, with its expected mutual information summed
    over every term of the hypergeometric model.
  * ``mlp``: FP64 forward/backward/Adam for the core-point surrogate network;
    ``gate_decisions``: the rule by which that network gates the points.

Parity status per function is listed in each docstring; every function here is
pinned by a ``-m "not gpu"`` test against something other than itself.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sng_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_OMP_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp_lib = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile ``sng_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, FP64,
    no contraction, no fast-math), or with ``openmp`` the same source with
    -fopenmp into ``liboracle_omp.so`` (the multi-core CPU baseline).
    Rebuilds when the source is newer."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    path = _OMP_LIB_PATH if openmp else _LIB_PATH
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared"] + (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


class _Graph(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("num_edges", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("col", ctypes.POINTER(ctypes.c_int32)), ("band_pairs", ctypes.c_int64)]


def _load(openmp: bool = False):
    global _lib, _omp_lib
    with _lock:
        if openmp and _omp_lib is not None:
            return _omp_lib
        if not openmp and _lib is not None:
            return _lib
        lib = ctypes.CDLL(build(openmp=openmp))
        P = ctypes.c_void_p
        i64, i32, u64, f32, f64 = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                   ctypes.c_float, ctypes.c_double)
        lib.orc_mix64.argtypes = [u64]
        lib.orc_mix64.restype = u64
        lib.orc_partner.argtypes = [u64, i64, i64, i64, i32]
        lib.orc_partner.restype = i64
        lib.orc_partners.argtypes = [u64, i64, i64, i64, i64, i32, P]
        lib.orc_partners.restype = None
        lib.orc_dist2.argtypes = [P, P, i32]
        lib.orc_dist2.restype = f64
        lib.orc_build_rows.argtypes = [i64, i32, i64, P, f32, u64, i64, i32, f64, P, i64,
                                       ctypes.POINTER(_Graph), P]
        lib.orc_build_rows.restype = i32
        lib.orc_build_rows_m.argtypes = [i64, i32, i64, P, f32, u64, i64, i32, f64, P, i64,
                                         ctypes.POINTER(_Graph), P, P]
        lib.orc_build_rows_m.restype = i32
        lib.orc_build_rows_metric.argtypes = [i64, i32, i64, P, f32, u64, i64, i32, f64, P, i64,
                                              ctypes.POINTER(_Graph), P, P, i32]
        lib.orc_build_rows_metric.restype = i32
        lib.orc_dot.argtypes = [P, P, i32]
        lib.orc_dot.restype = f64
        lib.orc_cosine.argtypes = [P, P, i32]
        lib.orc_cosine.restype = f64
        lib.orc_l1.argtypes = [P, P, i32]
        lib.orc_l1.restype = f64
        lib.orc_linf.argtypes = [P, P, i32]
        lib.orc_linf.restype = f64
        lib.orc_cluster_graph_forced.argtypes = [i64, P, P, i32, i32, P, P, P, P, P]
        lib.orc_cluster_graph_forced.restype = i32
        lib.orc_cluster_graph_gated.argtypes = [i64, P, P, i32, i32, P, P, P, P, P, P]
        lib.orc_cluster_graph_gated.restype = i32
        lib.orc_graph_free.argtypes = [ctypes.POINTER(_Graph)]
        lib.orc_graph_free.restype = None
        lib.orc_degrees.argtypes = [i64, P, P, i32, P]
        lib.orc_degrees.restype = i32
        lib.orc_components_bfs.argtypes = [i64, P, P, P, P]
        lib.orc_components_bfs.restype = i64
        lib.orc_components_uf.argtypes = [i64, P, P, P, P]
        lib.orc_components_uf.restype = i64
        lib.orc_border_labels.argtypes = [i64, P, P, P, P, P]
        lib.orc_border_labels.restype = None
        lib.orc_cluster_graph.argtypes = [i64, P, P, i32, i32, P, P, P, P]
        lib.orc_cluster_graph.restype = i32
        lib.orc_cluster.argtypes = [i64, i32, i64, P, f32, u64, i64, i32, i32, i32, f64, P, P,
                                    P, P, P]
        lib.orc_cluster.restype = i32
        lib.orc_cluster_metric.argtypes = [i64, i32, i64, P, f32, u64, i64, i32, i32, i32, f64,
                                           P, P, P, P, P, i32]
        lib.orc_cluster_metric.restype = i32
        lib.orc_dbscan_bruteforce.argtypes = [i64, i32, i64, P, f32, i32, P, P]
        lib.orc_dbscan_bruteforce.restype = i32
        lib.orc_build_rows_blocks.argtypes = [i64, i32, i64, P, f32, u64, i64, i32, f64, i64,
                                              i64, ctypes.POINTER(_Graph)]
        lib.orc_build_rows_blocks.restype = i32
        lib.orc_threads.argtypes = []
        lib.orc_threads.restype = i32
        if openmp:
            _omp_lib = lib
        else:
            _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32_rows(x) -> tuple[np.ndarray, int, int, int]:
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim != 2:
        raise ValueError("x must be 2-D (n, d)")
    return x, x.shape[0], x.shape[1], x.shape[1]


# ------------------------------------------------------------------ hash

def mix64(z: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood 2014).  Pinned by the
    generator's published output vectors."""
    return int(_load().orc_mix64(ctypes.c_uint64(z & (2**64 - 1))))


def partner(seed: int, i: int, j: int, n: int, sample_all: bool = False) -> int:
    """Partner j of point i (Algorithm 1, step 2), never i itself."""
    return int(_load().orc_partner(seed & (2**64 - 1), i, j, n, int(sample_all)))


def partners(seed: int, n: int, i0: int, ni: int, m: int, sample_all: bool = False) -> np.ndarray:
    """All partners of rows i0..i0+ni-1 as an (ni, m) int64 array."""
    out = np.empty((ni, m), dtype=np.int64)
    _load().orc_partners(seed & (2**64 - 1), n, i0, ni, m, int(sample_all), _ptr(out))
    return out


def dist2(a, b) -> float:
    """FP64 squared distance, summed left to right without fused operations."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(_load().orc_dist2(_ptr(a), _ptr(b), a.size))


# neighbourhood tests: Euclidean ball, inner product, cosine similarity
METRIC_L2, METRIC_DOT, METRIC_COSINE, METRIC_L1, METRIC_LINF = 0, 1, 2, 3, 4


def dot(a, b) -> float:
    """FP64 inner product, products and sums left to right, unfused."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(_load().orc_dot(_ptr(a), _ptr(b), a.size))


def cosine(a, b) -> float:
    """FP64 cosine similarity <a,b> / (sqrt(<a,a>) sqrt(<b,b>)); NaN when
    either vector is zero."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(_load().orc_cosine(_ptr(a), _ptr(b), a.size))


def l1(a, b) -> float:
    """FP64 Manhattan distance: differences, absolute values and sums left to
    right; NaN when a difference is NaN."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(_load().orc_l1(_ptr(a), _ptr(b), a.size))


def linf(a, b) -> float:
    """FP64 Chebyshev distance (largest |a_k - b_k|); NaN when a difference
    is NaN."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(_load().orc_linf(_ptr(a), _ptr(b), a.size))


# ------------------------------------------------------------ graph build

def build_rows(x, eps: float, seed: int, m: int, sample_all: bool = False,
               band_rel: float = 1e-5, rows=None, m_row=None, metric: int = METRIC_L2):
    """Algorithm 1, step 2 for the given rows (default all).  ``m_row`` (int32
    per point) limits point i to its first m_row[i] draws (surrogate form).
    ``metric``: METRIC_L2 (edge iff d2 <= eps^2), METRIC_DOT / METRIC_COSINE
    (edge iff similarity >= eps), METRIC_L1 / METRIC_LINF (edge iff the
    Manhattan / Chebyshev distance <= eps).

    Returns ``(row_ptr int64[nr+1], col int32[E], band_pairs, band_point uint8[n])``.
    """
    x, n, d, ld = _f32_rows(x)
    lib = _load()
    g = _Graph()
    bp = np.zeros(n, dtype=np.uint8)
    if rows is None:
        rows_arr, nr, rp = None, n, None
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        nr, rp = rows_arr.size, _ptr(rows_arr)
    mr = None if m_row is None else np.ascontiguousarray(m_row, dtype=np.int32)
    rc = lib.orc_build_rows_metric(n, d, ld, _ptr(x), ctypes.c_float(eps), seed & (2**64 - 1),
                                   m, int(sample_all), band_rel, rp, nr, ctypes.byref(g),
                                   _ptr(bp), _ptr(mr) if mr is not None else None, metric)
    if rc != 0:
        raise ValueError("orc_build_rows failed (bad arguments or out of memory)")
    try:
        row_ptr = np.ctypeslib.as_array(g.row_ptr, shape=(g.n_rows + 1,)).copy()
        ne = int(g.num_edges)
        col = (np.ctypeslib.as_array(g.col, shape=(ne,)).copy() if ne
               else np.zeros(0, dtype=np.int32))
        band_pairs = int(g.band_pairs)
    finally:
        lib.orc_graph_free(ctypes.byref(g))
    return row_ptr, col, band_pairs, bp


def build_rows_blocks(x, eps: float, seed: int, m: int, block: int = 4096,
                      openmp: bool = False, n_rows: int | None = None
                      ) -> tuple[np.ndarray, np.ndarray, int]:
    """Step 2 over the source rows 0..n_rows-1 (default all) in blocks of
    consecutive rows joined in order (the same graph as ``build_rows``); with
    ``openmp`` the blocks run on all host cores (the liboracle_omp.so build of
    the same source).  Returns ``(row_ptr, col, band_pairs)``."""
    x, n, d, ld = _f32_rows(x)
    nr = n if n_rows is None else int(n_rows)
    lib = _load(openmp)
    g = _Graph()
    if lib.orc_build_rows_blocks(n, d, ld, _ptr(x), ctypes.c_float(eps), seed & (2**64 - 1), m,
                                 0, 1e-5, block, nr, ctypes.byref(g)) != 0:
        raise ValueError("orc_build_rows_blocks failed (bad arguments or out of memory)")
    try:
        row_ptr = np.ctypeslib.as_array(g.row_ptr, shape=(nr + 1,)).copy()
        ne = int(g.num_edges)
        col = (np.ctypeslib.as_array(g.col, shape=(ne,)).copy() if ne
               else np.zeros(0, dtype=np.int32))
        return row_ptr, col, int(g.band_pairs)
    finally:
        lib.orc_graph_free(ctypes.byref(g))


def threads(openmp: bool = True) -> int:
    """Host threads the OpenMP build uses (1 for the plain build)."""
    return int(_load(openmp).orc_threads())


def degrees(n: int, row_ptr, col, mode: int = 0) -> np.ndarray:
    """Vertex degrees (Algorithm 1, step 3); mode 0 undirected multigraph,
    1 out-degree, 2 distinct neighbours."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    deg = np.empty(n, dtype=np.int32)
    if _load().orc_degrees(n, _ptr(rp), _ptr(cl), mode, _ptr(deg)) != 0:
        raise ValueError("orc_degrees failed")
    return deg


def components(n: int, row_ptr, col, core, method: str = "bfs") -> tuple[np.ndarray, int]:
    """Components of the core subgraph (Algorithm 1, step 3); label = min index."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    cr = np.ascontiguousarray(core, dtype=np.uint8)
    comp = np.empty(n, dtype=np.int32)
    fn = _load().orc_components_bfs if method == "bfs" else _load().orc_components_uf
    k = fn(n, _ptr(rp), _ptr(cl), _ptr(cr), _ptr(comp))
    if k < 0:
        raise MemoryError("oracle components: out of memory")
    return comp, int(k)


def border_labels(n: int, row_ptr, col, core, comp) -> np.ndarray:
    """Algorithm 1, steps 4-5 (border points take the smallest adjacent label)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    cr = np.ascontiguousarray(core, dtype=np.uint8)
    cp = np.ascontiguousarray(comp, dtype=np.int32)
    labels = np.empty(n, dtype=np.int32)
    _load().orc_border_labels(n, _ptr(rp), _ptr(cl), _ptr(cr), _ptr(cp), _ptr(labels))
    return labels


def cluster_graph(n: int, row_ptr, col, min_pts: int, deg_mode: int = 0, forced=None,
                  w_row=None) -> dict:
    """Algorithm 1, steps 3-5 on a given sampled graph (CSR by source).
    ``forced`` (uint8 per point: 1 core, 2 not core, 0 by degree) overrides
    the core test and ``w_row`` (int32 per point) weights each kept draw of
    a row (surrogate form; min_pts is then in the weights' units)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    fc = None if forced is None else np.ascontiguousarray(forced, dtype=np.uint8)
    wr = None if w_row is None else np.ascontiguousarray(w_row, dtype=np.int32)
    labels = np.empty(n, dtype=np.int32)
    core = np.empty(n, dtype=np.uint8)
    deg = np.empty(n, dtype=np.int32)
    stats = np.zeros(8, dtype=np.int64)
    if _load().orc_cluster_graph_gated(n, _ptr(rp), _ptr(cl), deg_mode, min_pts,
                                       _ptr(fc) if fc is not None else None,
                                       _ptr(wr) if wr is not None else None, _ptr(labels),
                                       _ptr(core), _ptr(deg), _ptr(stats)) != 0:
        raise MemoryError("orc_cluster_graph failed")
    return dict(labels=labels, core=core, deg=deg, kept_edges=int(stats[1]),
                cores=int(stats[4]), clusters=int(stats[5]), noise=int(stats[6]))


def cluster(x, eps: float, seed: int, m: int, min_pts: int, deg_mode: int = 0,
            sample_all: bool = False, band_rel: float = 1e-5, metric: int = METRIC_L2) -> dict:
    """The whole of Algorithm 1 in FP64.  Returns labels (int32, -1 noise, else
    the smallest core index of the cluster), core mask, degrees, band points
    and the counters (queries, kept edges, band pairs/points, cores, clusters,
    noise)."""
    x, n, d, ld = _f32_rows(x)
    labels = np.empty(n, dtype=np.int32)
    core = np.empty(n, dtype=np.uint8)
    deg = np.empty(n, dtype=np.int32)
    bp = np.zeros(n, dtype=np.uint8)
    stats = np.zeros(8, dtype=np.int64)
    rc = _load().orc_cluster_metric(n, d, ld, _ptr(x), ctypes.c_float(eps), seed & (2**64 - 1),
                                    m, int(sample_all), deg_mode, min_pts, band_rel,
                                    _ptr(labels), _ptr(core), _ptr(deg), _ptr(bp), _ptr(stats),
                                    metric)
    if rc != 0:
        raise ValueError("orc_cluster failed (bad arguments or out of memory)")
    return dict(labels=labels, core=core, deg=deg, band_point=bp, queries=int(stats[0]),
                kept_edges=int(stats[1]), band_pairs=int(stats[2]), band_points=int(stats[3]),
                cores=int(stats[4]), clusters=int(stats[5]), noise=int(stats[6]))


def cluster_gated(x, eps: float, seed: int, m: int, min_pts: int, forced, m_row,
                  deg_mode: int = 0, w_row=None, deg_unit: int = 16) -> dict:
    """The surrogate-gated form of Algorithm 1: point i draws its first
    m_row[i] partners, and forced[i] (1 core, 2 not core, 0 by degree)
    overrides the core test; with ``w_row`` each kept draw of row i counts
    w_row[i] / deg_unit in the degree.  Steps 3-5 as in the plain form."""
    rp, col, _, _ = build_rows(x, eps, seed, m, m_row=m_row)
    mp = min_pts * deg_unit if w_row is not None else min_pts
    r = cluster_graph(np.asarray(x).shape[0], rp, col, mp, deg_mode=deg_mode, forced=forced,
                      w_row=w_row)
    r["queries"] = int(np.minimum(np.asarray(m_row, dtype=np.int64), m).sum())
    return r


GATE_DEG_UNIT = 16   # degree units per kept draw when the gate reweights


def gate_decisions(prob, m: int, p_noise: float, p_core: float, core_draw_frac: float,
                   noise_draw_frac: float = 0.0, reweight: bool = False,
                   deg_unit: int = GATE_DEG_UNIT, by_degree: bool = False):
    """The surrogate gate's rule (an extension; the paper has no learned part):
    a point whose core probability is below ``p_noise`` is declared not core
    and draws the first ceil(noise_draw_frac * m) partners of its stream; one
    above ``p_core`` is declared core and draws ceil(core_draw_frac * m);
    every other point draws all m and is tested by its degree (both
    comparisons strict).  Thresholds and fractions are read as the float32
    values the caller passes.  With ``reweight`` each kept draw of a point
    that drew m_i partners counts round(deg_unit * m / m_i) degree units (an
    unbiased estimate of its full count; deg_unit when m_i = 0).

    With ``by_degree`` the gate sets only the draw budgets (and weights):
    every point keeps the degree test, so nothing is forced.

    Returns forced (uint8: 0 by degree, 1 core, 2 not core), draws per point
    (int32) and the per-point weights (int32, or None without reweighting).
    Pinned by the hand-worked cases of tests/golden/gate_rule.txt."""
    prob = np.asarray(prob, dtype=np.float64).ravel()
    lo = float(np.float32(p_noise))
    hi = float(np.float32(p_core))
    forced = np.zeros(prob.size, dtype=np.uint8)
    forced[prob > hi] = 1
    forced[prob < lo] = 2
    m_core = int(math.ceil(float(np.float32(core_draw_frac)) * m))
    m_noise = int(math.ceil(float(np.float32(noise_draw_frac)) * m))
    draws = {0: m, 1: m_core, 2: m_noise}
    m_row = np.array([draws[int(f)] for f in range(3)], dtype=np.int32)[forced]
    cls = forced
    if by_degree:
        forced = np.zeros_like(forced)
    if not reweight:
        return forced, m_row, None

    def weight(mi: int) -> int:
        if mi <= 0:
            return deg_unit
        return int(math.floor(deg_unit * m / mi + 0.5))

    w = np.array([weight(draws[f]) for f in range(3)], dtype=np.int32)
    return forced, m_row, w[cls]


def dbscan_bruteforce(x, eps: float, min_pts_db: int) -> tuple[np.ndarray, np.ndarray]:
    """Textbook DBSCAN (Ester et al. 1996) from all n^2 FP64 distances; the
    neighbourhood counts the point itself; border -> smallest adjacent label."""
    x, n, d, ld = _f32_rows(x)
    labels = np.empty(n, dtype=np.int32)
    core = np.empty(n, dtype=np.uint8)
    if _load().orc_dbscan_bruteforce(n, d, ld, _ptr(x), ctypes.c_float(eps), min_pts_db,
                                     _ptr(labels), _ptr(core)) != 0:
        raise MemoryError("orc_dbscan_bruteforce failed")
    return labels, core


# --------------------------------------------------------------- metrics

def ari(a, b) -> float:
    """Adjusted Rand index (Hubert & Arabie 1985) from the contingency table,
    in FP64 (exact integer pair counts).  Noise (-1) is one label."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    if a.shape != b.shape:
        raise ValueError("label arrays differ in length")
    n = a.size
    if n < 2:
        return 1.0
    _, ia = np.unique(a, return_inverse=True)
    _, ib = np.unique(b, return_inverse=True)
    pair = ia.astype(np.int64) * (int(ib.max()) + 1) + ib
    _, nij = np.unique(pair, return_counts=True)
    ai = np.bincount(ia)
    bj = np.bincount(ib)

    def c2(v):
        v = np.asarray(v, dtype=np.int64)
        return int(np.sum(v * (v - 1) // 2))

    index = c2(nij)
    sa, sb = c2(ai), c2(bj)
    total = n * (n - 1) // 2
    expected = sa * sb / total
    max_index = 0.5 * (sa + sb)
    if max_index == expected:
        return 1.0
    return float((index - expected) / (max_index - expected))


def canonical(labels) -> np.ndarray:
    """Relabel a partition so every cluster carries its smallest point index
    (noise stays -1)."""
    labels = np.asarray(labels)
    out = np.full(labels.shape, -1, dtype=np.int64)
    mask = labels >= 0
    idx = np.nonzero(mask)[0]
    if idx.size:
        lab = labels[mask]
        first = {}
        for i, l in zip(idx.tolist(), lab.tolist()):
            if l not in first:
                first[l] = i
        out[mask] = np.array([first[l] for l in lab.tolist()], dtype=np.int64)
    return out


def _contingency(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    if a.shape != b.shape:
        raise ValueError("label arrays differ in length")
    _, ia = np.unique(a, return_inverse=True)
    _, ib = np.unique(b, return_inverse=True)
    table = np.zeros((int(ia.max()) + 1, int(ib.max()) + 1), dtype=np.int64)
    np.add.at(table, (ia, ib), 1)
    return table


def entropy(counts, n: int) -> float:
    """H = -sum_i (a_i/n) log(a_i/n) over the clusters of one labelling."""
    c = np.asarray(counts, dtype=np.float64)
    c = c[c > 0]
    return float(-np.sum(c / n * np.log(c / n)))


def mutual_info(table) -> float:
    """MI = sum_ij (n_ij/n) log(n n_ij / (a_i b_j)) over the non-empty cells of
    the contingency table (natural logarithm)."""
    t = np.asarray(table, dtype=np.int64)
    n = float(t.sum())
    a = t.sum(axis=1).astype(np.float64)
    b = t.sum(axis=0).astype(np.float64)
    i, j = np.nonzero(t)
    c = t[i, j].astype(np.float64)
    return float(np.sum(c / n * np.log(n * c / (a[i] * b[j]))))


def expected_mutual_info(a_counts, b_counts, n: int) -> float:
    """E[MI] when the labels of one side are permuted uniformly at random (the
    hypergeometric model of Vinh, Epps & Bailey 2010): for every pair of
    cluster sizes (a, b), sum over every feasible cell count k >= 1 of
    (k/n) log(n k / (a b)) times the hypergeometric probability of k, the
    latter from log-gamma values."""
    from scipy.special import gammaln
    total = 0.0
    lg_n = gammaln(n + 1.0)
    for a in np.asarray(a_counts, dtype=np.int64):
        for b in np.asarray(b_counts, dtype=np.int64):
            lo, hi = max(1, a + b - n), min(a, b)
            if lo > hi:
                continue
            k = np.arange(lo, hi + 1, dtype=np.float64)
            logp = (gammaln(a + 1.0) + gammaln(b + 1.0) + gammaln(n - a + 1.0)
                    + gammaln(n - b + 1.0) - lg_n - gammaln(k + 1.0) - gammaln(a - k + 1.0)
                    - gammaln(b - k + 1.0) - gammaln(n - a - b + k + 1.0))
            total += float(np.sum(k / n * np.log(n * k / (float(a) * float(b))) * np.exp(logp)))
    return total


AMI_AVERAGES = ("min", "geometric", "arithmetic", "max")


def ami(a, b, average: str = "arithmetic") -> dict:
    """Adjusted mutual information (MI - E[MI]) / (avg(H_a, H_b) - E[MI]),
    avg one of min / geometric / arithmetic / max (Vinh, Epps & Bailey 2010).
    Two trivial labellings of the same kind (both one cluster, or both all
    singletons) score 1; a vanishing normaliser otherwise scores 0.  Noise
    (-1) is one label.  Returns the score and its terms."""
    t = _contingency(a, b)
    n = int(t.sum())
    ra, rb = t.sum(axis=1), t.sum(axis=0)
    ha, hb = entropy(ra, n), entropy(rb, n)
    mi = mutual_info(t)
    emi = expected_mutual_info(ra, rb, n)
    out = dict(mi=mi, emi=emi, h_a=ha, h_b=hb)
    if (ra.size == 1 and rb.size == 1) or (ra.size == n and rb.size == n):
        return dict(out, ami=1.0)
    norm = {"min": min(ha, hb), "geometric": float(np.sqrt(ha * hb)),
            "arithmetic": 0.5 * (ha + hb), "max": max(ha, hb)}[average]
    den = norm - emi
    if den <= 0.0:
        return dict(out, ami=0.0)
    return dict(out, ami=(mi - emi) / den)
