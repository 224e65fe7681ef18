"""Autotuner for the gather mapping (and the batched form's tiling).

The gather's cost depends on how a warp is split over pairs (lanes per pair),
how many partner rows each warp keeps in flight, the block size and, for
point sets larger than L2, how many L2-resident slices of the partner range
the launch is split into, whether the L2-tiled form (draws bucketed by
source and partner slice, then tested tile by tile) beats the direct gather,
and, for FP32 points, whether testing pairs on a certified BF16 copy (with
CUDA-core sums or tensor-core dot products) pays.
The library picks a rule-of-thumb mapping; this
module times a small set of candidates on the caller's own data, through the
library's per-phase CUDA-event timers, and caches the fastest per
(dtype, d, row stride, n bucket, m bucket) in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import time

from . import (SNG_FLAG_PREFETCH, SNG_FLAG_SCREEN8, SNG_FLAG_SCREEN16, SNG_FLAG_SCREEN_MMA,
               SNG_FLAG_TCGEN05, SNG_FLAG_TILED,
               SNG_FLAG_TIMING, Params, SngError, cluster)

CACHE_ENV = "SNG_AUTOTUNE_CACHE"


def _cache_path(path: str | None) -> str:
    if path:
        return path
    if os.environ.get(CACHE_ENV):
        return os.environ[CACHE_ENV]
    return os.path.join(os.path.expanduser("~"), ".cache", "sng_gb300", "autotune.json")


def _bucket(v: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1, v)))))


def key_for(x, p: Params) -> str:
    n, d = x.shape
    key = (f"{str(x.dtype).replace('torch.', '')}-d{d}-ld{x.stride(0)}-n{_bucket(n)}"
           f"-m{_bucket(p.draws(n))}-mode{p.sample_mode}")
    return key + (f"-metric{p.metric}" if p.metric else "")


def _default_group(d: int, vec: int) -> int:
    chunks = -(-d // vec)
    g = 1
    while g < chunks and g < 32:
        g <<= 1
    return g


def candidates(x, p: Params, screen: bool = True) -> list[dict]:
    import torch
    n, d = x.shape
    if p.metric in (3, 4):
        # Manhattan / Chebyshev: the pair-kernel gather over a certified BF16
        # copy of FP32 points (2 bytes per value of scratch) where it fits,
        # and over the points themselves
        plain = dict(map_group=0, map_unroll=0, map_block=256, map_passes=0, prefetch=False)
        if screen and x.dtype == torch.float32:
            free = torch.cuda.mem_get_info(x.device)[0] if x.is_cuda else 0
            if n * (-(-d // 8) * 8) * 2 < 0.25 * free:
                return [dict(plain, screen=True), plain]
        return [plain]
    esize = 2 if x.dtype == torch.bfloat16 else 4
    vec = 8 if esize == 2 else 4
    if x.stride(0) % vec:
        vec = 1
    g0 = _default_group(d, vec)
    groups = sorted({g for g in (g0 // 8, g0 // 4, g0 // 2, g0, g0 * 2) if 1 <= g <= 32})
    x_bytes = n * x.stride(0) * esize
    passes = [1]
    if x_bytes > (48 << 20) and not p.metric:   # the similarity form runs in one pass
        base = max(2, int(math.ceil(x_bytes / (48 << 20))))
        passes += sorted({2, base, base + 2, 2 * base} - {1})
    out = []
    free = None
    # the certified BF16 screen of FP32 points (Euclidean, hashed draws): the
    # gather reads a BF16 copy (2 bytes per value of scratch), directly or
    # tiled with the slice count of the copy's size
    # (the similarity metrics: the tensor-core forms only)
    if screen and esize == 4 and p.sample_mode == 0 and (not p.metric or d <= 128):
        free = torch.cuda.mem_get_info(x.device)[0] if x.is_cuda else 0
        gb = _default_group(d, 8)
        ldb = -(-d // 8) * 8
        xb_bytes = n * ldb * 2
        if xb_bytes < 0.25 * free:
            if d <= 128:    # tensor-core dot products; map_unroll = blocks per SM budgeted
                for u in ((0, 4, 2) if d <= 64 else (0, 3)):
                    out.append(dict(map_group=0, map_unroll=u, map_block=256, map_passes=0,
                                    prefetch=False, screen=True, mma=True))
                # the FP8 copy (1 byte per value; more pairs left open)
                out.append(dict(map_group=0, map_unroll=0, map_block=256, map_passes=0,
                                prefetch=False, screen=True, fp8=True))
        if xb_bytes < 0.25 * free and not p.metric:   # the screen on CUDA cores
            for g in sorted({max(1, gb // 2), gb}):
                for u in (2, 4):
                    out.append(dict(map_group=g, map_unroll=u, map_block=256, map_passes=0,
                                    prefetch=False, screen=True))
        if (not p.metric and xb_bytes > (48 << 20)
                and 8.4 * n * p.draws(n) + xb_bytes < 0.5 * free):
            kb = min(32, max(2, -(-2 * xb_bytes // (88 << 20))))
            for k in sorted({kb, min(32, kb + 1)}):
                for g in sorted({0, gb}):
                    for u in (2, 4):
                        out.append(dict(map_group=g, map_unroll=u, map_block=256, map_passes=0,
                                        prefetch=False, tiled=True, map_tile=k, screen=True))
    # the L2-tiled form (Euclidean, hashed draws): its slice count from the
    # library's rule (two slices in about 88 MiB of L2) and one finer; it
    # needs ~8.4 bytes of scratch per draw, so it is tried only where that
    # leaves half the free memory
    if x_bytes > (48 << 20) and not p.metric and p.sample_mode == 0:
        if free is None:
            free = torch.cuda.mem_get_info(x.device)[0] if x.is_cuda else 0
        if 8.4 * n * p.draws(n) < 0.5 * free:
            k0 = min(32, max(2, -(-2 * x_bytes // (88 << 20))))
            for k in sorted({0, max(2, k0 // 2), min(32, k0 + 2)}):
                for u in (2, 4):
                    out.append(dict(map_group=0, map_unroll=u, map_block=256, map_passes=0,
                                    prefetch=False, tiled=True, map_tile=k))
    for ps in passes:
        for g in groups:
            for u in (1, 2, 4, 8):
                for b in (256, 128):
                    for pf in (False, True):
                        out.append(dict(map_group=g, map_unroll=u, map_block=b, map_passes=ps,
                                        prefetch=pf))
    return out


def _params_for(base: dict, cand: dict) -> Params:
    c = dict(cand)
    pf = c.pop("prefetch", False)
    tiled = c.pop("tiled", False)
    screen = c.pop("screen", False)
    mma = c.pop("mma", False)
    fp8 = c.pop("fp8", False)
    flags = base.get("flags", 0) & ~(SNG_FLAG_PREFETCH | SNG_FLAG_TILED | SNG_FLAG_SCREEN16 |
                                     SNG_FLAG_SCREEN_MMA | SNG_FLAG_SCREEN8 | SNG_FLAG_TCGEN05)
    if mma:
        flags |= SNG_FLAG_SCREEN_MMA
    if fp8:
        flags |= SNG_FLAG_SCREEN8
    if pf:
        flags |= SNG_FLAG_PREFETCH
    if screen:
        flags |= SNG_FLAG_SCREEN16
    if tiled:
        flags |= SNG_FLAG_TILED
    else:
        c.setdefault("map_tile", 0)
    return Params(**{**base, **c, "flags": flags})


def _time(x, p: Params, reps: int, x_master=None) -> float:
    import torch
    ms = []
    for _ in range(reps):
        _, st = cluster(x, p, x_master=x_master)
        ms.append(st["ms"]["gather"])
    torch.cuda.synchronize()
    return statistics.median(ms)


def tune(x, p: Params, x_master=None, reps: int = 3, budget_s: float = 60.0,
         cache: str | None = None, force: bool = False, verbose: bool = False,
         screen: bool = True) -> dict:
    """Fastest gather mapping for (x, p); returns the Params overrides and
    the timing table.  Results are cached per shape bucket.  ``screen``
    False leaves out the BF16 screen of FP32 points (the plain FP32 form)."""
    path = _cache_path(cache)
    key = key_for(x, p) + ("" if screen else "-noscreen")
    table = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if not force and key in table:
        return table[key]
    base = dict(p.__dict__)
    base["flags"] = base.get("flags", 0) | SNG_FLAG_TIMING
    results = []
    t_start = time.perf_counter()
    for cand in candidates(x, p, screen=screen):
        if time.perf_counter() - t_start > budget_s:
            break
        q = _params_for(base, cand)
        try:
            _time(x, q, 1, x_master)            # warm-up
            t = _time(x, q, reps, x_master)
        except SngError as e:                   # mapping not compiled for this shape
            if verbose:
                print("skip", cand, e)
            continue
        results.append((t, cand))
        if verbose:
            print(f"{t:9.3f} ms  {cand}")
    if not results:
        return {"mapping": {}, "gather_ms": None, "tried": 0}
    results.sort(key=lambda r: r[0])
    best = {"mapping": results[0][1], "gather_ms": results[0][0], "tried": len(results),
            "table": [[t, c] for t, c in results[:12]]}
    table[key] = best
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(table, f, indent=1)
    except OSError:
        pass
    return best


def apply(p: Params, best: dict) -> Params:
    return _params_for(dict(p.__dict__), best.get("mapping", {}))


def tune_batched(x_concat, offsets, p: Params, sample_clouds: int = 256, reps: int = 2,
                 budget_s: float = 60.0, cache: str | None = None, force: bool = False,
                 verbose: bool = False) -> dict:
    """Fastest persistent-kernel mapping (partner batches in flight, block
    size, rows per work item) for a batch of clouds, timed with CUDA events
    on the first ``sample_clouds`` clouds through sng_cluster_batched."""
    import ctypes

    import numpy as np
    import torch

    from . import SNG_F32, _check, lib
    path = _cache_path(cache)
    off = np.asarray(offsets, dtype=np.int64)
    k = min(sample_clouds, off.size - 1)
    sizes = np.diff(off[:k + 1])
    key = (f"batched-d{p.__dict__.get('d', x_concat.shape[1])}-ld{x_concat.stride(0)}"
           f"-mean{_bucket(int(sizes.mean()))}-m{_bucket(p.m or 1)}")
    if p.flags & 8:   # one warp per source row (rows of one float4 default to lanes)
        key += "-warprows"
    table = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if not force and key in table:
        return table[key]
    sub = off[:k + 1].copy()
    labels = torch.empty(int(sub[-1]), dtype=torch.int32, device=x_concat.device)
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    t0 = time.perf_counter()
    for u in (1, 2, 4, 8):
        for b in (256, 128):
            for tile in (256, 1024, 4096):
                if time.perf_counter() - t0 > budget_s:
                    break
                q = Params(**{**p.__dict__, "map_unroll": u, "map_block": b, "map_tile": tile})
                cp = q.to_c(0, x_concat.shape[1], x_concat.stride(0), SNG_F32)
                ms = []
                try:
                    for r in range(reps + 1):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record()
                        _check(lib().sng_cluster_batched(x_concat.data_ptr(), sub.ctypes.data, k,
                                                         ctypes.byref(cp), None, labels.data_ptr(),
                                                         None, stream))
                        e1.record()
                        e1.synchronize()
                        if r:
                            ms.append(e0.elapsed_time(e1))
                except SngError as e:
                    if verbose:
                        print("skip", u, b, tile, e)
                    continue
                t = statistics.median(ms)
                results.append((t, {"map_unroll": u, "map_block": b, "map_tile": tile}))
                if verbose:
                    print(f"{t:9.3f} ms  unroll={u} block={b} tile={tile}")
    if not results:
        return {"mapping": {}, "ms": None, "tried": 0}
    results.sort(key=lambda r: r[0])
    best = {"mapping": results[0][1], "ms": results[0][0], "tried": len(results),
            "table": [[t, c] for t, c in results[:8]]}
    table[key] = best
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(table, f, indent=1)
    except OSError:
        pass
    return best
