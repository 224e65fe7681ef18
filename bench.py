"""Benchmark: SNG-DBSCAN on one GB300, n = 1,000,000 points in d = 64.

Workload (the headline configuration): a mixture of 100 Gaussians in R^64
(centres N(0, 4 I), per-cluster std U[0.5, 1], Dirichlet(1) sizes) plus 2%
uniform noise in the bounding box; s = 0.001 (m = 1000 partner draws per
point, 1e9 distance queries); eps = the 1% quantile of distances over 1e6
seeded random pairs; MinPts = 10.  Synthetic data of the shape of the paper's
million-point datasets (Section 5), which are not available here.

One step = one whole pass of Algorithm 1 on the device-resident points:
partner draws + eps-test + FP64 guard-band recheck (gather), row-pointer scan,
CSR fill, core mask + union-find components, border labels, finalize.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (n, d, k, noise, s, min_pts)
    "mixture-n1M-d64": (1_000_000, 64, 100, 0.02, 0.001, 10),
    "mixture-n100k-d64": (100_000, 64, 100, 0.02, 0.01, 10),
    # profiling case of the same gather: same points (256 MB > L2), 100 draws
    "mixture-n1M-d64-s1e-4": (1_000_000, 64, 100, 0.02, 0.0001, 10),
    # profiling case of the tiled form: the headline's 1000 draws per point on
    # 4e5 points (102 MB, 3 x 3 tiles, 3.2 GB of tile buckets)
    "mixture-n400k-d64-m1000": (400_000, 64, 100, 0.02, 0.0025, 10),
}


def make_workload(name: str, seed: int = 0):
    from paper_2006_06743_gb300 import datagen
    n, d, k, noise, s, min_pts = WORKLOADS[name]
    x, truth = datagen.gaussian_mixture(n, d, k, noise, seed=seed, return_truth=True)
    eps = datagen.eps_quantile(x, q=0.01, n_pairs=1_000_000, seed=seed)
    return dict(x=x, truth=truth, n=n, d=d, s=s, min_pts=min_pts, eps=eps, seed=seed,
                m=int(math.ceil(s * n)))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region.

    The sampler starts before the timed region and waits for its first
    line, so that the 100 ms sampling loop is already running when the
    region begins; only the samples taken between start() returning and
    stop() being called (plus one sampling period) are reported."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 100

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line))

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()
        deadline = time.monotonic() + 5.0
        while not self.lines and time.monotonic() < deadline and self.proc.poll() is None:
            time.sleep(0.01)
        self.t0 = time.monotonic()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.t1 = time.monotonic()
        # one more period, so that a region shorter than it still has a sample
        time.sleep(self.PERIOD_MS / 1000.0 + 0.02)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        late = self.t1 + self.PERIOD_MS / 1000.0 + 0.02
        inside = [ln for t, ln in self.lines if self.t0 <= t <= late]
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in inside:
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm), "period_ms": self.PERIOD_MS,
                "region_s": round(self.t1 - self.t0, 3)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# The headline metric, as the benchmark definition states it: sampled
# eps-queries per second of the whole pass, with the end-to-end time, the
# HBM roofline fraction and the ARI reported beside it.
HEADLINE_METRIC = "sampled \u03b5-queries/s, e2e cluster time at n=1M d=64; %HBM roofline; ARI"

# Warp instructions per query of the batched kernel (smsp__inst_executed.sum
# over the queries of one launch), from one ncu capture of 256 clouds of the
# same size distribution; the 4096-cloud launch runs the same per-query code,
# so its count scales with the queries.
BATCHED_INST_PER_QUERY = {"batched_kernel<4, 1, 1, 4, 1>": 14_119_942_974 / 3_518_330_800,
                          "batched_kernel<4, 1, 1, 2, 1>": 13_978_125_782 / 3_518_330_800}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one gather
# launch, from one ncu capture of this workload and kernel.  Reported only
# while the timed launch uses that same kernel and mapping.
CAPTURED_TRAFFIC = {
    ("mixture-n1M-d64", "gather_kernel<float, 4, 4, 4, 2, 0, 1, 0>"): 168_524_939_776 + 456_195_584,
    # the tiled form: the partition launch plus all 36 tile tests of one step
    ("mixture-n1M-d64",
     "tile_partition_kernel + 36 x tile_test_kernel<float, 4, 4, 4, 2, 1, 1>"):
        21_680_128 + 8_046_274_048 + 11_679_285_760 + 172_615_680,
    # the tensor-core screen: one gather_mma_kernel launch and the queue of
    # open pairs (profiles/gather_mma_mixture-n1M-d64.md)
    ("mixture-n1M-d64", "gather_mma_kernel<4, 3, false> + screen_queue_kernel"):
        54_903_795_968 + 432_543_232 + 174_607_104 + 7_820_288,
}


def gather_algorithmic_bytes(n: int, d: int, m: int, esize: int, kept: int) -> int:
    """Bytes the gather must move per launch: one partner row per query, each
    point's own row once, its keep-bit words and row count once, and a 4-byte
    read-modify-write degree update per kept draw (in-degree) and per row."""
    words = (m + 31) // 32
    return n * m * d * esize + n * d * esize + n * words * 4 + n * 4 + kept * 8 + n * 8


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the arch)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def gather_kernel_name_and_bytes(stats: dict, n: int, d: int, m: int) -> tuple[str, int]:
    """Kernels of the gather phase as they ran, and the bytes the SMs must
    move in it: partner and own rows of the form's layout (a 16 * k-tile-wide
    BF16 copy for the tensor-core screen, d rounded up to 8 for the CUDA-core
    screen, FP32 otherwise), the squared norm per partner (tensor-core
    screen), the tiled form's 8-byte bucket entry per draw (written once,
    read once) and source row per run, keep words, degree updates, the FP32
    rows of every pair the screen left open, and the making of the copy."""
    kept = stats["kept_edges"]
    words = (m + 31) // 32
    screen, tiles = stats["map_screen"], stats["map_tiles"]
    full = stats["map_group"] * stats["map_nch"] * stats["map_vec"] == d
    common = n * words * 4 + n * 4 + kept * 8 + n * 8
    if screen == 4:
        ks = stats["map_nch"]
        row = 32 * ks
        byts = n * m * (row + 8) + n * (row + 8) + common
        name = f"gather_mma8_kernel<{ks}, {stats['map_unroll'] or 2}, false>"
    elif screen == 3:
        row = 128
        byts = n * m * (row + 4) + n * (row + 8) + common
        name = "gather_tc05_kernel"
    elif screen == 2:
        kt = stats["map_nch"]
        row = 16 * kt * 2
        byts = n * m * (row + 4) + n * (row + 8) + common
        name = f"gather_mma_kernel<{kt}, {stats['map_unroll'] or (3 if kt <= 4 else 2)}, false>"
    else:
        esize, vec = (2, 8) if screen else (4, 4)
        row = (-(-d // 8) * 8 if screen else d) * esize
        typ = "unsigned short" if screen else "float"
        if tiles:
            byts = n * m * (row + 16) + n * tiles * (row + 16) + common
            name = (f"tile_partition_kernel + {tiles * tiles} x tile_test_kernel<{typ}, "
                    f"{stats['map_vec']}, {stats['map_group']}, {stats['map_nch']}, "
                    f"{stats['map_unroll']}, {int(full)}, {stats['map_tex']}>")
        else:
            byts = n * m * row + n * row + common
            name = (f"gather_kernel<{typ}, {stats['map_vec']}, {stats['map_group']}, "
                    f"{stats['map_nch']}, {stats['map_unroll']}, 0, {int(full)}, 0>")
        if screen:
            name = "shadow_kernel + " + ("slice_max_kernel + " if tiles else "") + name
    # (kernel_ms is the whole gather phase: with the screen it includes
    # making the copy, 0.15 ms at the headline, and with the tensor-core
    # forms the queue of open pairs)
    if screen:
        copy_row = {2: 32 * stats["map_nch"], 3: 128, 4: 32 * stats["map_nch"]}.get(
            screen, -(-d // 8) * 8 * 2)
        byts += n * (d * 4 + copy_row + 12)              # the copy: read FP32, write the copy
        if screen == 4:
            byts += n * d * 4                            # the FP8 copy's scale pass
        open_pairs = stats.get("screen_pairs", 0)
        byts += open_pairs * 2 * d * 4                   # open pairs from the FP32 rows
        if screen in (2, 4):
            byts += open_pairs * 32                      # queue entry written and read
            name += " + screen_queue_kernel"
    return name, int(byts)


def run_cpu_baseline(w: dict, budget_s: float = 8.0, omp_budget_s: float = 30.0) -> dict:
    """The FP64 oracle as written, timed on the host's cores.

    Multi-core (the reported value): the OpenMP build of the same oracle
    source, step 2 over row blocks on every host core, then steps 3-5 (degrees,
    core mask, BFS components, border labels) on the whole graph: the whole
    pass when its estimate fits ``omp_budget_s``, else step 2 over the leading
    rows that fit.  Single-core beside it: the plain build, step 2 on a random
    sample of source rows.  queries/s scaled by the rows processed."""
    import numpy as np

    import oracle
    oracle.build()
    oracle.build(openmp=True)
    x, n, m = w["x"], w["n"], w["m"]
    rng = np.random.default_rng(1)
    probe = np.sort(rng.choice(n, size=200, replace=False))
    t0 = time.perf_counter()
    oracle.build_rows(x, w["eps"], w["seed"], m, rows=probe)
    dt = time.perf_counter() - t0
    rows = int(min(n, max(200, budget_s / max(dt, 1e-6) * 200)))
    sample = np.sort(rng.choice(n, size=rows, replace=False))
    t0 = time.perf_counter()
    oracle.build_rows(x, w["eps"], w["seed"], m, rows=sample)
    dt1 = time.perf_counter() - t0
    single = {"value": rows * m / dt1, "unit": "queries/s", "cores": 1, "seconds": dt1,
              "sample": f"step 2 of Algorithm 1 on {rows} random source rows "
                        f"({rows * m:.3g} FP64 queries), plain build"}
    threads = oracle.threads(openmp=True)
    est = n * m / (single["value"] * threads)
    if est <= omp_budget_s:
        t0 = time.perf_counter()
        rp, col, _ = oracle.build_rows_blocks(x, w["eps"], w["seed"], m, openmp=True,
                                              block=max(16, n // (16 * threads)))
        t1 = time.perf_counter()
        r = oracle.cluster_graph(n, rp, col, w["min_pts"])
        t2 = time.perf_counter()
        q = n * m
        sample_txt = (f"whole pass (steps 2-5 of Algorithm 1) over all {n} points, "
                      f"{q:.3g} FP64 queries; step 2 on {threads} threads, steps 3-5 on one")
        extra = {"step2_seconds": t1 - t0, "steps345_seconds": t2 - t1,
                 "clusters": r["clusters"], "kept_edges": r["kept_edges"]}
        secs = t2 - t0
    else:
        nr = int(max(1, min(n, omp_budget_s * single["value"] * threads / m)))
        t0 = time.perf_counter()
        oracle.build_rows_blocks(x, w["eps"], w["seed"], m, openmp=True, n_rows=nr,
                                 block=max(16, nr // (16 * threads)))
        secs = time.perf_counter() - t0
        q = nr * m
        sample_txt = (f"step 2 of Algorithm 1 on the first {nr} source rows "
                      f"({q:.3g} FP64 queries) on {threads} threads")
        extra = {}
    return {"value": q / secs, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "seconds": secs, "sample": sample_txt, "build": "gcc -O2 -fopenmp, FP64",
            "nproc": os.cpu_count(), "cpu_model": cpu_model(), **extra,
            "single_core": single}


def bench_sng(args, w):
    import numpy as np
    import torch

    import paper_2006_06743_gb300 as sng

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    # N > 1 (default, strong scaling): one dataset, step 2 split by source
    # rows, degrees all-reduced and edges all-gathered over NCCL.
    # --replicas (weak scaling): every rank clusters its own independent
    # dataset (no collective on the data path); rank r uses seed base + r.
    if rank > 0 and args.replicas:
        w = make_workload(args.workload, seed=args.seed + rank)
    x_host = torch.from_numpy(w["x"]).pin_memory()
    x = x_host.to(dev)
    n, d, m = w["n"], w["d"], w["m"]
    params = sng.Params(eps=w["eps"], min_pts=w["min_pts"], s=w["s"], seed=w["seed"],
                        flags=sng.SNG_FLAG_TIMING, map_group=args.map_group,
                        map_unroll=args.map_unroll, map_block=args.map_block,
                        map_passes=args.map_passes, degree_mode=args.degree_mode,
                        map_tile=args.map_tile)
    if args.tiled:
        params.flags |= sng.SNG_FLAG_TILED
    if args.screen:
        if args.screen == 4:
            params.flags |= sng.SNG_FLAG_SCREEN8
        else:
            params.flags |= sng.SNG_FLAG_SCREEN16 | (sng.SNG_FLAG_SCREEN_MMA if args.screen >= 2 else 0)
            params.flags |= sng.SNG_FLAG_TCGEN05 if args.screen == 3 else 0
    tuned = None
    if args.autotune and not (args.map_group or args.map_unroll or args.map_block
                              or args.map_passes or args.tiled or args.screen):
        from paper_2006_06743_gb300 import autotune
        tuned = autotune.tune(x, params, reps=2, budget_s=args.tune_budget,
                              verbose=args.verbose, force=args.retune)
        params = autotune.apply(params, tuned)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    if world > 1 and not args.replicas:
        out = bench_sharded(args, w, x, x_host, params, rank, world, dev, flush)
        dist.destroy_process_group()
        return out
    for _ in range(args.warmup):
        labels, st = sng.cluster(x, params)
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    launches0 = sng.launch_count()
    step_ms, gather_ms, stats = [], [], None
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    for _ in range(args.steps):
        flush.fill_(1)                      # evict L2 between steps (512 MB > 129 MB L2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        labels, stats = sng.cluster(x, params)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        gather_ms.append(stats["ms"]["gather"])
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    barrier()
    launches = sng.launch_count() - launches0
    t_step = statistics.mean(step_ms)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step = float(t.item())

    # end to end through the public API: pinned host points in, labels out
    # (sng_cluster_host: pinned host points in, host labels out; the library
    # copies, clusters and copies back inside the call)
    e2e_ms = []
    for it in range(max(1, args.warmup) + max(2, min(args.steps, 5))):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        labels_host, _ = sng.cluster_host(x_host, params)
        torch.cuda.synchronize(dev)
        if it >= max(1, args.warmup):   # untimed warm-up calls first
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    t_e2e = statistics.mean(e2e_ms)
    # the copy alone, for scale: one pinned 256 MB host-to-device transfer
    xd = torch.empty_like(x_host, device=dev)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    xd.copy_(x_host, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize(dev)
    h2d_one_stream_ms = h0.elapsed_time(h1)
    del xd

    Q = n * m
    peak, peak_kind = peaks()
    g_ms = statistics.mean(gather_ms)
    # the HBM model: every partner row from HBM (FP32 rows)
    alg = gather_algorithmic_bytes(n, d, m, 4, stats["kept_edges"])
    kname, alg_l2 = gather_kernel_name_and_bytes(stats, n, d, m)
    traffic = None
    if params.map_passes <= 1 and not (params.flags & sng.SNG_FLAG_PREFETCH):
        traffic = CAPTURED_TRAFFIC.get((args.workload, kname))
    # the roofline that bounds the gather: its working set (the BF16 copy of
    # the points, or one tile's two slices) stays in L2, so the peak is the
    # rate the SMs read from L2, measured here by the library's own probe
    l2_peak = sng.measure_l2_read(48 << 20, 200)
    achieved_l2 = alg_l2 / (g_ms * 1e-3) / 1e9
    # the tensor-core forms fetch one row of the copy per query: their
    # ceiling is the rate at which the SMs fetch random rows of that size
    # from a buffer of the copy's size (the library's random-row probe)
    random_rows = None
    if stats["map_screen"] in (2, 3, 4):
        rb = {2: 32 * stats["map_nch"], 3: 128, 4: 32 * stats["map_nch"]}[stats["map_screen"]]
        if rb in (64, 128, 256):
            probe = sng.measure_random_rows(n, rb, 1 << 30)
            fetched = Q / (g_ms * 1e-3)
            random_rows = {"row_bytes": rb, "probe_rows_per_s": probe,
                           "gather_rows_per_s": fetched, "frac": fetched / probe,
                           "note": "queries (one row of the copy each) per second of the "
                                   "gather phase against the probe's random-row rate"}
    truth = w["truth"].astype(np.int32)
    ari_truth = sng.ari(labels, torch.from_numpy(truth).to(dev))
    out = {
        "metric": HEADLINE_METRIC,
        "value": Q * world / (t_step * 1e-3),
        "unit": "queries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded Gaussian mixture, no dataset)",
        "config": {"workload": args.workload, "n": n, "d": d, "m": m, "s": w["s"],
                   "eps": w["eps"], "min_pts": w["min_pts"], "queries_per_step": Q,
                   "degree": ["undirected multigraph", "out-degree",
                              "distinct neighbours"][args.degree_mode],
                   "l2": "flushed between steps (512 MB write)", "parallelism": f"dp{world}",
                   "gather_mapping": {**{k: getattr(params, k) for k in
                                         ("map_group", "map_unroll", "map_block", "map_passes",
                                          "map_tile")},
                                      "tiled": bool(params.flags & sng.SNG_FLAG_TILED),
                                      "tiles_per_axis": stats["map_tiles"],
                                      "screen": ["none", "bf16 copy", "bf16 copy, tensor cores",
                                                 "bf16 copy, TMA gathers + tcgen05",
                                                 "fp8 copy, tensor cores"]
                                                [stats["map_screen"]],
                                      "prefetch": bool(params.flags & sng.SNG_FLAG_PREFETCH)},
                   "autotuned": tuned is not None},
        "e2e": {"value": Q * world / (t_e2e * 1e-3), "unit": "queries/s",
                "seconds": t_e2e * 1e-3,
                "h2d_bytes_per_step": int(x_host.numel() * 4),
                "d2h_bytes_per_step": int(n * 4),
                "api": "sng_cluster_host (host buffers in and out)",
                "h2d_one_stream_ms": h2d_one_stream_ms, "step_ms": e2e_ms},
        "gpu_launches": int(launches),
        "roofline": {"bound": "l2", "achieved": achieved_l2, "peak": l2_peak, "unit": "GB/s",
                     "frac": achieved_l2 / l2_peak, "traffic": traffic,
                     "kernel": kname, "peak_kind": "measured (sng_measure_l2_read, this run)",
                     "algorithmic_bytes": alg_l2, "kernel_ms": g_ms,
                     "traffic_frac": (traffic / (g_ms * 1e-3) / 1e9 / peak) if traffic else None,
                     "random_rows": random_rows,
                     "hbm_model": {"bound": "hbm", "algorithmic_bytes": alg,
                                   "achieved": alg / (g_ms * 1e-3) / 1e9, "peak": peak,
                                   "peak_kind": peak_kind, "unit": "GB/s",
                                   "frac": alg / (g_ms * 1e-3) / 1e9 / peak,
                                   "note": "256 B of FP32 partner row per query, all from HBM "
                                           "(the per-query byte model); the gather reads a BF16 "
                                           "copy or L2-resident tiles instead"}},
        "phases_ms": {k: v for k, v in stats["ms"].items()},
        "stats": {k: stats[k] for k in ("kept_edges", "band_pairs", "band_points", "cores",
                                        "clusters", "noise", "recheck_pairs", "screen_pairs",
                                        "map_screen", "map_tiles")},
        "ari_vs_generating_mixture": ari_truth,
        "ami_vs_generating_mixture": sng.ami(labels, torch.from_numpy(truth).to(dev))["ami"],
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = run_cpu_baseline(w, budget_s=args.cpu_budget,
                                               omp_budget_s=args.omp_budget)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out if rank == 0 else None


def bench_sharded(args, w, x, x_host, params, rank, world, dev, flush):
    """One dataset across all ranks (strong scaling, the multi-GPU form of the
    plain path): each step is the whole pass, step 2 split by source rows,
    one NCCL all-reduce of the degrees and one all-gather of the kept edges,
    then steps 3-5 on every rank.  Timed with CUDA events on the launching
    stream (the collectives join it), max over ranks."""
    import torch
    import torch.distributed as dist

    import paper_2006_06743_gb300 as sng
    from paper_2006_06743_gb300.distributed import GpuCompute, cluster_sharded, row_range
    comp = GpuCompute(x, params)
    n, d, m = w["n"], w["d"], w["m"]
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        cluster_sharded(comp, n)
    torch.cuda.synchronize(dev)
    dist.barrier()
    launches0 = sng.launch_count()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    step_ms, gather_ms = [], []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        labels, core, _ = cluster_sharded(comp, n)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        gather_ms.append(comp.last_stats["ms"]["gather"])
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    dist.barrier()
    launches = sng.launch_count() - launches0
    t = torch.tensor([statistics.mean(step_ms), statistics.mean(gather_ms)], device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_step, g_ms = float(t[0].item()), float(t[1].item())
    # end to end through the same call: every rank copies the points from
    # pinned host memory (they are replicated) and reads the labels back
    e2e_ms = []
    for it in range(1 + max(2, min(args.steps, 5))):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        dist.barrier()
        t0 = time.perf_counter()
        comp.x = x_host.to(dev, non_blocking=True)
        lab, _, _ = cluster_sharded(comp, n)
        lab_host = lab.cpu()
        torch.cuda.synchronize(dev)
        if it >= 1:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    comp.x = x
    te = torch.tensor([statistics.mean(e2e_ms)], device=dev)
    dist.all_reduce(te, op=dist.ReduceOp.MAX)
    t_e2e = float(te.item())
    lo, hi = row_range(n, rank, world)
    st = comp.last_stats
    Q = n * m
    peak, peak_kind = peaks()
    # this rank's shard of the gather: its rows' queries and own rows
    alg = gather_algorithmic_bytes(hi - lo, d, m, 4, st["kept_edges"])
    out = {"metric": HEADLINE_METRIC,
           "value": Q / (t_step * 1e-3), "unit": "queries/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
           "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded Gaussian mixture, no dataset)",
           "config": {"workload": args.workload, "n": n, "d": d, "m": m, "s": w["s"],
                      "eps": w["eps"], "min_pts": w["min_pts"], "queries_per_step": Q,
                      "l2": "flushed between steps (512 MB write)",
                      "parallelism": f"rows-sharded x{world}: NCCL all-reduce of degrees + "
                                     f"all-gather of kept edges"},
           "e2e": {"value": Q / (t_e2e * 1e-3), "unit": "queries/s", "seconds": t_e2e * 1e-3,
                   "h2d_bytes_per_step": int(x_host.numel() * 4),
                   "d2h_bytes_per_step": int(n * 4),
                   "api": "distributed.cluster_sharded (points copied from pinned host memory "
                          "on every rank, labels read back)"},
           "gpu_launches": int(launches),
           "roofline": {"bound": "hbm", "achieved": alg / (g_ms * 1e-3) / 1e9, "peak": peak,
                        "unit": "GB/s", "frac": alg / (g_ms * 1e-3) / 1e9 / peak,
                        "traffic": None, "peak_kind": peak_kind,
                        "kernel": "gather of one rank's row shard (slowest rank)",
                        "algorithmic_bytes": alg, "kernel_ms": g_ms},
           "clocks": clk}
    return out if rank == 0 else None


def _timed(fn, reps: int):
    """Median wall time of fn() in ms with a device sync on both sides."""
    import torch
    out = None
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(ts), out


def bench_bf16(args):
    """BF16 form: n = 5,000,000 unit-norm vectors in d = 128 (1000 centres on
    the sphere, per-coordinate noise sigma, renormalised); s = 0.0002 (m =
    1000); eps = 0.6; MinPts = 8.  Beside it, on the same points: the plain
    FP32 form (FP32 rows read by the gather) and the FP32 form with the
    certified BF16 screen (which reads a BF16 copy and keeps every FP64
    decision)."""
    import torch

    import paper_2006_06743_gb300 as sng
    from paper_2006_06743_gb300 import datagen
    n, d, m = args.bf16_n, 128, 1000
    x = datagen.sphere_embeddings(n, d, 1000, args.bf16_sigma, seed=args.seed)
    xf = torch.from_numpy(x).cuda()
    del x
    xb = xf.to(torch.bfloat16)
    p = sng.Params(eps=0.6, min_pts=8, s=0.0002, seed=args.seed, flags=sng.SNG_FLAG_TIMING)
    pf = pb = ps = p
    tuned = {}
    if args.autotune:
        from paper_2006_06743_gb300 import autotune
        tf = autotune.tune(xf, p, reps=1, budget_s=args.tune_budget, force=args.retune,
                           verbose=args.verbose, screen=False)
        ts = autotune.tune(xf, p, reps=1, budget_s=args.tune_budget, force=args.retune,
                           verbose=args.verbose)
        tb = autotune.tune(xb, p, x_master=xf, reps=1, budget_s=args.tune_budget,
                           force=args.retune, verbose=args.verbose)
        pf, ps, pb = autotune.apply(p, tf), autotune.apply(p, ts), autotune.apply(p, tb)
        tuned = {"fp32": tf.get("mapping"), "fp32_screened": ts.get("mapping"),
                 "bf16": tb.get("mapping")}
    for _ in range(args.warmup):
        sng.cluster(xf, pf)
        sng.cluster(xf, ps)
        sng.cluster(xb, pb, x_master=xf)
    f_ms, (lf, sf) = _timed(lambda: sng.cluster(xf, pf), args.steps)
    s_ms, (ls, ss) = _timed(lambda: sng.cluster(xf, ps), args.steps)
    b_ms, (lb, sb) = _timed(lambda: sng.cluster(xb, pb, x_master=xf), args.steps)
    # edge-decision error of the BF16 form against FP64: the FP32 form's
    # decisions equal the FP64 ones on every pair (guard band + FP64
    # recheck), so the difference of the two edge sets is that error
    gf = sng.build_graph(xf, pf)
    gb = sng.build_graph(xb, pb, x_master=xf)

    def keys(g):
        src = torch.repeat_interleave(torch.arange(n, device="cuda", dtype=torch.int64),
                                      torch.diff(g["row_ptr"]))
        return torch.sort(src * n + g["col"].to(torch.int64)).values

    kf, kb = keys(gf), keys(gb)
    common = int(torch.isin(kb, kf).sum().item())
    edge_error = {"kept_fp64": int(kf.numel()), "kept_bf16": int(kb.numel()),
                  "false_keep": int(kb.numel()) - common,
                  "false_drop": int(kf.numel()) - common,
                  "rate_of_fp64_edges": (int(kb.numel()) + int(kf.numel()) - 2 * common)
                  / max(1, int(kf.numel()))}
    del gf, gb, kf, kb
    Q = n * m
    peak, kind = peaks()
    alg_b = gather_algorithmic_bytes(n, d, m, 2, sb["kept_edges"])
    alg_f = gather_algorithmic_bytes(n, d, m, 4, sf["kept_edges"])
    return {"form": "bf16", "metric": "sampled eps-queries/s, BF16 vs FP32 form",
            "value": Q / (b_ms * 1e-3), "unit": "queries/s", "fp32_value": Q / (f_ms * 1e-3),
            "speedup_vs_fp32": f_ms / b_ms, "ms_bf16": b_ms, "ms_fp32": f_ms,
            "ms_fp32_screened": s_ms, "speedup_vs_fp32_screened": s_ms / b_ms,
            "ari_bf16_vs_fp32": sng.ari(lb, lf),
            "fp32_screened_labels_equal_fp32": bool(torch.equal(ls, lf)),
            "fp32_screened_form": ["none", "bf16 copy", "bf16 copy, tensor cores",
                                   "bf16 copy, TMA gathers + tcgen05",
                                   "fp8 copy, tensor cores"][ss["map_screen"]],
            "fp32_screened_open_pairs": ss["screen_pairs"],
            "edge_decision_error_vs_fp64": edge_error,
            "roofline_bf16": {"achieved": alg_b / (sb["ms"]["gather"] * 1e-3) / 1e9, "peak": peak,
                              "frac": alg_b / (sb["ms"]["gather"] * 1e-3) / 1e9 / peak,
                              "kernel_ms": sb["ms"]["gather"], "peak_kind": kind},
            "roofline_fp32": {"achieved": alg_f / (sf["ms"]["gather"] * 1e-3) / 1e9, "peak": peak,
                              "frac": alg_f / (sf["ms"]["gather"] * 1e-3) / 1e9 / peak,
                              "kernel_ms": sf["ms"]["gather"]},
            "stats_bf16": {k: sb[k] for k in ("kept_edges", "band_pairs", "recheck_pairs",
                                              "clusters", "noise")},
            "stats_fp32": {k: sf[k] for k in ("kept_edges", "band_pairs", "clusters", "noise")},
            "config": {"workload": f"sphere-n{n}-d{d}-sigma{args.bf16_sigma}", "m": m,
                       "eps": 0.6, "min_pts": 8, "mappings": tuned}, "dtype": "bf16",
            "steps": args.steps}


def bench_cosine(args):
    """Similarity form on the embedding workload: n = 5,000,000 unit vectors in
    d = 128 (1000 centres on the sphere, per-coordinate sigma, renormalised),
    m = 1000.  Cosine similarity >= 1 - eps^2/2 (eps = 0.6: the same graph as
    the Euclidean ball of radius eps, up to rounding, for unit vectors) in
    FP32 and BF16, the inner product in FP32, and the Euclidean form beside
    them; gather mappings from the autotuner (--autotune 0: defaults)."""
    import numpy as np
    import torch

    import paper_2006_06743_gb300 as sng
    from paper_2006_06743_gb300 import datagen
    n, d, m = args.bf16_n, 128, 1000
    x = datagen.sphere_embeddings(n, d, 1000, args.cos_sigma, seed=args.seed)
    xf = torch.from_numpy(x).cuda()
    del x
    xb = xf.to(torch.bfloat16)
    tau = float(np.float32(1.0 - 0.6 * 0.6 / 2.0))
    base = dict(min_pts=8, m=m, seed=args.seed, flags=sng.SNG_FLAG_TIMING)
    runs = {
        "l2_fp32": (xf, None, sng.Params(eps=0.6, **base), 4, 0),
        "cosine_fp32": (xf, None, sng.Params(eps=tau, metric=sng.SNG_METRIC_COSINE, **base), 4, 0),
        "dot_fp32": (xf, None, sng.Params(eps=tau, metric=sng.SNG_METRIC_DOT, **base), 4, 0),
        "l2_bf16": (xb, xf, sng.Params(eps=0.6, **base), 2, 0),
        "cosine_bf16": (xb, xf, sng.Params(eps=tau, metric=sng.SNG_METRIC_COSINE, **base), 2, 0),
    }
    peak, kind = peaks()
    out, labels, tuned = {}, {}, {}
    if args.autotune:
        from paper_2006_06743_gb300 import autotune
        for name in list(runs):
            xx, master, p, esize, extra = runs[name]
            t = autotune.tune(xx, p, x_master=master, reps=1, budget_s=args.tune_budget / 2,
                              force=args.retune, verbose=args.verbose)
            tuned[name] = t.get("mapping")
            runs[name] = (xx, master, autotune.apply(p, t), esize, extra)
    for name, (xx, master, p, esize, extra) in runs.items():
        for _ in range(args.warmup):
            sng.cluster(xx, p, x_master=master)
        ms, (lab, st) = _timed(lambda: sng.cluster(xx, p, x_master=master), args.steps)
        labels[name] = lab
        alg = gather_algorithmic_bytes(n, d, m, esize, st["kept_edges"]) + n * m * extra
        g_ms = st["ms"]["gather"]
        out[name] = {"ms": ms, "queries_per_s": n * m / (ms * 1e-3), "gather_ms": g_ms,
                     "gather_gbs": alg / (g_ms * 1e-3) / 1e9,
                     "frac_of_hbm": alg / (g_ms * 1e-3) / 1e9 / peak,
                     "kept_edges": st["kept_edges"], "recheck_pairs": st["recheck_pairs"],
                     "clusters": st["clusters"], "noise": st["noise"],
                     "screen": ["none", "bf16 copy", "bf16 copy, tensor cores",
                                "bf16 copy, TMA gathers + tcgen05",
                                "fp8 copy, tensor cores"][st["map_screen"]],
                     "screen_pairs": st["screen_pairs"],
                     "mapping": [st["map_vec"], st["map_group"], st["map_nch"],
                                 st["map_unroll"]]}
    for name in ("cosine_fp32", "dot_fp32", "l2_bf16", "cosine_bf16"):
        out[name]["ari_vs_l2"] = sng.ari(labels[name], labels["l2_fp32"])
    return {"form": "cosine", "metric": "sampled similarity queries/s (cosine, FP32)",
            "value": out["cosine_fp32"]["queries_per_s"], "unit": "queries/s", "runs": out,
            "peak_gbs": peak, "peak_kind": kind,
            "config": {"workload": f"sphere-n{n}-d{d}-sigma{args.cos_sigma}", "m": m,
                       "tau": tau, "eps_l2": 0.6, "min_pts": 8, "mappings": tuned},
            "dtype": "f32",
            "steps": args.steps}


def bench_pairmetric(args):
    """Manhattan and Chebyshev distances at the headline's points (Gaussian
    mixture, n = 10^6, m = 1000, d = 64 and 128, eps at the 1% quantile of
    the metric over 2*10^5 seeded pairs): the pair-kernel gather over the
    FP32 points and over the certified BF16 copy (SNG_FLAG_SCREEN16), labels
    of the two compared, and the copy's partner-row reads against the
    measured L2 read rate."""
    import numpy as np
    import torch

    import paper_2006_06743_gb300 as sng
    from paper_2006_06743_gb300 import datagen
    n, m = args.pm_n, 1000
    l2_peak = sng.measure_l2_read(48 << 20, 200)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    runs = {}
    for d in args.pm_d:
        x = datagen.gaussian_mixture(n, d, 100, 0.02, seed=args.seed)
        xg = torch.from_numpy(x).cuda()
        rng = np.random.default_rng(args.seed)
        i, j = rng.integers(0, n, 200_000), rng.integers(0, n, 200_000)
        diff = np.abs(x[i].astype(np.float64) - x[j].astype(np.float64))
        del x
        for metric, name, v in ((sng.SNG_METRIC_L1, "l1", diff.sum(1)),
                                (sng.SNG_METRIC_LINF, "linf", diff.max(1))):
            eps = float(np.float32(np.quantile(v, 0.01)))
            labels = {}
            for form, f in (("fp32", 0), ("bf16_screen", sng.SNG_FLAG_SCREEN16)):
                p = sng.Params(eps=eps, min_pts=10, m=m, seed=args.seed, metric=metric,
                               flags=f | sng.SNG_FLAG_TIMING)
                for _ in range(args.warmup):
                    sng.cluster(xg, p)

                def step():
                    flush.fill_(1)
                    return sng.cluster(xg, p)
                ms, (lab, st) = _timed(step, args.steps)
                labels[form] = lab
                g_ms = st["ms"]["gather"]
                row = (2 if f else 4) * (-(-d // 8) * 8 if f else d)
                runs[f"{name}_d{d}_{form}"] = {
                    "ms": ms, "gather_ms": g_ms, "queries_per_s": n * m / (g_ms * 1e-3),
                    "partner_row_bytes": row,
                    "l2_frac": n * m * row / (g_ms * 1e-3) / 1e9 / l2_peak,
                    "open_pairs": st["screen_pairs"], "recheck_pairs": st["recheck_pairs"],
                    "band_pairs": st["band_pairs"], "kept_edges": st["kept_edges"],
                    "clusters": st["clusters"]}
            runs[f"{name}_d{d}_bf16_screen"]["labels_equal_fp32"] = bool(
                torch.equal(labels["fp32"], labels["bf16_screen"]))
            runs[f"{name}_d{d}_bf16_screen"]["speedup"] = (
                runs[f"{name}_d{d}_fp32"]["gather_ms"] / runs[f"{name}_d{d}_bf16_screen"]["gather_ms"])
        del xg
    return {"form": "pairmetric", "metric": "sampled distance queries/s of the gather phase",
            "value": runs[f"l1_d{args.pm_d[0]}_bf16_screen"]["queries_per_s"], "unit": "queries/s",
            "runs": runs, "l2_read_peak_gbs": l2_peak,
            "config": {"workload": f"mixture-n{n}", "d": args.pm_d, "m": m, "eps": "1% quantile",
                       "min_pts": 10, "l2_flush": "512 MB buffer written before each step"},
            "dtype": "f32", "steps": args.steps}


def bench_graph(args):
    """One whole pass launched directly (sng_cluster, host reads E mid-way)
    against the same pass captured once as a CUDA graph
    (SNG_FLAG_NO_SYNC, replayed): the small configuration (n = 10^4, d = 2,
    s = 0.01) where launches and the host round trip dominate, and the
    headline workload."""
    import numpy as np
    import torch

    import paper_2006_06743_gb300 as sng
    from paper_2006_06743_gb300 import datagen
    out = {}
    cases = {"mixture2d-n10k": (datagen.mixture_2d(10_000, seed=args.seed),
                                sng.Params(eps=0.03, min_pts=3, s=0.01, seed=args.seed))}
    w = make_workload("mixture-n1M-d64", seed=args.seed)
    # the headline workload through the tensor-core screen (its gather form),
    # which the no-sync form keeps
    cases["mixture-n1M-d64"] = (w["x"], sng.Params(
        eps=w["eps"], min_pts=w["min_pts"], s=w["s"], seed=w["seed"],
        flags=sng.SNG_FLAG_SCREEN16 | sng.SNG_FLAG_SCREEN_MMA))
    for name, (x, p) in cases.items():
        xg = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        n = xg.shape[0]
        ref, _ = sng.cluster(xg, p)
        reps = max(args.steps, 20) if n <= 100_000 else args.steps
        for _ in range(args.warmup):
            sng.cluster(xg, p)
        direct, _ = _timed(lambda: sng.cluster(xg, p), reps)
        labels = torch.empty(n, dtype=torch.int32, device="cuda")
        counters = torch.zeros(9, dtype=torch.int64, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            sng.cluster_async(xg, p, labels, counters)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            sng.cluster_async(xg, p, labels, counters)
        for _ in range(args.warmup):
            graph.replay()
        replay, _ = _timed(graph.replay, reps)
        out[name] = {"direct_ms": direct, "graph_replay_ms": replay,
                     "speedup": direct / replay,
                     "labels_equal": bool(torch.equal(labels, ref)),
                     "queries": int(n * p.draws(n))}
        del graph, xg
        torch.cuda.synchronize()
    return {"form": "graph", "metric": "whole-pass time, direct call vs CUDA graph replay",
            "value": out["mixture2d-n10k"]["speedup"], "unit": "x (small configuration)",
            "cases": out, "dtype": "f32", "steps": args.steps}


def bench_batched(args):
    """Batched form: 4096 3-D clouds of 2,000..130,000 points (Gaussian blobs
    plus a 30% ground layer), m = 200, eps = 0.3 m, MinPts = 4; one
    persistent launch replayed as a CUDA graph against one sng_cluster call
    per cloud."""
    import ctypes

    import numpy as np
    import torch

    import paper_2006_06743_gb300 as sng
    from paper_2006_06743_gb300 import datagen
    x, off = datagen.point_clouds(args.clouds, seed=args.seed)
    xg = torch.from_numpy(x).cuda()
    total = x.shape[0]
    del x
    labels = torch.empty(total, dtype=torch.int32, device="cuda")
    p = sng.Params(eps=0.3, min_pts=4, m=200, seed=args.seed,
                   flags=0 if args.lane_rows else sng.SNG_FLAG_WARP_ROWS)
    tuned = None
    if args.map_unroll or args.map_block:
        p = sng.Params(**{**p.__dict__, "map_unroll": args.map_unroll,
                          "map_block": args.map_block})
    elif args.autotune:
        from paper_2006_06743_gb300 import autotune
        tuned = autotune.tune_batched(xg, off, p, sample_clouds=1024, budget_s=args.tune_budget,
                                      force=args.retune, verbose=args.verbose)
        p = sng.Params(**{**p.__dict__, **tuned.get("mapping", {})})
    cp = p.to_c(0, 3, 4, sng.SNG_F32)
    L = sng.lib()
    plan = ctypes.c_void_p()
    offs = np.ascontiguousarray(off, dtype=np.int64)
    sng._check(L.sng_batch_plan_create(offs.ctypes.data, len(off) - 1, ctypes.byref(cp), None,
                                       ctypes.byref(plan)))
    st = sng.sng_stats()
    strm = torch.cuda.current_stream().cuda_stream

    def run():
        sng._check(L.sng_batch_run(plan, xg.data_ptr(), labels.data_ptr(), None, strm))
    for _ in range(args.warmup):
        run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(args.steps):
        e0.record()
        run()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    b_ms = statistics.median(ms)
    sng._check(L.sng_batch_run(plan, xg.data_ptr(), labels.data_ptr(), ctypes.byref(st), strm))
    stats = st.as_dict()
    L.sng_batch_plan_destroy(plan)
    # per-cloud sequential calls (each cloud its own sng_cluster)
    seq_labels = torch.empty_like(labels)
    ncl = min(args.clouds, args.seq_clouds)

    def seq():
        for b in range(ncl):
            xb = xg[off[b]:off[b + 1], :3]
            q = sng.Params(eps=0.3, min_pts=4, m=200, seed=args.seed + b)
            lb, _ = sng.cluster(xb, q)
            seq_labels[off[b]:off[b + 1]] = lb
    s_ms, _ = _timed(seq, 1)
    frac = float(off[ncl]) / float(off[-1])
    same = bool(torch.equal(seq_labels[:off[ncl]], labels[:off[ncl]]))
    Q = int(stats["queries"])
    # issue-rate roofline: the kernel is bound by instruction issue and L2
    # latency (clouds are L2-resident), not by HBM
    lanes = not (p.flags & sng.SNG_FLAG_WARP_ROWS)
    kname = f"batched_kernel<4, 1, 1, {p.map_unroll or 4}, {int(lanes)}>"
    ipq = BATCHED_INST_PER_QUERY.get(kname)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    issue_peak = sms * 4 * 2070e6           # 4 warp instructions per SM per cycle
    roof = {"bound": "alu", "unit": "warp-instr/s", "peak": issue_peak, "kernel": kname,
            "achieved": None, "frac": None, "traffic": None,
            "peak_basis": f"{sms} SMs x 4 issue slots x 2070 MHz"}
    if ipq is not None and p.map_block in (0, 256):
        roof["achieved"] = ipq * Q / (b_ms * 1e-3)
        roof["frac"] = roof["achieved"] / issue_peak
        roof["inst_per_query"] = ipq
    return {"form": "batched", "metric": "sampled eps-queries/s, 4096 clouds in one launch",
            "value": Q / (b_ms * 1e-3), "unit": "queries/s", "ms_batched": b_ms,
            "roofline": roof,
            "ms_sequential_est": s_ms / frac, "sequential_clouds_timed": ncl,
            "speedup_vs_sequential": (s_ms / frac) / b_ms, "labels_equal_sequential": same,
            "stats": {k: stats[k] for k in ("queries", "kept_edges", "cores", "clusters",
                                            "noise")},
            "config": {"workload": f"clouds-{args.clouds}-2k..130k-d3", "points": total,
                       "m": 200, "eps": 0.3, "min_pts": 4, "graph": "CUDA graph replay",
                       "mapping": {**{k: getattr(p, k) for k in ("map_unroll", "map_block",
                                                                 "map_tile")},
                                   "lane_rows": not (p.flags & sng.SNG_FLAG_WARP_ROWS)},
                       "autotuned": tuned is not None},
            "dtype": "f32", "steps": args.steps}


def bench_surrogate(args):
    """Learned-surrogate form: n = 2,000,000 points in d = 32 from a
    200-Gaussian mixture with 3% noise; s = 0.0005 (m = 1000); eps = 1%
    pair-distance quantile; MinPts = 8.  The network is trained on core masks
    of 10 sibling datasets (same mixture, new samples) labelled by the plain
    GPU method, then gates a fresh sibling."""
    import torch

    import paper_2006_06743_gb300 as sng
    from paper_2006_06743_gb300 import datagen, surrogate as sg
    n, d, m = args.surr_n, 32, 1000
    master = 2020
    xs, ys, eps = [], [], None
    t0 = time.perf_counter()
    for k in range(args.siblings + 1):
        x = datagen.gaussian_mixture(n, d, 200, 0.03, seed=10 + k, master_seed=master)
        if eps is None:
            eps = datagen.eps_quantile(x, 0.01, 1_000_000, seed=0)
        xg = torch.from_numpy(x).cuda()
        _, core, _ = sng.cluster(xg, sng.Params(eps=eps, min_pts=8, s=0.0005, seed=k),
                                 want_core=True)
        xs.append(xg)
        ys.append(core)
    t_label = time.perf_counter() - t0
    xt = xs.pop()
    ys.pop()
    xtr, ytr = torch.cat(xs).contiguous(), torch.cat(ys).contiguous()
    del xs, ys
    net = sg.Surrogate(datagen.mlp_init(d, 128, args.seed), cfg=sg.TrainConfig(batch=4096))
    net.standardize(xtr)
    t_train, trace = _timed(lambda: net.train(xtr, ytr, args.train_steps), 1)
    # plain and surrogate both through the tensor-core screen of the FP32
    # points (exact, the fastest form for this shape)
    p = sng.Params(eps=eps, min_pts=8, s=0.0005, seed=99,
                   flags=sng.SNG_FLAG_TIMING | sng.SNG_FLAG_SCREEN16 | sng.SNG_FLAG_SCREEN_MMA)
    gates = {
        # the configuration as written: confidence in [0.1, 0.9] falls back to
        # full queries (confident core draws core_frac of them, confident
        # noise none)
        "as_written": dict(p_noise=0.1, p_core=0.9, core_draw_frac=0.5,
                           noise_draw_frac=0.0, reweight=False),
        # the tuned gate: the same upper threshold, no noise gating (a point
        # gated as noise loses the draws that attach it to a cluster as a
        # border point)
        "tuned": dict(p_noise=args.p_noise, p_core=args.p_core, core_draw_frac=args.core_frac,
                      noise_draw_frac=args.noise_frac, reweight=bool(args.reweight)),
    }
    for _ in range(args.warmup):
        sng.cluster(xt, p)
        net.cluster(xt, p, **gates["tuned"])
    p_ms, (plain, pcore, pst) = _timed(lambda: sng.cluster(xt, p, want_core=True), args.steps)
    res = {}
    for name, g in gates.items():
        s_ms, (lab, core, sst) = _timed(lambda: net.cluster(xt, p, want_core=True, **g), args.steps)
        res[name] = {"gate": g, "ms": s_ms, "speedup_vs_plain": p_ms / s_ms,
                     "ari_vs_plain": sng.ari(lab, plain),
                     "core_mask_agreement": float((core == pcore).float().mean().item()),
                     "queries_issued_frac": sst["queries"] / pst["queries"],
                     "gated_core": sst["surrogate_core"], "gated_noise": sst["surrogate_noise"],
                     "phases_ms": sst["ms"]}
    t = res["tuned"]
    return {"form": "surrogate", "metric": "e2e cluster time, surrogate vs plain",
            "value": n * m / (t["ms"] * 1e-3), "unit": "queries/s (nominal n*m)",
            "ms_surrogate": t["ms"], "ms_plain": p_ms, "speedup_vs_plain": t["speedup_vs_plain"],
            "ari_vs_plain": t["ari_vs_plain"], "core_mask_agreement": t["core_mask_agreement"],
            "queries_issued_frac": t["queries_issued_frac"], "gates": res,
            "phases_ms_plain": pst["ms"],
            "train": {"steps": args.train_steps, "siblings": args.siblings,
                      "seconds": t_train * 1e-3,
                      "loss_first": float(trace[:50].mean()), "loss_last": float(trace[-200:].mean()),
                      "label_seconds": t_label},
            "config": {"workload": f"mixture-n{n}-d{d}-k200", "m": m, "eps": eps, "min_pts": 8},
            "dtype": "f32", "steps": args.steps}


def bench_balls(args):
    """The simulation of the paper's Figure 1: a uniform mixture of three unit
    balls in R^3 (centres 3 apart, so 1 apart at the closest), m =
    ceil(20 ln n) draws per point, eps = 0.5, MinPts = 2 (the caption fixes
    only the sampling rate; eps below the gap and the smallest MinPts are this
    reading).  ARI and AMI against the generating ball, for growing n."""
    import numpy as np
    import torch

    import paper_2006_06743_gb300 as sng
    from paper_2006_06743_gb300 import datagen
    rows = []
    for n in args.balls_n:
        x, truth = datagen.uniform_balls(n, seed=args.seed)
        m = int(math.ceil(20.0 * math.log(n)))
        xg = torch.from_numpy(x).cuda()
        p = sng.Params(eps=0.5, min_pts=2, m=m, seed=args.seed, flags=sng.SNG_FLAG_TIMING)
        sng.cluster(xg, p)
        t_ms, (lab, st) = _timed(lambda: sng.cluster(xg, p), 3)
        tg = torch.from_numpy(truth.astype(np.int32)).cuda()
        rows.append({"n": n, "m": m, "ari_vs_truth": sng.ari(lab, tg),
                     "ami_vs_truth": sng.ami(lab, tg)["ami"], "clusters": st["clusters"],
                     "noise": st["noise"], "ms": t_ms})
    return {"form": "balls", "metric": "ARI vs generating ball (Figure 1 simulation)",
            "value": rows[-1]["ari_vs_truth"], "unit": "ARI", "rows": rows,
            "config": {"workload": "3 uniform unit balls in R^3", "eps": 0.5, "min_pts": 2,
                       "m": "ceil(20 ln n)"}, "dtype": "f32"}


def bench_sweep(args):
    """Quality and time against the sampling rate s (the synthetic analogue of
    the paper's Figure 10): a Gaussian mixture (as the headline workload,
    smaller n), full DBSCAN computed on the GPU with every pair queried
    (s = 1, multigraph degree, MinPts = 2 (min_samples - 1)), and
    SNG-DBSCAN at decreasing s with MinPts scaled by s; ARI and AMI of each
    against full DBSCAN and against the generating mixture.  Then the
    radius sweep at one sampling rate (the synthetic analogue of the paper's
    ARI-against-eps figures): each eps against full DBSCAN at that eps."""
    import numpy as np
    import torch

    import paper_2006_06743_gb300 as sng
    from paper_2006_06743_gb300 import datagen
    n, d = args.sweep_n, 16
    x, truth = datagen.gaussian_mixture(n, d, 20, 0.02, seed=args.seed, return_truth=True)
    eps = datagen.eps_quantile(x, 0.01, 1_000_000, seed=args.seed)
    xg = torch.from_numpy(x).cuda()
    tg = torch.from_numpy(truth.astype(np.int32)).cuda()
    k_db = 10                                  # textbook min_samples (self included)
    full_p = sng.Params(eps=eps, min_pts=2 * (k_db - 1), sample_mode=sng.SNG_SAMPLE_ALL,
                        flags=sng.SNG_FLAG_TIMING)
    sng.cluster(xg, full_p)
    full_ms, (full, fst) = _timed(lambda: sng.cluster(xg, full_p), 1)
    rows = [{"s": 1.0, "ms": full_ms, "ari_vs_full": 1.0, "ari_vs_truth": sng.ari(full, tg),
             "ami_vs_full": 1.0, "ami_vs_truth": sng.ami(full, tg)["ami"],
             "clusters": fst["clusters"]}]
    for s in args.sweep_s:
        mp = max(2, int(round(2 * (k_db - 1) * s)))
        p = sng.Params(eps=eps, min_pts=mp, s=s, seed=args.seed)
        sng.cluster(xg, p)
        ms, (lab, st) = _timed(lambda: sng.cluster(xg, p), 3)
        rows.append({"s": s, "m": p.draws(n), "min_pts": mp, "ms": ms,
                     "speedup_vs_full": full_ms / ms, "ari_vs_full": sng.ari(lab, full),
                     "ari_vs_truth": sng.ari(lab, tg), "ami_vs_full": sng.ami(lab, full)["ami"],
                     "ami_vs_truth": sng.ami(lab, tg)["ami"], "clusters": st["clusters"]})
    # the eps sweep at a fixed sampling rate: each radius against full
    # DBSCAN at the same radius (eps from quantiles of the pairwise
    # distances)
    eps_rows = []
    s_eps = args.sweep_eps_s
    mp = max(2, int(round(2 * (k_db - 1) * s_eps)))
    for q in args.sweep_eps_q:
        e = datagen.eps_quantile(x, q, 1_000_000, seed=args.seed)
        fp = sng.Params(eps=e, min_pts=2 * (k_db - 1), sample_mode=sng.SNG_SAMPLE_ALL)
        ref, _ = sng.cluster(xg, fp)
        p = sng.Params(eps=e, min_pts=mp, s=s_eps, seed=args.seed)
        sng.cluster(xg, p)
        ms, (lab, st) = _timed(lambda: sng.cluster(xg, p), 3)
        eps_rows.append({"quantile": q, "eps": e, "ms": ms, "ari_vs_full": sng.ari(lab, ref),
                         "ari_full_vs_truth": sng.ari(ref, tg), "ari_vs_truth": sng.ari(lab, tg),
                         "ami_vs_full": sng.ami(lab, ref)["ami"], "clusters": st["clusters"]})
    return {"form": "sweep", "metric": "ARI vs full DBSCAN against sampling rate",
            "value": rows[-1]["ari_vs_full"], "unit": "ARI", "rows": rows,
            "eps_sweep": {"s": s_eps, "min_pts": mp, "rows": eps_rows},
            "config": {"workload": f"mixture-n{n}-d{d}-k20", "eps": eps, "min_samples": k_db,
                       "min_pts_rule": "round(2 (min_samples - 1) s), at least 2"},
            "dtype": "f32"}


def run_extensions(args) -> dict:
    """The extension forms' key results, folded into the default line (each
    at its stated size, fewer repetitions than their own lines): the BF16
    form against FP32 on the same points (the sigma = 0.0375 companion, where
    the graph has edges and the decision error means something), the batched
    form against per-cloud calls, and the learned surrogate against the plain
    method at the gate the configuration states and at the tuned gate."""
    import copy

    import torch
    out = {}
    a = copy.copy(args)
    a.steps, a.warmup, a.tune_budget = 3, 1, args.ext_tune_budget
    t0 = time.perf_counter()
    a.bf16_sigma = 0.0375
    r = bench_bf16(a)
    out["bf16"] = {"workload": r["config"]["workload"], "ms_bf16": r["ms_bf16"],
                   "ms_fp32": r["ms_fp32"], "speedup_vs_fp32": r["speedup_vs_fp32"],
                   "ms_fp32_screened": r["ms_fp32_screened"],
                   "fp32_screened_form": r["fp32_screened_form"],
                   "fp32_screened_labels_equal_fp32": r["fp32_screened_labels_equal_fp32"],
                   "speedup_vs_fp32_screened": r["speedup_vs_fp32_screened"],
                   "ari_vs_fp32": r["ari_bf16_vs_fp32"],
                   "edge_decision_error_vs_fp64": r["edge_decision_error_vs_fp64"],
                   "seconds": time.perf_counter() - t0}
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    a.seq_clouds = 256
    r = bench_batched(a)
    out["batched"] = {"workload": r["config"]["workload"], "ms_batched": r["ms_batched"],
                      "ms_sequential_est": r["ms_sequential_est"],
                      "speedup_vs_sequential": r["speedup_vs_sequential"],
                      "labels_equal_sequential": r["labels_equal_sequential"],
                      "queries_per_s": r["value"], "seconds": time.perf_counter() - t0}
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    r = bench_surrogate(a)
    out["surrogate"] = {k: r[k] for k in ("ms_surrogate", "ms_plain", "speedup_vs_plain",
                                          "ari_vs_plain", "core_mask_agreement",
                                          "queries_issued_frac") if k in r}
    out["surrogate"].update({"workload": r["config"]["workload"],
                             "gates": r.get("gates"), "seconds": time.perf_counter() - t0})
    torch.cuda.empty_cache()
    return out


def bench_reference(args, w):
    """The reference arm: the FP64 CPU oracle, timed as it stands on the host.
    Each step runs step 2 of Algorithm 1 (the OpenMP build of the oracle on
    every host core) over a block of consecutive source rows sized to about
    ``--ref-budget`` seconds; steps 3-5 of the whole pass are timed once on
    the whole graph during the warm-up and added to the per-step figure."""
    import oracle
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    oracle.build(openmp=True)
    oracle.build()
    x, n, m = w["x"], w["n"], w["m"]
    threads = oracle.threads(openmp=True)
    probe = 64 * threads
    t0 = time.perf_counter()
    oracle.build_rows_blocks(x, w["eps"], w["seed"], m, openmp=True, n_rows=probe, block=64)
    rate = probe * m / (time.perf_counter() - t0)
    nr = int(max(probe, min(n, args.ref_budget * rate / m)))
    block = max(16, nr // (16 * threads))            # blocks for every thread
    # steps 3-5 once, on the oracle's whole graph, when building it fits the
    # budget (the whole of step 2 on all cores)
    t345 = None
    if n * m / rate <= args.ref_whole_budget:
        rp, col, _ = oracle.build_rows_blocks(x, w["eps"], w["seed"], m, openmp=True,
                                              block=max(16, n // (16 * threads)))
        t1 = time.perf_counter()
        oracle.cluster_graph(n, rp, col, w["min_pts"])
        t345 = time.perf_counter() - t1
        del rp, col
    steps = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.build_rows_blocks(x, w["eps"], w["seed"], m, openmp=True, n_rows=nr, block=block)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            steps.append(dt)
    step2 = statistics.mean(steps) * n / nr          # whole step 2, scaled by rows
    ms = (step2 + (t345 or 0.0)) * 1e3
    v = n * m / (ms * 1e-3)
    sample = (f"step 2 on source rows 0..{nr - 1} ({nr * m:.3g} FP64 queries) per step on "
              f"{threads} threads, scaled to all {n} rows, "
              + (f"plus steps 3-5 on the whole graph on one thread ({t345:.3g} s)"
                 if t345 is not None else "steps 3-5 not timed (whole graph over budget)"))
    return {"impl": "reference",
            "metric": HEADLINE_METRIC,
            "value": v, "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian mixture, no dataset)",
            "config": {"workload": args.workload, "n": n, "d": w["d"], "m": m,
                       "eps": w["eps"], "min_pts": w["min_pts"],
                       "note": "FP64 CPU oracle (OpenMP build of the same C source) on a "
                               "block of source rows per step; ms_per_step scales step 2 "
                               "to all rows and adds steps 3-5"},
            "cpu_baseline": {"value": v, "unit": "queries/s", "cores": threads, "kind": "oracle",
                             "sample": sample, "nproc": os.cpu_count(),
                             "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sng", choices=["sng", "reference"])
    ap.add_argument("--workload", default="mixture-n1M-d64", choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--map-group", type=int, default=0)
    ap.add_argument("--map-unroll", type=int, default=0)
    ap.add_argument("--map-block", type=int, default=0)
    ap.add_argument("--map-passes", type=int, default=0)
    ap.add_argument("--map-tile", type=int, default=0)
    ap.add_argument("--tiled", type=int, default=0, help="1: the L2-tiled gather")
    ap.add_argument("--screen", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="1: certified BF16 screen of the FP32 points; 2: its tensor-core "
                         "form; 3: with TMA row gathers and tcgen05 dot products; 4: the "
                         "screen on an FP8 copy")
    ap.add_argument("--autotune", type=int, default=1, help="1: tune the gather mapping first")
    ap.add_argument("--degree-mode", type=int, default=0, choices=[0, 1, 2],
                    help="0 undirected multigraph, 1 out-degree, 2 distinct neighbours")
    ap.add_argument("--retune", action="store_true")
    ap.add_argument("--tune-budget", type=float, default=40.0)
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: independent datasets per rank (weak scaling) instead of one "
                         "dataset's rows split across ranks")
    ap.add_argument("--form", default="plain",
                    choices=["plain", "bf16", "batched", "surrogate", "balls", "sweep", "cosine",
                             "graph", "pairmetric"])
    ap.add_argument("--pm-n", type=int, default=1_000_000)
    ap.add_argument("--pm-d", type=int, nargs="+", default=[64, 128])
    ap.add_argument("--sweep-n", type=int, default=100_000)
    ap.add_argument("--sweep-eps-s", type=float, default=0.1,
                    help="sampling rate of the eps sweep (--form sweep)")
    ap.add_argument("--sweep-eps-q", type=float, nargs="+",
                    default=[0.002, 0.005, 0.01, 0.02, 0.05],
                    help="distance quantiles giving the eps values of the eps sweep")
    ap.add_argument("--sweep-s", type=float, nargs="+",
                    default=[0.3, 0.1, 0.03, 0.01, 0.003, 0.001])
    ap.add_argument("--balls-n", type=int, nargs="+",
                    default=[100, 300, 1000, 3000, 10_000, 100_000, 1_000_000, 10_000_000])
    ap.add_argument("--bf16-n", type=int, default=5_000_000)
    ap.add_argument("--bf16-sigma", type=float, default=0.15)
    ap.add_argument("--cos-sigma", type=float, default=0.0375)
    ap.add_argument("--clouds", type=int, default=4096)
    ap.add_argument("--seq-clouds", type=int, default=512)
    ap.add_argument("--lane-rows", type=int, default=1,
                    help="batched form: 1 = one lane per source row (default), 0 = one warp")
    ap.add_argument("--surr-n", type=int, default=2_000_000)
    ap.add_argument("--siblings", type=int, default=10)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--p-noise", type=float, default=0.0)
    ap.add_argument("--p-core", type=float, default=0.9)
    ap.add_argument("--core-frac", type=float, default=0.75)
    ap.add_argument("--noise-frac", type=float, default=0.0)
    ap.add_argument("--reweight", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extensions", type=int, default=1,
                    help="1: add the BF16, batched and surrogate forms' key results")
    ap.add_argument("--ext-tune-budget", type=float, default=12.0)
    ap.add_argument("--cpu-budget", type=float, default=8.0)
    ap.add_argument("--omp-budget", type=float, default=30.0)
    ap.add_argument("--ref-budget", type=float, default=5.0)
    ap.add_argument("--ref-whole-budget", type=float, default=60.0)
    args = ap.parse_args()
    rank, world, _ = dist_env()
    if args.impl == "reference" and rank != 0:
        return
    if args.form != "plain":
        import __graft_entry__
        __graft_entry__.build()
        fn = {"bf16": bench_bf16, "cosine": bench_cosine, "graph": bench_graph,
              "batched": bench_batched,
              "surrogate": bench_surrogate,
              "balls": bench_balls, "sweep": bench_sweep, "pairmetric": bench_pairmetric}
        print(json.dumps(fn[args.form](args)), flush=True)
        return
    w = make_workload(args.workload, seed=args.seed)
    if args.impl == "reference":
        out = bench_reference(args, w)
    else:
        import __graft_entry__
        __graft_entry__.build()
        out = bench_sng(args, w)
    if out is not None and rank == 0 and args.impl != "reference" and world == 1 \
            and args.extensions:
        out["extensions"] = run_extensions(args)
    if out is not None and rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
