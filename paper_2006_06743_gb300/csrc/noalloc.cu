// noalloc.cu -- SNG-DBSCAN on one small point set without allocating memory.
//
// Why it exists: some callers cannot allocate device memory at the moment
// they need a clustering.  A plugin inside an inference server, a game or
// robotics engine often reserves all device memory up front and forbids
// further cudaMalloc calls; a real-time loop cannot accept cudaMalloc's
// implicit device synchronisation or its failure under memory pressure; and
// code running under another component's allocator must not touch the CUDA
// memory pool.  sng_cluster_noalloc serves those callers: it runs the same
// persistent clustering kernel as the batched form, on a single point set,
// with every byte of scratch taken from a fixed array compiled into this
// library.  The caller still provides the points and the label array.
//
// The scratch array is part of this file's device code.  CUDA loads that code
// on a device when it is first used there (the default lazy module loading),
// which is during the first call of this entry point on that device: the
// driver then reserves the 16 MiB array (and the kernel images) on the
// device, once, and keeps them until the process exits.  That first call can
// therefore fail for lack of device memory; callers that reserve all device
// memory up front make one small call first.  Later calls allocate nothing.
// A point set needs n * (4 * ceil(m / 32) + 10) bytes plus a few kilobytes;
// larger requests are rejected with SNG_EINVAL.
//
// All calls share the one array.  Calls whose work overlaps on the GPU (on
// different streams, or from different host threads without ordering) race
// on it and corrupt each other's results; callers must serialise them.  The
// array keeps the previous call's contents, so every call clears the parts
// that must start at zero (counters, degrees, band flags) before its kernel.
//
// In host code the symbol names a host-side stand-in, not device memory; the
// device address is looked up once per device with cudaGetSymbolAddress, on
// the first call made with that device current.  That first call therefore
// does set-up work and should come before any stream capture.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "batched.cuh"

namespace sng {

constexpr size_t kNoAllocBytes = size_t(16) << 20;  // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once
// per device); nullptr with *err set on failure.
static unsigned char *scratch_base(cudaError_t *err) {
  static std::mutex mu;
  static void *addr[64] = {nullptr};
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[dev] = p;
  }
  return static_cast<unsigned char *>(addr[dev]);
}

// Writes the one-cloud table and its tile list into the scratch array.
__global__ void noalloc_tables_kernel(CloudInfo c, CloudInfo *cloud, int2 *items) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *cloud = c;
  if (t < c.ntiles) items[t] = make_int2(0, t);
}

}  // namespace sng

using namespace sng;

extern "C" {

sng_status sng_cluster_noalloc(const float *x, const sng_params *params, int32_t *labels,
                               sng_stats *stats, void *stream) {
  NvtxRange nvtx_range("sng_cluster_noalloc");
  Resolved r;
  sng_status rc = validate(x, params, &r);
  if (rc) return rc;
  if (!labels) return fail(SNG_EINVAL, "labels is NULL");
  if (params->dtype != SNG_F32) return fail(SNG_EINVAL, "the no-allocation path takes FP32 points");
  if (params->flags & SNG_FLAG_NO_SYNC)
    return fail(SNG_EINVAL, "SNG_FLAG_NO_SYNC is for sng_cluster only");
  if (params->metric != SNG_METRIC_L2)
    return fail(SNG_EINVAL, "the no-allocation path uses the Euclidean ball (metric 0)");
  if (params->degree_mode == SNG_DEG_SIMPLE)
    return fail(SNG_EINVAL, "simple-graph degree needs a pair set; not in the no-allocation path");
  if (r.row_begin != 0 || r.row_end != r.n)
    return fail(SNG_EINVAL, "a source-row range is for sng_build_graph only");
  const int tile = params->map_tile > 0 ? params->map_tile : 1024;
  const int block = params->map_block > 0 ? params->map_block : 256;
  const int64_t n = r.n;
  const int64_t ntiles = (n + tile - 1) / tile;
  // scratch layout, each part 256-byte aligned
  size_t off = 0;
  const size_t o_cloud = off;
  off = align256(off + sizeof(CloudInfo));
  const size_t o_items = off;
  off = align256(off + sizeof(int2) * (size_t)ntiles);
  const size_t o_counters = off;
  off = align256(off + kCntSlots * 8);
  const size_t o_next = off;
  off = align256(off + 2 * sizeof(unsigned int));
  const size_t o_bitmask = off;
  off = align256(off + (size_t)n * r.W * 4);
  const size_t o_deg = off;
  off = align256(off + (size_t)n * 4);
  const size_t o_parent = off;
  off = align256(off + (size_t)n * 4);
  const size_t o_core = off;
  off = align256(off + (size_t)n);
  const size_t o_band = off;
  off = align256(off + (size_t)n);
  if (off > kNoAllocBytes)
    return fail(SNG_EINVAL,
                "n = %lld with m = %lld needs %zu bytes of scratch; the no-allocation path "
                "holds %zu (use sng_cluster)",
                (long long)n, (long long)r.m, off, kNoAllocBytes);
  // the persistent kernel's compiled row shapes: 16-byte rows of up to 16
  // float4 chunks take one chunk per lane (4, 8 or 16 lanes per pair) unless
  // the caller chose the lanes per pair; rows of at most four values (any
  // vector width) take one lane per pair as validate() chose
  BatchMap map{r.map.vec, r.map.group, r.map.nch,
               params->map_unroll > 0 ? params->map_unroll : 4, 0};
  const int chunks = (params->d + r.map.vec - 1) / r.map.vec;
  if (params->map_group == 0 && r.map.vec == 4 && chunks > 1 && chunks <= 16) {
    int g = 4;
    while (g < chunks) g <<= 1;
    map.group = g;
    map.nch = 1;
  }
  // one float4 per row: one lane per source row (as the batched form does),
  // unless one warp per row is asked for
  if (map.vec == 4 && map.group == 1 && map.nch == 1 && (map.unroll == 2 || map.unroll == 4) &&
      !(params->flags & SNG_FLAG_WARP_ROWS))
    map.lanes = 1;
  int occ = 0;
  BatchArgs probe{};
  if (!launch_batched_kernel(map, probe, 0, block, nullptr, &occ))
    return fail(SNG_EINVAL,
                "no compiled persistent mapping for d = %d, ld = %d (vec=%d group=%d nch=%d)",
                params->d, params->ld, map.vec, map.group, map.nch);
  cudaError_t e;
  unsigned char *base = scratch_base(&e);
  if (!base) return cuda_fail(e, "scratch array address");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  CloudInfo c;
  c.off = 0;
  c.bm_off = 0;
  c.seed = params->seed;
  c.fm = make_fastmod(n);
  c.n = (int32_t)n;
  c.m = (int32_t)r.m;
  c.W = r.W;
  c.ntiles = (int32_t)ntiles;
  // clear what must start at zero: counters, work counters, degrees, flags
  cudaMemsetAsync(base + o_counters, 0, kCntSlots * 8, st);
  cudaMemsetAsync(base + o_next, 0, 2 * sizeof(unsigned int), st);
  cudaMemsetAsync(base + o_deg, 0, (size_t)n * 4, st);
  cudaMemsetAsync(base + o_band, 0, (size_t)n, st);
  noalloc_tables_kernel<<<(int)((ntiles + 255) / 256), 256, 0, st>>>(
      c, reinterpret_cast<CloudInfo *>(base + o_cloud), reinterpret_cast<int2 *>(base + o_items));
  note_launch();

  BatchArgs a;
  a.x = x;
  a.ld = params->ld;
  a.d = params->d;
  a.n_items = (int32_t)ntiles;
  a.tile_rows = tile;
  a.min_pts = params->min_pts;
  a.deg_mode = params->degree_mode;
  a.sample_all = params->sample_mode == SNG_SAMPLE_ALL;
  a.lo_thr = r.lo_thr;
  a.hi_thr = r.hi_thr;
  a.eps2 = r.eps2;
  a.band = r.band;
  a.clouds = reinterpret_cast<const CloudInfo *>(base + o_cloud);
  a.items = reinterpret_cast<const int2 *>(base + o_items);
  a.bitmask = reinterpret_cast<uint32_t *>(base + o_bitmask);
  a.deg = reinterpret_cast<int32_t *>(base + o_deg);
  a.parent = reinterpret_cast<int32_t *>(base + o_parent);
  a.core = base + o_core;
  a.band_flag = base + o_band;
  a.labels = labels;
  a.next_item = reinterpret_cast<unsigned int *>(base + o_next);
  a.done = a.next_item + 1;
  a.counters = reinterpret_cast<unsigned long long *>(base + o_counters);
  a.loop_limit = kLoopLimit;
  const int grid = (int)std::min<int64_t>((int64_t)sms * (occ > 0 ? occ : 1), ntiles);
  launch_batched_kernel(map, a, grid, block, st, nullptr);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "no-allocation launch");

  // status word and counters: a plain copy into host memory (no allocation)
  unsigned long long h[kCntSlots];
  e = cudaMemcpyAsync(h, a.counters, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "no-allocation read-back");
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->queries = n * r.m;
    stats->kept_edges = (int64_t)h[kCntEdges];
    stats->band_pairs = (int64_t)h[kCntBandPairs];
    stats->band_points = (int64_t)h[kCntBandPoints];
    stats->cores = (int64_t)h[kCntCores];
    stats->clusters = (int64_t)h[kCntClusters];
    stats->noise = (int64_t)h[kCntNoise];
    stats->recheck_pairs = (int64_t)h[kCntRecheck];
  }
  const uint32_t status = (uint32_t)h[kCntStatus];
  if (status & (kErrUnionLimit | kErrFindLimit | kErrBatchLimit))
    return fail(SNG_ETIMEOUT, "a bounded device loop gave up (status 0x%x)", status);
  if (status) return fail(SNG_EINTERNAL, "device check failed (status 0x%x)", status);
  return SNG_OK;
}

}  // extern "C"
