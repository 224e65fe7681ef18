// batched.cu -- many independent point clouds in one persistent launch.
//
// Algorithm 1 (Jiang, Jang & Lacki 2020, Section 3) runs on every cloud
// separately; the clouds share nothing, so the batch is one work list of
// (cloud, tile of source rows) items handed out by an atomic counter to a
// persistent grid.  For each item a CTA runs step 2 (partner draws, eps-test,
// keep bits, degree atomics) on its rows.  The CTA that completes a cloud's
// last tile (an atomic per-cloud tile counter, preceded by a release fence)
// then runs steps 3-5 for that whole cloud on its own: core mask, union-find
// components over the kept draws (partners re-derived from the hash), border
// labels and noise.  No CTA ever waits for another, so there is no spin loop
// and no deadlock however the hardware schedules the grid.  Items are ordered
// largest cloud first so the per-cloud tails start early.
//
// The plan object validates the cloud table once, lays out scratch, and
// replays the whole batch (memsets + the persistent kernel) as a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "api_common.cuh"
#include "batched.cuh"
#include "graph.cuh"

namespace sng {

// Steps 3-5 for one cloud, by one CTA, after all of its tiles are complete.
__device__ void cloud_components(const BatchArgs &a, const CloudInfo &c) {
  const int32_t n = c.n;
  int32_t *parent = a.parent + c.off;
  uint8_t *core = a.core + c.off;
  int32_t *labels = a.labels + c.off;
  const int32_t *deg = a.deg + c.off;
  const uint32_t *bm = a.bitmask + c.bm_off;
  uint32_t *status = reinterpret_cast<uint32_t *>(a.counters + kCntStatus);

  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint8_t cr = __ldcg(deg + i) >= a.min_pts ? 1 : 0;
    core[i] = cr;
    parent[i] = i;
    labels[i] = cr ? i : kNoLabel;
  }
  __syncthreads();
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    if (!core[i]) continue;
    const uint64_t key = row_key(c.seed, i);
    for (int w = 0; w < c.W; ++w) {
      uint32_t word = __ldcg(bm + (int64_t)i * c.W + w);
      while (word) {
        const int bit = __ffs(word) - 1;
        word &= word - 1;
        const int64_t j = (int64_t)w * 32 + bit;
        const int32_t p = a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, c.fm);
        if (core[p]) uf_unite(parent, i, p, status, a.loop_limit);
      }
    }
  }
  __syncthreads();
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint64_t key = row_key(c.seed, i);
    const bool ci = core[i] != 0;
    int32_t r = ci ? uf_root(parent, i, status, a.loop_limit) : kNoLabel;
    if (ci) labels[i] = r;
    int32_t best = kNoLabel;
    for (int w = 0; w < c.W; ++w) {
      uint32_t word = __ldcg(bm + (int64_t)i * c.W + w);
      while (word) {
        const int bit = __ffs(word) - 1;
        word &= word - 1;
        const int64_t j = (int64_t)w * 32 + bit;
        const int32_t p = a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, c.fm);
        const bool cp = core[p] != 0;
        if (ci && !cp) atomicMin(labels + p, r);
        if (!ci && cp) {
          const int32_t rp = uf_root(parent, p, status, a.loop_limit);
          best = rp < best ? rp : best;
        }
      }
    }
    if (!ci && best != kNoLabel) atomicMin(labels + i, best);
  }
  __syncthreads();
  unsigned long long cores = 0, clusters = 0, noise = 0, band = 0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    int32_t l = __ldcg(labels + i);
    if (l == kNoLabel) {
      l = -1;
      labels[i] = -1;
    }
    const bool ci = core[i] != 0;
    cores += ci;
    clusters += (ci && l == i);
    noise += (l < 0);
    band += __ldcg(a.band_flag + c.off + i) != 0;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    cores += __shfl_xor_sync(kFullMask, cores, o);
    clusters += __shfl_xor_sync(kFullMask, clusters, o);
    noise += __shfl_xor_sync(kFullMask, noise, o);
    band += __shfl_xor_sync(kFullMask, band, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (cores) atomicAdd(a.counters + kCntCores, cores);
    if (clusters) atomicAdd(a.counters + kCntClusters, clusters);
    if (noise) atomicAdd(a.counters + kCntNoise, noise);
    if (band) atomicAdd(a.counters + kCntBandPoints, band);
  }
}

// Lane per row: 4 resident blocks of 256 threads (64 registers; 6 blocks at
// 2 batches in flight fit in 40 registers but measured slower, and 8 in
// flight would leave 2 blocks).  Warp per row: no occupancy bound (the
// compiler's 80 registers measured faster than a 64-register bound).
template <int VEC, int G, int NCH, int U, bool LANES = false>
__global__ void __launch_bounds__(256, LANES ? 4 : 1) batched_kernel(BatchArgs a) {
  extern __shared__ int32_t smem_partner[];
  __shared__ int s_item;
  __shared__ int s_last;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int warps = blockDim.x >> 5;
  int32_t *sp = smem_partner + warp * 64 * U;   // two stages of 32*U partners
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(a.next_item, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= a.n_items) return;
    const int2 it = a.items[item];
    const CloudInfo c = a.clouds[it.x];
    GatherArgs g;
    g.x = a.x + c.off * a.ld;
    g.ld = a.ld;
    g.xm = static_cast<const float *>(g.x);
    g.ldm = a.ld;
    g.n = c.n;
    g.row_begin = 0;
    g.row_end = c.n;
    g.d = a.d;
    g.m = c.m;
    g.W = c.W;
    g.seed = c.seed;
    g.fm = c.fm;
    g.lo_thr = a.lo_thr;
    g.hi_thr = a.hi_thr;
    g.eps2 = a.eps2;
    g.band = a.band;
    g.sample_all = a.sample_all;
    g.deg_mode = a.deg_mode;
    g.m_row = nullptr;
    g.w_row = nullptr;
    g.pf_bytes = 0;
    g.screen = 0;
    g.nrm = nullptr;
    g.nrm_max = nullptr;
    g.bitmask = a.bitmask + c.bm_off;
    g.out_cnt = nullptr;
    g.deg = a.deg + c.off;
    g.band_flag = a.band_flag + c.off;
    g.counters = a.counters;
    const int32_t r0 = it.y * a.tile_rows;
    const int32_t r1 = min(c.n, r0 + a.tile_rows);
    unsigned long long kept = 0;
    if constexpr (LANES) {
      kept = gather_rows_lanes<float, 4, 1, U>(g, r0, r1, lane, warp, warps);
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) kept += __shfl_xor_sync(kFullMask, kept, o);
    } else {
      for (int32_t row = r0 + warp; row < r1; row += warps)
        kept += (unsigned long long)gather_row<float, VEC, G, NCH, U>(g, row, c.m, sp, lane);
    }
    if (lane == 0 && kept) atomicAdd(a.counters + kCntEdges, kept);
    // release this tile's keep bits / degree updates, then count the tile
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int prev = atomicAdd(a.done + it.x, 1u);
      s_last = (prev + 1u == (unsigned int)c.ntiles);
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      cloud_components(a, c);
    }
    __syncthreads();
  }
}


template <int VEC, int G, int NCH, int U, bool LANES = false>
static bool try_batched(const BatchMap &m, const BatchArgs &a, int grid, int block,
                        cudaStream_t st, int *occ) {
  if (m.vec != VEC || m.group != G || m.nch != NCH || m.unroll != U || (m.lanes != 0) != LANES)
    return false;
  const size_t smem = LANES ? 0 : (size_t)(block / 32) * 64 * U * sizeof(int32_t);
  if (occ) {
    *occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, batched_kernel<VEC, G, NCH, U, LANES>,
                                                  block, smem);
    return true;
  }
  batched_kernel<VEC, G, NCH, U, LANES><<<grid, block, smem, st>>>(a);
  return true;
}

// compiled batched mappings: small-d point clouds (thread-per-pair with
// float4 / float2 / scalar rows, or a few lanes per pair up to d = 64)
static bool dispatch_batched(const BatchMap &m, const BatchArgs &a, int grid, int block,
                             cudaStream_t st, int *occ) {
#define SNG_B(V, G, N, U) \
  if (try_batched<V, G, N, U>(m, a, grid, block, st, occ)) return true;
  SNG_B(4, 1, 1, 1) SNG_B(4, 1, 1, 2) SNG_B(4, 1, 1, 4) SNG_B(4, 1, 1, 8)
  SNG_B(4, 4, 1, 4) SNG_B(4, 8, 1, 4) SNG_B(4, 16, 1, 4)
  SNG_B(2, 1, 1, 2) SNG_B(2, 1, 1, 4) SNG_B(2, 1, 2, 4)
  SNG_B(1, 1, 1, 4) SNG_B(1, 1, 2, 4) SNG_B(1, 1, 4, 2) SNG_B(1, 1, 4, 4)
#undef SNG_B
  // one lane per source row (float4 rows)
  if (try_batched<4, 1, 1, 2, true>(m, a, grid, block, st, occ)) return true;
  if (try_batched<4, 1, 1, 4, true>(m, a, grid, block, st, occ)) return true;
  return false;
}

bool launch_batched_kernel(const BatchMap &m, const BatchArgs &a, int grid, int block,
                           cudaStream_t st, int *occ) {
  return dispatch_batched(m, a, grid, block, st, occ);
}

}  // namespace sng

using namespace sng;

struct sng_batch_plan {
  int32_t n_clouds = 0;
  int64_t total = 0;
  int64_t queries = 0;
  sng_params base{};
  Resolved r{};
  BatchMap map{};
  int block = 256;
  int tile_rows = 1024;
  int grid = 1;
  int32_t n_items = 0;
  CloudInfo *d_clouds = nullptr;
  int2 *d_items = nullptr;
  uint32_t *bitmask = nullptr;
  int64_t bitmask_words = 0;
  int32_t *deg = nullptr;
  int32_t *parent = nullptr;
  uint8_t *core = nullptr;
  uint8_t *band_flag = nullptr;
  unsigned int *next_item = nullptr;
  unsigned int *done = nullptr;
  unsigned long long *counters = nullptr;
  cudaStream_t capture = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void *g_x = nullptr;
  int32_t *g_labels = nullptr;
};

namespace sng {

static void plan_free(sng_batch_plan *p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->capture) cudaStreamDestroy(p->capture);
  cudaFree(p->d_clouds);
  cudaFree(p->d_items);
  cudaFree(p->bitmask);
  cudaFree(p->deg);
  cudaFree(p->parent);
  cudaFree(p->core);
  cudaFree(p->band_flag);
  cudaFree(p->next_item);
  cudaFree(p->counters);
  delete p;
}

static sng_status plan_enqueue(sng_batch_plan *p, const void *x, int32_t *labels,
                               cudaStream_t st) {
  cudaMemsetAsync(p->next_item, 0, sizeof(unsigned int) * (1 + (size_t)p->n_clouds), st);
  cudaMemsetAsync(p->counters, 0, kCntSlots * 8, st);
  cudaMemsetAsync(p->deg, 0, (size_t)p->total * 4, st);
  cudaMemsetAsync(p->band_flag, 0, (size_t)p->total, st);
  BatchArgs a;
  a.x = static_cast<const float *>(x);
  a.ld = p->base.ld;
  a.d = p->base.d;
  a.n_items = p->n_items;
  a.tile_rows = p->tile_rows;
  a.min_pts = p->base.min_pts;
  a.deg_mode = p->base.degree_mode;
  a.sample_all = p->base.sample_mode == SNG_SAMPLE_ALL;
  a.lo_thr = p->r.lo_thr;
  a.hi_thr = p->r.hi_thr;
  a.eps2 = p->r.eps2;
  a.band = p->r.band;
  a.clouds = p->d_clouds;
  a.items = p->d_items;
  a.bitmask = p->bitmask;
  a.deg = p->deg;
  a.parent = p->parent;
  a.core = p->core;
  a.band_flag = p->band_flag;
  a.labels = labels;
  a.next_item = p->next_item;
  a.done = p->done;
  a.counters = p->counters;
  a.loop_limit = loop_limit();
  if (!dispatch_batched(p->map, a, p->grid, p->block, st, nullptr))
    return fail(SNG_EINVAL, "no compiled batched mapping vec=%d group=%d nch=%d unroll=%d",
                p->map.vec, p->map.group, p->map.nch, p->map.unroll);
  note_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "batched launch");
}

static sng_status plan_stats(sng_batch_plan *p, sng_stats *stats, cudaStream_t st) {
  Resolved r = p->r;
  r.n = 1;
  r.m = p->queries;
  return read_stats(p->counters, r, stats, st, nullptr);
}

}  // namespace sng

extern "C" {

sng_status sng_batch_plan_create(const int64_t *offsets, int32_t n_clouds, const sng_params *base,
                                 const int64_t *m_per_cloud, sng_batch_plan **plan) {
  NvtxRange nvtx_range("sng_batch_plan_create");
  if (!plan) return fail(SNG_EINVAL, "plan is NULL");
  *plan = nullptr;
  if (!offsets || !base) return fail(SNG_EINVAL, "offsets / base is NULL");
  if (n_clouds < 1) return fail(SNG_EINVAL, "n_clouds must be >= 1");
  if (base->dtype != SNG_F32) return fail(SNG_EINVAL, "batched form takes FP32 points");
  if (base->flags & SNG_FLAG_NO_SYNC)
    return fail(SNG_EINVAL, "SNG_FLAG_NO_SYNC is for sng_cluster only (plans replay as graphs)");
  if (base->metric != SNG_METRIC_L2)
    return fail(SNG_EINVAL, "the batched form uses the Euclidean ball (metric 0)");
  if (base->degree_mode == SNG_DEG_SIMPLE)
    return fail(SNG_EINVAL, "simple-graph degree is not available in the batched form");
  if (base->row_begin != 0 || base->row_end != 0)
    return fail(SNG_EINVAL, "a source-row range is for sng_build_graph only");
  if (offsets[0] != 0) return fail(SNG_EINVAL, "offsets[0] must be 0");
  int64_t nmax = 0;
  for (int32_t b = 0; b < n_clouds; ++b) {
    const int64_t nb = offsets[b + 1] - offsets[b];
    if (nb < 2 || nb > 0x7fffffffLL)
      return fail(SNG_EINVAL, "cloud %d has %lld points (need 2..2^31-1)", b, (long long)nb);
    nmax = std::max(nmax, nb);
  }
  // parameters shared by all clouds, validated on a stand-in cloud
  sng_params probe = *base;
  probe.n = 2;
  probe.m_override = 1;
  probe.sample_mode = SNG_SAMPLE_HASH;
  Resolved r;
  alignas(16) static float aligned_probe[4];
  sng_status rc = validate(aligned_probe, &probe, &r);
  if (rc) return rc;
  if (base->sample_mode == SNG_SAMPLE_HASH && base->m_override <= 0 && !m_per_cloud &&
      !(base->s > 0.0 && base->s <= 1.0))
    return fail(SNG_EINVAL, "s must be in (0, 1]");
  if (base->sample_mode != SNG_SAMPLE_HASH && base->sample_mode != SNG_SAMPLE_ALL)
    return fail(SNG_EINVAL, "unknown sample_mode");

  sng_batch_plan *p = new sng_batch_plan();
  p->n_clouds = n_clouds;
  p->total = offsets[n_clouds];
  p->base = *base;
  p->r = r;
  p->block = base->map_block > 0 ? base->map_block : 256;
  p->tile_rows = base->map_tile > 0 ? base->map_tile : 1024;
  p->map.vec = r.map.vec;
  p->map.group = r.map.group;
  p->map.nch = r.map.nch;
  p->map.unroll = base->map_unroll > 0 ? base->map_unroll : 4;
  // rows of one float4: one lane per source row unless asked otherwise (or
  // unless an unroll the lane-per-row kernel is not compiled for is asked)
  const bool one_vec = p->map.vec == 4 && p->map.nch == 1 && p->map.group == 1;
  const bool lane_unroll = p->map.unroll == 2 || p->map.unroll == 4;
  p->map.lanes = (one_vec && lane_unroll && !(base->flags & SNG_FLAG_WARP_ROWS)) ? 1 : 0;

  std::vector<CloudInfo> clouds(n_clouds);
  int64_t bm = 0, q = 0;
  for (int32_t b = 0; b < n_clouds; ++b) {
    CloudInfo &c = clouds[b];
    const int64_t nb = offsets[b + 1] - offsets[b];
    int64_t mb;
    if (base->sample_mode == SNG_SAMPLE_ALL) mb = nb - 1;
    else if (m_per_cloud) mb = m_per_cloud[b];
    else if (base->m_override > 0) mb = base->m_override;
    else mb = (int64_t)std::ceil(base->s * (double)nb);
    if (mb < 1 || mb > kMaxDraws) {
      plan_free(p);
      return fail(SNG_EINVAL, "cloud %d: draws per point must be >= 1", b);
    }
    c.off = offsets[b];
    c.n = (int32_t)nb;
    c.m = (int32_t)mb;
    c.W = (int32_t)((mb + 31) / 32);
    c.bm_off = bm;
    c.seed = base->seed + (uint64_t)b;
    c.fm = make_fastmod(nb);
    c.ntiles = (int32_t)((nb + p->tile_rows - 1) / p->tile_rows);
    bm += nb * c.W;
    q += nb * mb;
  }
  p->bitmask_words = bm;
  p->queries = q;
  std::vector<int32_t> order(n_clouds);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return clouds[a].n > clouds[b].n; });
  std::vector<int2> items;
  for (int32_t b : order)
    for (int32_t t = 0; t < clouds[b].ntiles; ++t) items.push_back(make_int2(b, t));
  if (items.size() > 0x7fffffffULL) {
    plan_free(p);
    return fail(SNG_EINVAL, "too many work items");
  }
  p->n_items = (int32_t)items.size();

  cudaError_t e = cudaSuccess;
  auto A = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes ? bytes : 16);
  };
  A((void **)&p->d_clouds, sizeof(CloudInfo) * n_clouds);
  A((void **)&p->d_items, sizeof(int2) * items.size());
  A((void **)&p->bitmask, (size_t)bm * 4);
  A((void **)&p->deg, (size_t)p->total * 4);
  A((void **)&p->parent, (size_t)p->total * 4);
  A((void **)&p->core, (size_t)p->total);
  A((void **)&p->band_flag, (size_t)p->total);
  A((void **)&p->next_item, sizeof(unsigned int) * (1 + (size_t)n_clouds));
  A((void **)&p->counters, kCntSlots * 8);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_clouds, clouds.data(), sizeof(CloudInfo) * n_clouds,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_items, items.data(), sizeof(int2) * items.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    plan_free(p);
    return cuda_fail(e, "batched plan scratch");
  }
  p->done = p->next_item + 1;
  int occ = 0;
  BatchArgs dummy{};
  if (!dispatch_batched(p->map, dummy, 0, p->block, nullptr, &occ)) {
    const BatchMap m = p->map;
    plan_free(p);
    return fail(SNG_EINVAL, "no compiled batched mapping vec=%d group=%d nch=%d unroll=%d",
                m.vec, m.group, m.nch, m.unroll);
  }
  p->grid = device_sms() * std::max(1, occ);
  *plan = p;
  return SNG_OK;
}

sng_status sng_batch_run(sng_batch_plan *p, const void *x, int32_t *labels, sng_stats *stats,
                         void *stream) {
  NvtxRange nvtx_range("sng_batch_run");
  if (!p || !x || !labels) return fail(SNG_EINVAL, "NULL argument");
  if ((uintptr_t)x % (p->map.vec * 4)) return fail(SNG_EINVAL, "x_concat misaligned for its rows");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (!p->exec || p->g_x != x || p->g_labels != labels) {
    if (p->exec) {
      cudaGraphExecDestroy(p->exec);
      p->exec = nullptr;
    }
    if (!p->capture && (e = cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking)))
      return cuda_fail(e, "capture stream");
    if ((e = cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal)))
      return cuda_fail(e, "begin capture");
    sng_status rc = plan_enqueue(p, x, labels, p->capture);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(p->capture, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      p->exec = nullptr;
      return cuda_fail(e, "graph instantiate");
    }
    p->g_x = x;
    p->g_labels = labels;
    note_launch(-1);  // the capture recorded, not launched, the kernel
  }
  if ((e = cudaGraphLaunch(p->exec, st))) return cuda_fail(e, "graph launch");
  note_launch();
  if (stats) return plan_stats(p, stats, st);
  return SNG_OK;
}

void sng_batch_plan_destroy(sng_batch_plan *p) {
  if (!p) return;
  cudaDeviceSynchronize();
  plan_free(p);
}

sng_status sng_cluster_batched(const void *x_concat, const int64_t *offsets, int32_t n_clouds,
                               const sng_params *base, const int64_t *m_per_cloud,
                               int32_t *labels, sng_stats *stats, void *stream) {
  if (!x_concat || !labels) return fail(SNG_EINVAL, "NULL argument");
  sng_batch_plan *p = nullptr;
  sng_status rc = sng_batch_plan_create(offsets, n_clouds, base, m_per_cloud, &p);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((uintptr_t)x_concat % (p->map.vec * 4)) {
    plan_free(p);
    return fail(SNG_EINVAL, "x_concat misaligned for its rows");
  }
  rc = plan_enqueue(p, x_concat, labels, st);
  if (!rc) rc = plan_stats(p, stats, st);
  cudaStreamSynchronize(st);
  plan_free(p);
  return rc;
}

}  // extern "C"
