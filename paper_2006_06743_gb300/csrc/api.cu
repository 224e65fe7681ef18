// api.cu -- the extern "C" entry points of libsng.so (declared in include/sng.h).
//
// Host-side work only: argument validation, the gather mapping policy, the
// FP32 guard band, device scratch (stream-ordered pool allocations) and the
// order of kernel launches for Algorithm 1 (Jiang, Jang & Lacki 2020, Sec. 3).
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "api_common.cuh"
#include "gather.cuh"
#include "graph.cuh"
#include "gather_mma.cuh"
#include "gather_mma8.cuh"
#include "gather_pair.cuh"
#include "screen_queue.cuh"
#include "gather_tc05.cuh"
#include "screen.cuh"
#include "tiled.cuh"

namespace sng {

static std::atomic<int64_t> g_launches{0};
void note_launch(int count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

static thread_local std::string g_last_error;

// Copies of the point coordinates still in flight on other streams (the
// host-buffer entry point's input pieces): the first kernel that reads the
// coordinates waits for them, so work that does not (the tiled form's
// partition) overlaps the copy.
static thread_local std::vector<cudaEvent_t> g_inputs_pending;

void wait_inputs(cudaStream_t st) {
  for (cudaEvent_t ev : g_inputs_pending) cudaStreamWaitEvent(st, ev, 0);
  g_inputs_pending.clear();
}

sng_status fail(sng_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

sng_status cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(SNG_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(SNG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int device_sms() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  std::lock_guard<std::mutex> lk(mu);
  if (!cache[dev]) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = sms > 0 ? sms : 148;
    // keep freed pool memory for reuse instead of releasing it to the OS
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  return cache[dev];
}

// ------------------------------------------------------------- scratch

Scratch::~Scratch() { release(); }

void Scratch::release() {
  if (!textures.empty()) {
    cudaStreamSynchronize(stream);
    for (unsigned long long t : textures) cudaDestroyTextureObject((cudaTextureObject_t)t);
    textures.clear();
  }
  for (void *p : ptrs) cudaFreeAsync(p, stream);
  ptrs.clear();
}

sng_status Scratch::alloc(void **out, size_t bytes, const char *what) {
  *out = nullptr;
  const char *fault = std::getenv("SNG_FAULT_ALLOC");
  if (fault && *fault) {
    // SNG_FAULT_ALLOC=k: host-side fault injection for tests.  The k-th
    // scratch allocation counted from the moment this value was set fails.
    static std::mutex mu;
    static std::string seen;
    static int64_t count = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (seen != fault) {
      seen = fault;
      count = 0;
    }
    if (++count == std::atoll(fault))
      return fail(SNG_ENOMEM, "injected allocation failure (%s)", what);
  }
  void *p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes ? bytes : 16, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, what);
  }
  ptrs.push_back(p);
  *out = p;
  return SNG_OK;
}

// ------------------------------------------------------------ validation

static int64_t ceil_s_n(double s, int64_t n) { return (int64_t)std::ceil(s * (double)n); }

// Smallest float not below v.
static float round_up_f(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, INFINITY);
  return f;
}

// FP32 guard band around eps^2 for a squared distance summed with `fmas`
// fused multiply-adds per lane and `levels` shuffle levels: twice a bound on
// the relative error (one rounding for each difference, one per fused
// multiply-add, one per level, plus slack) and the reported band; the FP32
// thresholds are rounded outwards.
static void fp32_guard(double eps2, float band_rel, int fmas, int levels, float *lo_thr,
                       float *hi_thr) {
  const double u = std::ldexp(1.0, -24);
  const double delta = 2.0 * (double)(fmas + levels + 3) * u + std::ldexp(1.0, -22);
  const double screen = (double)band_rel + delta;
  const double lo = eps2 * (1.0 - screen), hi = eps2 * (1.0 + screen);
  float lof = (float)lo, hif = (float)hi;
  if ((double)lof > lo) lof = std::nextafter(lof, 0.f);
  if ((double)hif < hi) hif = std::nextafter(hif, INFINITY);
  *lo_thr = lof;
  *hi_thr = hif;
}

sng_status validate(const void *x, const sng_params *p, Resolved *r) {
  if (!p) return fail(SNG_EINVAL, "params is NULL");
  if (!x) return fail(SNG_EINVAL, "x is NULL");
  if (p->n < 2 || p->n > 0x7fffffffLL) return fail(SNG_EINVAL, "n must be in [2, 2^31-1]");
  if (p->d < 1) return fail(SNG_EINVAL, "d must be >= 1");
  if (p->ld < p->d) return fail(SNG_EINVAL, "ld must be >= d");
  if (p->dtype != SNG_F32 && p->dtype != SNG_BF16) return fail(SNG_EINVAL, "unknown dtype");
  if (p->degree_mode != SNG_DEG_UNDIRECTED_MULTI && p->degree_mode != SNG_DEG_OUT &&
      p->degree_mode != SNG_DEG_SIMPLE)
    return fail(SNG_EINVAL, "unknown degree_mode");
  if (p->sample_mode != SNG_SAMPLE_HASH && p->sample_mode != SNG_SAMPLE_ALL)
    return fail(SNG_EINVAL, "unknown sample_mode");
  if (p->min_pts < 1) return fail(SNG_EINVAL, "min_pts must be >= 1");
  if (p->metric != SNG_METRIC_L2 && p->metric != SNG_METRIC_DOT &&
      p->metric != SNG_METRIC_COSINE && p->metric != SNG_METRIC_L1 &&
      p->metric != SNG_METRIC_LINF)
    return fail(SNG_EINVAL, "unknown metric");
  const bool pair_metric = p->metric == SNG_METRIC_L1 || p->metric == SNG_METRIC_LINF;
  if (!std::isfinite(p->eps)) return fail(SNG_EINVAL, "eps must be finite");
  if ((p->metric == SNG_METRIC_L2 || pair_metric) && (p->eps < 1e-15f || p->eps > 1e18f))
    return fail(SNG_EINVAL, "eps must be in [1e-15, 1e18]");
  if (pair_metric && p->dtype != SNG_F32)
    return fail(SNG_EINVAL, "the Manhattan and Chebyshev forms take FP32 points");
  if (p->metric != SNG_METRIC_L2 && p->map_passes > 1)
    return fail(SNG_EINVAL, "the similarity form runs in one pass (map_passes <= 1)");
  if (p->flags & SNG_FLAG_NO_SYNC) {
    if (p->flags & SNG_FLAG_TIMING)
      return fail(SNG_EINVAL, "phase timing reads events on the host: not with SNG_FLAG_NO_SYNC");
    if (p->degree_mode == SNG_DEG_SIMPLE)
      return fail(SNG_EINVAL, "the distinct-neighbour degree sizes its pair set from E: "
                              "not with SNG_FLAG_NO_SYNC");
  }
  if (!(p->band_rel >= 0.f) || p->band_rel > 0.25f)
    return fail(SNG_EINVAL, "band_rel must be in [0, 0.25]");
  const size_t esize = p->dtype == SNG_F32 ? 4 : 2;
  if ((uintptr_t)x % esize) return fail(SNG_EINVAL, "x is not aligned to its element size");
  if (p->dtype == SNG_BF16) {
    if (!p->x_f32_master) return fail(SNG_EINVAL, "BF16 form needs x_f32_master");
    if ((uintptr_t)p->x_f32_master % 4) return fail(SNG_EINVAL, "x_f32_master misaligned");
  }
  int64_t m;
  if (p->sample_mode == SNG_SAMPLE_ALL) {
    m = p->n - 1;
  } else if (p->m_override > 0) {
    m = p->m_override;
  } else {
    if (!(p->s > 0.0) || !(p->s <= 1.0)) return fail(SNG_EINVAL, "s must be in (0, 1]");
    m = ceil_s_n(p->s, p->n);
  }
  if (m < 1 || m > kMaxDraws) return fail(SNG_EINVAL, "m must be in [1, 2^31-1025]");
  r->n = p->n;
  r->d = p->d;
  r->m = m;
  r->W = (int32_t)((m + 31) / 32);
  r->band_rel = p->band_rel > 0.f ? p->band_rel : (p->dtype == SNG_BF16 ? 1e-3f : 1e-5f);

  // gather mapping: widest aligned vector, then lanes per pair
  const int vmax = p->dtype == SNG_F32 ? 4 : 8;
  int vec = vmax;
  while (vec > 1 && ((p->ld % vec) != 0 || ((uintptr_t)x % (vec * esize)) != 0)) vec >>= 1;
  const int chunks = (p->d + vec - 1) / vec;
  int group, nch;
  auto pow2ceil = [](int v) {
    int q = 1;
    while (q < v) q <<= 1;
    return q;
  };
  if (p->map_group > 0) {
    group = p->map_group;
    if (group > 32 || (group & (group - 1))) return fail(SNG_EINVAL, "map_group must be 1..32, pow2");
    nch = pow2ceil((chunks + group - 1) / group);
  } else if (chunks <= 4) {
    // thread per pair: the whole row in one lane
    group = 1;
    nch = pow2ceil(chunks);
  } else if (vec == vmax) {
    // about 16 elements of the row per lane (4 float4 or 2 x 8 bf16 chunks):
    // enough pairs per warp step to amortise the group reduction and the
    // ballot, few enough registers for 3-4 blocks per SM (the autotuner's
    // winners at d = 64 FP32 and d = 128 BF16)
    const int per_lane = 16 / vec;
    group = pow2ceil((chunks + per_lane - 1) / per_lane);
    if (group > 32) group = 32;
    nch = pow2ceil((chunks + group - 1) / group);
  } else {
    // rows that cannot use 16-byte vectors: widest groups first
    group = pow2ceil(chunks);
    if (group > 32) group = 32;
    nch = pow2ceil((chunks + group - 1) / group);
  }
  if (nch > 8)
    return fail(SNG_EINVAL, "d = %d is wider than the compiled gather mappings (d <= %d)", p->d,
                32 * 8 * vec);
  r->map.vec = vec;
  r->map.group = group;
  r->map.nch = nch;
  r->map.sim = p->metric != SNG_METRIC_L2;
  r->map.full = group * nch * vec == p->d;
  r->map.unroll = p->map_unroll > 0 ? p->map_unroll : (vec == vmax && nch * vec >= 16 ? 2 : 4);
  // one lane per pair and short rows: one lane per source row (compiled for
  // 2 and 4 partner rows in flight), unless one warp per row is asked for or
  // there are too few rows (32 rows per warp).  Hashed draws want 64 warps
  // per SM (with fewer a warp per row hides latency better: measured slower
  // at 10^5 rows, faster at 10^6); with every pair queried the 32 lanes walk
  // the same partners and 16 warps per SM suffice (faster at 10^5 rows).
  const int64_t rows = (p->row_begin == 0 && p->row_end == 0) ? p->n : p->row_end - p->row_begin;
  const int64_t min_warps_per_sm = p->sample_mode == SNG_SAMPLE_ALL ? 16 : 64;
  r->map.lanes = group == 1 && p->metric == SNG_METRIC_L2 &&
                 (r->map.unroll == 2 || r->map.unroll == 4) &&
                 !(p->flags & SNG_FLAG_WARP_ROWS) &&
                 rows >= 32LL * min_warps_per_sm * device_sms();
  if (p->map_passes < 0 || p->map_passes > 64) return fail(SNG_EINVAL, "map_passes must be in [0, 64]");
  r->map.passes = p->map_passes > 0 ? p->map_passes : 1;
  if (r->map.passes > p->n) r->map.passes = (int)p->n;
  r->map.block = p->map_block > 0 ? p->map_block : 256;
  if (r->map.block % 32 || r->map.block < 32 || r->map.block > 256)
    return fail(SNG_EINVAL, "map_block must be a multiple of 32 in [32, 256]");
  if (p->map_tile < 0) return fail(SNG_EINVAL, "map_tile must be >= 0");
  if (p->row_begin == 0 && p->row_end == 0) {
    r->row_begin = 0;
    r->row_end = p->n;
  } else {
    if (p->row_begin < 0 || p->row_begin > p->row_end || p->row_end > p->n)
      return fail(SNG_EINVAL, "need 0 <= row_begin <= row_end <= n");
    r->row_begin = p->row_begin;
    r->row_end = p->row_end;
  }

  // eps^2 in FP64 exactly as the oracle forms it; the FP32 screen is widened
  // by twice a bound on the FP32 relative error of the kernel's sum: one
  // rounding for the difference, one per fused multiply-add in a lane
  // (nch*vec), one per shuffle level (log2 group), plus slack.
  r->eps2 = (double)p->eps * (double)p->eps;
  r->band = (double)r->band_rel * r->eps2;
  int lg = 0;
  while ((1 << lg) < group) ++lg;
  const double u = std::ldexp(1.0, -24);
  fp32_guard(r->eps2, r->band_rel, nch * vec, lg, &r->lo_thr, &r->hi_thr);

  // similarity form: |dot32 - dot| <= (K + 1) u sum|a_k b_k| <= (K + 1) u
  // |a| |b| with K roundings per term (nch*vec fused multiply-adds, log2
  // group shuffle levels).  The squared norms are summed with the same K
  // roundings, so |a| |b| from them (and its correctly rounded square roots
  // and products) is within a few K u relative; c1 = twice the bound plus
  // 2^-22 covers that and the FP64 result's own rounding.  With both norms
  // in [2^-50, 2^50] products that underflow cost at most K 2^-150 absolute,
  // far below c1 |a| |b|.  Cosine divides by |a| |b| through two reciprocal
  // square roots within e_inv = (K/2 + 5) u each, adding c2 |cos32|.  All
  // constants are rounded up.
  r->metric = p->metric;
  if (p->metric != SNG_METRIC_L2) {
    const double tau = (double)p->eps;
    r->band = (double)r->band_rel * std::fabs(tau);
    const double c1 = 2.0 * (double)(nch * vec + lg + 3) * u + std::ldexp(1.0, -22);
    // rsqrtf is within 2 ulp = 4u (CUDA's documented bound)
    const double e_inv = ((double)(nch * vec + lg) / 2.0 + 5.0) * u;
    const double c2 = p->metric == SNG_METRIC_COSINE ? 2.0 * (2.0 * e_inv + 3.0 * u) : 0.0;
    auto up = [](double v) {
      float f = (float)v;
      if ((double)f < v) f = std::nextafter(f, INFINITY);
      return f;
    };
    r->sim_c1 = up(c1);
    r->sim_c2 = up(c2);
    r->band_f = up(r->band);
  }
  // Manhattan / Chebyshev distance: one lane sums |a_k - b_k| in order (each
  // difference and each addition rounded once: within (d + 1) u relative of
  // the exact sum of the non-negative terms) or takes their maximum (each
  // term within u); the FP32 value decides outside the guard band eps (1 -+
  // (band_rel + c)), c twice that bound plus 2^-22 for the FP64 result's own
  // rounding, the thresholds rounded outwards; inside it the FP64 value does.
  if (pair_metric) {
    const double c = (p->metric == SNG_METRIC_L1 ? 2.0 * (double)(p->d + 2) : 4.0) * u +
                     std::ldexp(1.0, -22);
    const double eps = (double)p->eps;
    const double lo = eps * (1.0 - (double)r->band_rel - c);
    const double hi = eps * (1.0 + (double)r->band_rel + c);
    float lof = (float)lo, hif = (float)hi;
    if ((double)lof > lo) lof = std::nextafter(lof, 0.f);
    if ((double)hif < hi) hif = std::nextafter(hif, INFINITY);
    r->lo_thr = lof;
    r->hi_thr = hif;
  }
  return SNG_OK;
}

bool fill_gather_args(const void *x, const sng_params *p, const Resolved &r, GatherArgs *g) {
  g->x = x;
  g->ld = p->ld;
  g->xm = p->dtype == SNG_F32 ? static_cast<const float *>(x) : p->x_f32_master;
  g->ldm = p->ld;
  g->n = (int32_t)r.n;
  g->row_begin = (int32_t)r.row_begin;
  g->row_end = (int32_t)r.row_end;
  g->d = r.d;
  g->m = (int32_t)r.m;
  g->W = r.W;
  g->seed = p->seed;
  g->fm = make_fastmod(r.n);
  g->lo_thr = r.lo_thr;
  g->hi_thr = r.hi_thr;
  g->eps2 = r.eps2;
  g->band = r.band;
  g->sample_all = p->sample_mode == SNG_SAMPLE_ALL;
  g->deg_mode = p->degree_mode;
  g->m_row = nullptr;
  g->w_row = nullptr;
  g->cosine = p->metric == SNG_METRIC_COSINE;
  g->tau = p->eps;
  g->tau64 = (double)p->eps;
  g->sim_c1 = r.sim_c1;
  g->sim_c2 = r.sim_c2;
  g->band_f = r.band_f;
  g->screen = 0;
  g->screen_vec4 = 0;
  g->screen_lo_eps = g->screen_hi_eps = 0.f;
  g->screen_u = g->screen_abs = g->screen_g = 0.f;
  g->screen_kexp = nullptr;
  g->nbe = nullptr;
  g->err_max = nullptr;
  g->openq = nullptr;
  g->openq_cnt = nullptr;
  g->openq_cap = 0;
  g->q_lo_thr = g->q_hi_thr = 0.f;
  g->sim_screen = 0;
  g->sim_keep_thr = g->sim_drop_thr = g->sim_cm = 0.f;
  g->nrm = nullptr;
  g->nrm_max = nullptr;
  // L2 prefetch of partner rows when rows start on 16 bytes (16-byte vectors)
  const int esize = p->dtype == SNG_F32 ? 4 : 2;
  g->pf_bytes = 0;
  if (r.map.vec * esize == 16 && (p->flags & SNG_FLAG_PREFETCH))
    g->pf_bytes = ((r.d * esize + 15) / 16) * 16;
  return true;
}

int gather_grid(int dtype, const GatherMap &map, int64_t n) {
  const int sms = device_sms();
  int per_sm = map.passes > 1 ? gather_blocked_max_blocks_per_sm(dtype, map)
                              : gather_max_blocks_per_sm(dtype, map);
  if (per_sm < 1) per_sm = 1;
  const int64_t warps_per_block = map.block / 32;
  const int64_t rows_per_warp = map.lanes ? 32 : 1;
  int64_t need = (n + warps_per_block * rows_per_warp - 1) / (warps_per_block * rows_per_warp);
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > need) grid = need;
  return (int)(grid < 1 ? 1 : grid);
}

// Steps shared by sng_build_graph and sng_cluster: the gather (step 2 with the
// degree counts of step 3), the row-pointer scan and the CSR fill.
// Degrees of the simple undirected graph of an edge list (deg is
// overwritten; counters receives device status bits).
sng_status simple_degrees(int64_t n, const int32_t *src, const int32_t *col, int64_t num_edges,
                          int32_t *deg, unsigned long long *counters, Scratch &s) {
  cudaStream_t st = s.stream;
  cudaMemsetAsync(deg, 0, (size_t)n * 4, st);
  if (num_edges == 0) return SNG_OK;
  const uint64_t cap = simple_table_slots(num_edges);
  unsigned long long *table = nullptr;
  sng_status rc;
  if ((rc = s.alloc((void **)&table, (size_t)cap * 8, "pair set"))) return rc;
  cudaMemsetAsync(table, 0xff, (size_t)cap * 8, st);
  SimpleDegArgs a{n, src, col, num_edges, table, cap - 1, deg, counters};
  launch_simple_degree(a, device_sms(), st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "simple-degree launch");
}

// The L2-tiled gather (SNG_FLAG_TILED): partition every draw into k x k tile
// buckets, then test tile by tile.  *done = false when the form does not
// apply or a bucket overflowed (the caller runs the direct gather).
static sng_status run_tiled(const sng_params *p, const Resolved &r, Scratch &s,
                            const GatherArgs &ga, GraphBufs *gb, bool *done,
                            const Shadow *sh) {
  *done = false;
  cudaStream_t st = s.stream;
  const int64_t n = r.n;
  const int blocks = tile_test_blocks_per_sm(p->dtype, r.map);
  // not for the similarity form, one lane per row or slice passes; and not
  // in the no-sync form (the overflow check reads the status on the host)
  if (blocks < 0 || r.map.sim || r.map.lanes || r.map.passes > 1 ||
      (p->flags & SNG_FLAG_NO_SYNC))
    return SNG_OK;
  const size_t esize = p->dtype == SNG_F32 ? 4 : 2;
  int k = p->map_tile > 0 ? p->map_tile
                          : (int)((2 * (int64_t)n * p->ld * esize + (88ll << 20) - 1) / (88ll << 20));
  if (k < 2) k = 2;
  if (k > kMaxTiles) k = kMaxTiles;
  const int64_t slice = (n + k - 1) / k;
  const int tiles = k * k;
  std::vector<int64_t> cap(tiles), eoff(tiles), roff(tiles);
  int64_t etot = 0, rtot = 0;
  for (int b = 0; b < tiles; ++b) {
    const int rs = b / k, ps = b % k;
    const int64_t rows = std::max<int64_t>(0, std::min<int64_t>(slice, n - (int64_t)rs * slice));
    const int64_t plen = std::max<int64_t>(0, std::min<int64_t>(slice, n - (int64_t)ps * slice));
    double expect;
    if (p->sample_mode == SNG_SAMPLE_ALL)
      expect = (double)rows * (double)plen;   // every other point once: at most plen per row
    else
      expect = (double)rows * (double)r.m * (double)plen / (double)(n - 1);
    cap[b] = (int64_t)(expect + 8.0 * std::sqrt(expect) + 1024.0);
    eoff[b] = etot;
    roff[b] = rtot;
    etot += cap[b];
    rtot += rows;
  }
  int64_t *d_cap = nullptr, *d_eoff = nullptr, *d_roff = nullptr;
  unsigned long long *d_entries = nullptr, *d_cursor = nullptr;
  int4 *d_runs = nullptr;
  unsigned int *d_rcur = nullptr;
  sng_status rc;
  if ((rc = s.alloc((void **)&d_entries, (size_t)etot * 8, "tile buckets")) ||
      (rc = s.alloc((void **)&d_runs, (size_t)(rtot > 0 ? rtot : 1) * 16, "tile runs")) ||
      (rc = s.alloc((void **)&d_cap, (size_t)tiles * 8, "tile capacities")) ||
      (rc = s.alloc((void **)&d_eoff, (size_t)tiles * 8, "tile offsets")) ||
      (rc = s.alloc((void **)&d_roff, (size_t)tiles * 8, "tile run offsets")) ||
      (rc = s.alloc((void **)&d_cursor, (size_t)tiles * 8, "tile cursors")) ||
      (rc = s.alloc((void **)&d_rcur, (size_t)tiles * 4, "tile run cursors")))
    // no room for the buckets (about 8.4 bytes per draw): the direct gather
    // runs instead, as for any case the tiled form does not cover
    return rc == SNG_ENOMEM ? SNG_OK : rc;
  cudaMemcpyAsync(d_cap, cap.data(), (size_t)tiles * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_eoff, eoff.data(), (size_t)tiles * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_roff, roff.data(), (size_t)tiles * 8, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(d_cursor, 0, (size_t)tiles * 8, st);
  cudaMemsetAsync(d_rcur, 0, (size_t)tiles * 4, st);
  TileArgs t{k, slice, d_entries, d_eoff, d_cap, d_cursor, d_runs, d_roff, d_rcur, 0, 0};
  // FP32 rows: one of each partner row's four 16-byte chunks comes through
  // the texture unit, whose data path runs beside the load/store unit's (the
  // tile test is bound by the latter; one chunk in four measured fastest)
  // (compiled for full rows with four lanes per pair and two steps in flight)
  if (p->dtype == SNG_F32 && r.map.vec == 4 && r.map.group == 4 && r.map.nch == 4 &&
      r.map.unroll == 2 && r.map.full) {
    int dev = 0, align = 0, width = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&align, cudaDevAttrTextureAlignment, dev);
    cudaDeviceGetAttribute(&width, cudaDevAttrMaxTexture1DLinearWidth, dev);
    // the rows' extent, (n - 1) * ld + d floats (d = 64 here; ld % 4 == 0)
    const int64_t texels = ((n - 1) * p->ld + p->d) / 4;
    if (align > 0 && (uintptr_t)ga.x % (uintptr_t)align == 0 && texels <= (int64_t)width) {
      cudaResourceDesc rd{};
      rd.resType = cudaResourceTypeLinear;
      rd.res.linear.devPtr = const_cast<void *>(ga.x);
      rd.res.linear.desc = cudaCreateChannelDesc<float4>();
      rd.res.linear.sizeInBytes = (size_t)texels * 16;
      cudaTextureDesc td{};
      td.readMode = cudaReadModeElementType;
      cudaTextureObject_t tex = 0;
      if (cudaCreateTextureObject(&tex, &rd, &td, nullptr) == cudaSuccess) {
        s.textures.push_back((unsigned long long)tex);
        t.tex = (unsigned long long)tex;
        t.tex_chunks = 1;
      } else {
        cudaGetLastError();
      }
    }
  }
  // the BF16 screen bounds each tile's partners by its slice's largest norm
  if (sh && (rc = shadow_slice_max(*sh, n, slice, k, st))) return rc;
  launch_tile_partition(ga, t, device_sms() * 16, st);
  note_launch();
  // a bucket overflow (far outside the binomial spread) falls back
  unsigned long long status = 0;
  cudaError_t e = cudaMemcpyAsync(&status, gb->counters + kCntStatus, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "tile partition");
  if (status & kErrTileOverflow) {
    cudaMemsetAsync(gb->counters + kCntStatus, 0, 8, st);
    return SNG_OK;
  }
  // the test kernels set keep bits and add counts: both start at zero
  cudaMemsetAsync(gb->bitmask, 0, (size_t)n * r.W * 4, st);
  cudaMemsetAsync(gb->out_cnt, 0, (size_t)n * 4, st);
  const int grid = device_sms() * (blocks > 0 ? blocks : 1);
  wait_inputs(st);   // the partition read no coordinates; the tests do
  for (int b = 0; b < tiles; ++b) {
    if (!launch_tile_test(p->dtype, r.map, ga, t, b, grid, st))
      return fail(SNG_EINTERNAL, "tile test mapping vanished");
    note_launch();
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tile test launches");
  gb->tiles = k;
  gb->tex_chunks = t.tex_chunks;
  *done = true;
  return SNG_OK;
}

sng_status run_graph(const void *x, const sng_params *p, const Resolved &r, Scratch &s,
                     GraphBufs *gb, const int32_t *m_row, Timer *tm, const int32_t *w_row) {
  cudaStream_t st = s.stream;
  const int64_t n = r.n;
  sng_status rc;
  if ((rc = s.alloc((void **)&gb->bitmask, (size_t)n * r.W * 4, "keep bits"))) return rc;
  if ((rc = s.alloc((void **)&gb->out_cnt, (size_t)n * 4, "row counts"))) return rc;
  if ((rc = s.alloc((void **)&gb->deg, (size_t)n * 4, "degrees"))) return rc;
  if ((rc = s.alloc((void **)&gb->band_flag, (size_t)n, "band flags"))) return rc;
  if ((rc = s.alloc((void **)&gb->counters, kCntSlots * 8, "counters"))) return rc;
  if ((rc = s.alloc((void **)&gb->tile_tmp, (size_t)scan_tiles(n) * 8, "scan tiles"))) return rc;
  if ((rc = s.alloc((void **)&gb->row_ptr, (size_t)(n + 1) * 8, "row_ptr"))) return rc;
  cudaMemsetAsync(gb->deg, 0, (size_t)n * 4, st);
  cudaMemsetAsync(gb->band_flag, 0, (size_t)n, st);
  cudaMemsetAsync(gb->counters, 0, kCntSlots * 8, st);

  GatherArgs ga;
  fill_gather_args(x, p, r, &ga);
  ga.m_row = m_row;
  ga.w_row = w_row;
  ga.bitmask = gb->bitmask;
  ga.out_cnt = gb->out_cnt;
  ga.deg = gb->deg;
  ga.band_flag = gb->band_flag;
  ga.counters = gb->counters;
  if (r.map.passes > 1 || r.row_begin > 0 || r.row_end < n) {
    // rows outside the processed range (or filled slice by slice) start empty
    cudaMemsetAsync(gb->bitmask, 0, (size_t)n * r.W * 4, st);
    cudaMemsetAsync(gb->out_cnt, 0, (size_t)n * 4, st);
  }
  tm->mark(st, 0);
  NvtxRange nvtx_graph("step 2: sampled graph");
  // The BF16 screen (SNG_FLAG_SCREEN16): the gather runs over a BF16 copy
  // of the FP32 points with the BF16 mapping; the FP32 points stay the
  // source of every decision the screen leaves open.
  const sng_params *pg = p;   // parameters the gather's mapping follows
  const Resolved *rg = &r;
  sng_params pb;
  Resolved rb;
  Shadow sh;
  const bool pair_metric = p->metric == SNG_METRIC_L1 || p->metric == SNG_METRIC_LINF;
  const bool sim = p->metric != SNG_METRIC_L2 && !pair_metric;
  // (no host read on this path: the no-sync form and graph capture keep it;
  // only the tiled form below needs one)
  const bool want_screen = (p->flags & (SNG_FLAG_SCREEN16 | SNG_FLAG_SCREEN8)) &&
                           p->dtype == SNG_F32 && r.map.passes <= 1 && !r.map.lanes &&
                           !pair_metric;
  // the FP8 form: k-tiles of 32 values (rows of 64 or 128 bytes)
  const int fp8_ks = want_screen && (p->flags & SNG_FLAG_SCREEN8) && p->d <= 128
                         ? (p->d <= 64 ? 2 : 4) : 0;
  const int mma_kt = want_screen && !fp8_ks &&
                             (p->flags & (SNG_FLAG_SCREEN_MMA | SNG_FLAG_SCREEN8))
                         ? mma_tiles_for(p->d) : 0;
  // the similarity metrics are screened by the tensor-core forms only
  const bool screen = want_screen && (!sim || fp8_ks || mma_kt);
  // the TMA + tcgen05 form reads rows of 64 BF16 values (zero past d);
  // Euclidean only
  const bool tc05 = mma_kt && !sim && (p->flags & SNG_FLAG_TCGEN05) && p->d <= 64;
  // Manhattan / Chebyshev distance: the BF16 copy screened on CUDA cores
  // (either screen flag; gather_pair.cu)
  const bool pair_screen =
      pair_metric && (p->flags & (SNG_FLAG_SCREEN16 | SNG_FLAG_SCREEN8)) && p->dtype == SNG_F32;
  if (screen) {
    wait_inputs(st);
    if (fp8_ks) {
      if ((rc = make_shadow8(static_cast<const float *>(x), p->ld, p->d, n, 32 * fp8_ks, s, &sh)))
        return rc;
    } else if ((rc = make_shadow(static_cast<const float *>(x), p->ld, p->d, n,
                                 tc05 ? 64 : 16 * mma_kt, s, &sh))) {
      return rc;
    }
    pb = *p;
    pb.dtype = SNG_BF16;
    pb.ld = (int32_t)sh.ldb;
    pb.x_f32_master = static_cast<const float *>(x);
    pb.band_rel = r.band_rel;
    if ((rc = validate(sh.xb, &pb, &rb))) return rc;
    rb.map.lanes = 0;
    fill_gather_args(sh.xb, &pb, rb, &ga);
    ga.m_row = m_row;
    ga.w_row = w_row;
    ga.bitmask = gb->bitmask;
    ga.out_cnt = gb->out_cnt;
    ga.deg = gb->deg;
    ga.band_flag = gb->band_flag;
    ga.counters = gb->counters;
    ga.xm = static_cast<const float *>(x);
    ga.ldm = p->ld;
    ga.eps2 = r.eps2;
    ga.band = r.band;
    ga.screen = 1;
    ga.screen_vec4 = (p->d % 4 == 0) && (p->ld % 4 == 0) && ((uintptr_t)x % 16 == 0);
    {
      float lo_e = (float)((double)p->eps * std::sqrt(1.0 - (double)r.band_rel));
      if ((double)lo_e > (double)p->eps * std::sqrt(1.0 - (double)r.band_rel))
        lo_e = std::nextafter(lo_e, 0.f);
      ga.screen_lo_eps = lo_e;
      ga.screen_hi_eps = round_up_f((double)p->eps * std::sqrt(1.0 + (double)r.band_rel));
    }
    ga.nrm = sh.nrm;
    ga.nrm_max = sh.nmax;
    ga.nb2 = sh.nb2;
    ga.nbe = sh.nbe;
    ga.err_max = sh.nmax + kErrMaxSlot;
    ga.screen_cabs = std::ldexp(1.0f, -15);
    // the FP32 sum over the BF16 values: one rounding per difference, one
    // per fused multiply-add in a lane, one per shuffle level (as the
    // plain guard band); g adds 2^-20 for the rounding of the thresholds
    // themselves and of the FP64 reference decision
    int lg = 0;
    while ((1 << lg) < rb.map.group) ++lg;
    const double u = std::ldexp(1.0, -24);
    const double delta = 2.0 * (double)(rb.map.nch * rb.map.vec + lg + 3) * u + std::ldexp(1.0, -22);
    ga.screen_g = round_up_f(delta + std::ldexp(1.0, -20));
    ga.screen_u = round_up_f(std::ldexp(1.0, -8) * (1.0 + std::ldexp(1.0, -20)));
    ga.screen_abs = std::ldexp(1.0f, -60);
    if (fp8_ks) {
      // E4M3: eta from the rows' own rounding-error bounds (nbe), and a
      // wider allowance for the FP8 tensor core's accumulation
      ga.screen_u = 0.f;
      ga.screen_kexp = sh.kexp;
      ga.screen_cabs = std::ldexp(1.0f, -9);
    }
    if (sim) {
      // keep at or above tau + band, drop below tau - band (the band
      // widened by 2^-20, the thresholds rounded outwards); the MMA's
      // accumulation allowance as for the Euclidean form's c_abs
      const double tau = (double)p->eps;
      const double bw = (double)r.band * (1.0 + std::ldexp(1.0, -20));
      ga.sim_screen = 1;
      ga.sim_keep_thr = round_up_f(tau + bw);
      float dt = (float)(tau - bw);
      if ((double)dt > tau - bw) dt = std::nextafter(dt, -INFINITY);
      ga.sim_drop_thr = dt;
      ga.sim_cm = fp8_ks ? std::ldexp(1.0f, -11) : std::ldexp(1.0f, -17);
    }
    // open pairs are summed in order with one fused multiply-add per element
    fp32_guard(r.eps2, r.band_rel, p->d, 0, &ga.lo_thr, &ga.hi_thr);
    pg = &pb;
    rg = &rb;
  }
  if (pair_screen) {
    wait_inputs(st);
    if ((rc = make_shadow(static_cast<const float *>(x), p->ld, p->d, n, 0, s, &sh))) return rc;
    ga.x = sh.xb;
    ga.ld = sh.ldb;
    ga.nbe = sh.nbe;
    ga.err_max = sh.nmax + kErrMaxSlot;
    ga.screen_vec4 = (p->d % 4 == 0) && (p->ld % 4 == 0) && ((uintptr_t)x % 16 == 0);
    // the copy's FP32 distance: each term rounded at most 2 ceil(chunks / 4)
    // + 5 times for L1 (difference, its partial, two combining levels, two
    // shuffle levels), once for L-inf; c twice that plus 2^-22
    const double u = std::ldexp(1.0, -24);
    const int64_t chunks = sh.ldb / 8;
    const double cpp = p->metric == SNG_METRIC_L1 ? (double)(2 * ((chunks + 3) / 4) + 5) * u : u;
    const double c = 2.0 * cpp + std::ldexp(1.0, -22);
    const double eps = (double)p->eps;
    const double lo = eps * (1.0 - (double)r.band_rel - c);
    float lof = (float)lo;
    if ((double)lof > lo) lof = std::nextafter(lof, -INFINITY);
    ga.pm_lo = lof;
    ga.pm_hi = round_up_f(eps * (1.0 + (double)r.band_rel + c));
    // |v|_1 <= sqrt(d) |v|_2, |v|_inf <= |v|_2 for the copy's error bounds
    const double scale = p->metric == SNG_METRIC_L1 ? std::sqrt((double)p->d) : 1.0;
    ga.pm_escale = round_up_f(scale * (1.0 + std::ldexp(1.0, -10)));
  }
  const int grid = gather_grid(pg->dtype, rg->map, r.row_end - r.row_begin);
  bool tiled = false;
  if (!mma_kt && !fp8_ks && (p->flags & SNG_FLAG_TILED) &&
      (rc = run_tiled(pg, *rg, s, ga, gb, &tiled, screen ? &sh : nullptr)))
    return rc;
  gb->screened = screen || pair_screen;
  gb->map = rg->map;
  if (fp8_ks || mma_kt || pair_screen) {
    // the queue of open pairs of the tensor-core forms: room for 1 in 32
    // draws of the row range (at most 2^26 entries); past it, or without
    // the memory, the gather decides open pairs itself
    const int64_t draws = (r.row_end - r.row_begin) * (int64_t)r.m;
    int64_t cap = draws / 32 > 4096 ? draws / 32 : 4096;
    if (cap > (int64_t)1 << 26) cap = (int64_t)1 << 26;
    if ((rc = s.alloc((void **)&ga.openq_cnt, 8, "open-pair count"))) return rc;
    cudaMemsetAsync(ga.openq_cnt, 0, 8, st);
    if (s.alloc((void **)&ga.openq, (size_t)cap * sizeof(uint4), "open-pair queue") == SNG_OK) {
      ga.openq_cap = cap;
    } else {
      ga.openq = nullptr;
      ga.openq_cap = 0;
    }
    fp32_guard(r.eps2, r.band_rel, (p->d + 31) / 32, 5, &ga.q_lo_thr, &ga.q_hi_thr);
  }
  if (pair_screen) {
    // Manhattan / Chebyshev over the BF16 copy, four lanes per pair; the
    // open pairs from the FP32 points after it
    int kc = 0;
    if ((rc = launch_gather_pair16(p->metric, ga, &kc, st))) return rc;
    if ((rc = launch_pair_queue(p->metric, ga, st))) return rc;
    gb->map.vec = 8;
    gb->map.group = 4;
    gb->map.nch = kc;
    gb->map.unroll = 0;
  } else if (pair_metric) {
    // Manhattan / Chebyshev: four lanes per pair over the FP32 points
    wait_inputs(st);
    if ((rc = launch_gather_pair(p->metric, ga, st))) return rc;
  } else if (fp8_ks) {
    // the FP8 copy: 16 partners per MMA, fp8_ks k-tiles of 32 values
    gb->mma = true;
    gb->fp8 = true;
    gb->map.group = 16;
    gb->map.nch = fp8_ks;
    gb->map.unroll = p->map_unroll;
    if (!launch_gather_mma8(fp8_ks, p->map_unroll, ga, r.row_end - r.row_begin, st))
      return fail(SNG_EINVAL, "no FP8 tensor-core gather for d = %d with map_unroll = %d", p->d,
                  p->map_unroll);
    note_launch();
    if ((rc = launch_screen_queue(ga, st))) return rc;
  } else if (tc05) {
    // partner rows by TMA, 128 partners x 4 source rows per tcgen05 MMA
    gb->mma = true;
    gb->tc05 = true;
    gb->map.group = 128;
    gb->map.nch = 4;
    // map_unroll selects the ring's stages; stats report the count used
    if ((rc = launch_gather_tc05(ga, n, sh.ldb, p->map_unroll, &gb->map.unroll, st))) return rc;
    if ((rc = launch_screen_queue(ga, st))) return rc;
  } else if (mma_kt) {
    // the tensor-core form of the screen (direct gather only): 16 partners
    // per MMA, mma_kt k-tiles of 16 values per row
    gb->mma = true;
    gb->map.group = 16;
    gb->map.nch = mma_kt;
    // map_unroll selects the register budget (resident blocks per SM)
    gb->map.unroll = p->map_unroll;
    if (!launch_gather_mma(mma_kt, p->map_unroll, ga, r.row_end - r.row_begin, st))
      return fail(SNG_EINVAL, "no tensor-core gather for d = %d with map_unroll = %d", p->d,
                  p->map_unroll);
    note_launch();
    if ((rc = launch_screen_queue(ga, st))) return rc;
  } else if (tiled) {
    // done by the tiled form
  } else if (rg->map.passes <= 1) {
    wait_inputs(st);
    if (!launch_gather(pg->dtype, rg->map, ga, grid, st))
      return fail(SNG_EINVAL, "no compiled gather for vec=%d group=%d nch=%d unroll=%d",
                  rg->map.vec, rg->map.group, rg->map.nch, rg->map.unroll);
    note_launch();
  } else {
    // slices of the partner range, each small enough to stay in L2
    wait_inputs(st);
    const int64_t slice = (n + r.map.passes - 1) / r.map.passes;
    for (int64_t lo = 0; lo < n; lo += slice) {
      const int64_t hi = lo + slice < n ? lo + slice : n;
      if (!launch_gather_blocked(p->dtype, r.map, ga, grid, (int32_t)lo, (int32_t)hi, st))
        return fail(SNG_EINVAL,
                    "no compiled L2-blocked gather for vec=%d group=%d nch=%d unroll=%d",
                    r.map.vec, r.map.group, r.map.nch, r.map.unroll);
      note_launch();
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "gather launch");
  tm->mark(st, 1);
  launch_scan(gb->out_cnt, n, gb->tile_tmp, gb->row_ptr, gb->counters, st);
  tm->mark(st, 2);
  unsigned long long E = 0;
  if (p->flags & SNG_FLAG_NO_SYNC) {
    // no host read of E: the edge arrays get room for every draw and the
    // later kernels read E from row_ptr[n] on the device
    E = (unsigned long long)n * (unsigned long long)r.m;
    gb->num_edges_dev = gb->row_ptr + n;
  } else {
    e = cudaMemcpyAsync(&E, gb->counters + kCntEdges, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "edge count read-back");
  }
  gb->num_edges = (int64_t)E;
  if (gb->col_owned_by_caller) {
    e = cudaMalloc((void **)&gb->col, (size_t)(E ? E : 1) * 4);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "col");
    }
  } else if ((rc = s.alloc((void **)&gb->col, (size_t)E * 4, "col"))) {
    return rc;
  }
  tm->mark(st, 8);
  FillArgs fa;
  fa.n = n;
  fa.W = r.W;
  fa.sample_all = p->sample_mode == SNG_SAMPLE_ALL;
  fa.seed = p->seed;
  fa.fm = make_fastmod(n);
  fa.bitmask = gb->bitmask;
  fa.row_ptr = gb->row_ptr;
  fa.col = gb->col;
  fa.src = nullptr;
  const bool simple = p->degree_mode == SNG_DEG_SIMPLE;
  if (gb->want_src || simple) {
    if ((rc = s.alloc((void **)&gb->src, (size_t)E * 4, "edge sources"))) return rc;
    fa.src = gb->src;
  }
  launch_fill(fa, device_sms(), st);
  tm->mark(st, 3);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fill launch");
  // the gather left out-degrees; the simple-graph degree replaces them
  if (simple && (rc = simple_degrees(n, gb->src, gb->col, gb->num_edges, gb->deg, gb->counters, s)))
    return rc;
  return SNG_OK;
}

sng_status read_stats(const unsigned long long *counters, const Resolved &r, sng_stats *stats,
                      cudaStream_t st, const Timer *tm) {
  unsigned long long c[kCntSlots];
  cudaError_t e = cudaMemcpyAsync(c, counters, sizeof(c), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stats read-back");
  const uint32_t status = (uint32_t)c[kCntStatus];
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->queries = r.n * r.m;
    stats->kept_edges = (int64_t)c[kCntEdges];
    stats->band_pairs = (int64_t)c[kCntBandPairs];
    stats->band_points = (int64_t)c[kCntBandPoints];
    stats->cores = (int64_t)c[kCntCores];
    stats->clusters = (int64_t)c[kCntClusters];
    stats->noise = (int64_t)c[kCntNoise];
    stats->recheck_pairs = (int64_t)c[kCntRecheck];
    stats->screen_pairs = (int64_t)c[kCntScreen];
    if (tm) tm->fill(stats->ms);
    stats->map_vec = r.map.vec;
    stats->map_group = r.map.group;
    stats->map_nch = r.map.nch;
    stats->map_unroll = r.map.unroll;
  }
  if (status & (kErrUnionLimit | kErrFindLimit | kErrBatchLimit | kErrDeviceWait))
    return fail(SNG_ETIMEOUT, "a bounded device loop gave up (status 0x%x)", status);
  if (status & kErrIndex) return fail(SNG_EINTERNAL, "device index check failed (0x%x)", status);
  return SNG_OK;
}

void note_mapping(const GraphBufs &gb, sng_stats *stats) {
  if (!stats) return;
  stats->map_tiles = gb.tiles;
  stats->map_tex = gb.tex_chunks;
  stats->map_screen = gb.screened ? (gb.fp8 ? 4 : gb.tc05 ? 3 : gb.mma ? 2 : 1) : 0;
  if (gb.screened) {
    stats->map_vec = gb.map.vec;
    stats->map_group = gb.map.group;
    stats->map_nch = gb.map.nch;
    stats->map_unroll = gb.map.unroll;
  }
}

// ----------------------------------------------------------------- timer

Timer::Timer(bool on) : on_(on) {
  if (!on_) return;
  for (int k = 0; k < kMarks; ++k) cudaEventCreate(&ev_[k]);
}
Timer::~Timer() {
  if (!on_) return;
  for (int k = 0; k < kMarks; ++k) cudaEventDestroy(ev_[k]);
}
void Timer::mark(cudaStream_t st, int k) {
  if (on_ && k < kMarks) {
    cudaEventRecord(ev_[k], st);
    used_[k] = true;
  }
}
void Timer::fill(float *ms) const {
  if (!on_) return;
  // ms[0] gather (0->1), [1] scan (1->2), [2] fill (2->3 after the host
  // read-back: 3 is recorded after the fill launch), [3] core+union (4->5),
  // [4] labels (5->6), [5] finalize (6->7), [6] total (0->7)
  // [7] surrogate gate (9 -> 0), when the gated form recorded mark 9
  const int pairs[8][2] = {{0, 1}, {1, 2}, {8, 3}, {3, 5}, {5, 6}, {6, 7}, {0, 7}, {9, 0}};
  for (int q = 0; q < 8; ++q) {
    const int a = pairs[q][0], b = pairs[q][1];
    float v = 0.f;
    if (used_[a] && used_[b]) cudaEventElapsedTime(&v, ev_[a], ev_[b]);
    ms[q] = v;
  }
}

}  // namespace sng

using namespace sng;

extern "C" {

int64_t sng_launch_count(void) { return g_launches.load(); }

const char *sng_last_error(void) { return g_last_error.c_str(); }

const char *sng_strerror(sng_status s) {
  switch (s) {
    case SNG_OK: return "ok";
    case SNG_EINVAL: return "invalid argument";
    case SNG_ENOMEM: return "out of device memory";
    case SNG_ECUDA: return "CUDA runtime error";
    case SNG_ETIMEOUT: return "bounded device loop gave up";
    case SNG_EINTERNAL: return "internal consistency check failed";
    default: return "unknown status";
  }
}

sng_status sng_gather_mapping(const void *x, const sng_params *params, int32_t *mapping) {
  if (!mapping) return fail(SNG_EINVAL, "mapping is NULL");
  Resolved r;
  sng_status rc = validate(x, params, &r);
  if (rc) return rc;
  mapping[0] = r.map.vec;
  mapping[1] = r.map.group;
  mapping[2] = r.map.nch;
  mapping[3] = r.map.unroll;
  mapping[4] = r.map.block;
  mapping[5] = r.map.passes;
  mapping[6] = r.map.passes > 1 ? gather_blocked_is_compiled(params->dtype, r.map)
                                : gather_is_compiled(params->dtype, r.map);
  return SNG_OK;
}

sng_status sng_cluster_edges(int64_t n, const int32_t *src, const int32_t *col, int64_t num_edges,
                             const int32_t *deg, const sng_params *params, int32_t *labels,
                             uint8_t *core, sng_stats *stats, void *stream) {
  NvtxRange nvtx_range("sng_cluster_edges");
  if (!params || !labels) return fail(SNG_EINVAL, "NULL argument");
  const bool simple = params->degree_mode == SNG_DEG_SIMPLE;
  if (!deg && !simple) return fail(SNG_EINVAL, "deg is NULL");
  if (n < 1 || n > 0x7fffffffLL) return fail(SNG_EINVAL, "n must be in [1, 2^31-1]");
  if (num_edges < 0) return fail(SNG_EINVAL, "num_edges must be >= 0");
  if (num_edges > 0 && (!src || !col)) return fail(SNG_EINVAL, "src / col is NULL");
  if (params->min_pts < 1) return fail(SNG_EINVAL, "min_pts must be >= 1");
  device_sms();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s(st);
  Resolved r;
  r.n = n;
  r.m = 0;
  uint8_t *core_buf = core;
  int32_t *parent = nullptr;
  unsigned long long *counters = nullptr;
  sng_status rc;
  if (!core_buf && (rc = s.alloc((void **)&core_buf, (size_t)n, "core"))) return rc;
  if ((rc = s.alloc((void **)&parent, (size_t)n * 4, "parent"))) return rc;
  if ((rc = s.alloc((void **)&counters, kCntSlots * 8, "counters"))) return rc;
  cudaMemsetAsync(counters, 0, kCntSlots * 8, st);
  cudaMemcpyAsync(counters + kCntEdges, &num_edges, 8, cudaMemcpyHostToDevice, st);
  if (simple) {
    // degrees of the simple graph come from the edge list itself (the
    // caller's deg, if any, is not read)
    int32_t *sdeg = nullptr;
    if ((rc = s.alloc((void **)&sdeg, (size_t)n * 4, "degrees"))) return rc;
    if ((rc = simple_degrees(n, src, col, num_edges, sdeg, counters, s))) return rc;
    deg = sdeg;
  }
  const int sms = device_sms();
  CoreArgs ca{n, params->min_pts, deg, nullptr, core_buf, parent, labels};
  launch_core_init(ca, sms, st);
  UnionArgs ua{n, nullptr, col, src, num_edges, core_buf, parent, labels, counters, loop_limit()};
  launch_union(ua, sms, st);
  launch_label(ua, sms, st);
  FinalizeArgs fa{n, core_buf, nullptr, labels, counters, parent, loop_limit()};
  launch_finalize(fa, sms, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "cluster_edges launches");
  if (stats) {
    rc = read_stats(counters, r, stats, st, nullptr);
  } else {
    // still surface device-side status (bounded loops, out-of-range edges)
    rc = read_stats(counters, r, nullptr, st, nullptr);
  }
  s.release();
  return rc;
}

sng_status sng_cluster(const void *x, const sng_params *params, int32_t *labels, uint8_t *core,
                       sng_stats *stats, void *stream) {
  NvtxRange nvtx_range("sng_cluster");
  Resolved r;
  sng_status rc = validate(x, params, &r);
  if (rc) return rc;
  if (r.row_begin != 0 || r.row_end != r.n)
    return fail(SNG_EINVAL, "a source-row range is for sng_build_graph only");
  if (!labels) return fail(SNG_EINVAL, "labels is NULL");
  if ((params->flags & SNG_FLAG_NO_SYNC) && stats)
    return fail(SNG_EINVAL, "stats are read on the host: pass NULL with SNG_FLAG_NO_SYNC "
                            "(counters_out receives the counters)");
  device_sms();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s(st);
  Timer tm((params->flags & SNG_FLAG_TIMING) != 0);
  GraphBufs gb;
  gb.want_src = true;
  if ((rc = run_graph(x, params, r, s, &gb, nullptr, &tm))) return rc;
  uint8_t *core_buf = core;
  int32_t *parent = nullptr;
  if (!core_buf && (rc = s.alloc((void **)&core_buf, (size_t)r.n, "core"))) return rc;
  if ((rc = s.alloc((void **)&parent, (size_t)r.n * 4, "parent"))) return rc;
  const int sms = device_sms();
  CoreArgs ca{r.n, params->min_pts, gb.deg, nullptr, core_buf, parent, labels};
  launch_core_init(ca, sms, st);
  tm.mark(st, 4);
  UnionArgs ua{r.n,      gb.row_ptr, gb.col,      gb.src,      gb.num_edges,
               core_buf, parent,     labels,      gb.counters, loop_limit(),
               gb.num_edges_dev};
  launch_union(ua, sms, st);
  tm.mark(st, 5);
  launch_label(ua, sms, st);
  tm.mark(st, 6);
  FinalizeArgs fa{r.n, core_buf, gb.band_flag, labels, gb.counters, parent, loop_limit()};
  launch_finalize(fa, sms, st);
  tm.mark(st, 7);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "cluster launches");
  if (params->flags & SNG_FLAG_NO_SYNC) {
    // counters (and device status bits) to the caller's device memory
    if (params->counters_out) {
      e = cudaMemcpyAsync(params->counters_out, gb.counters, kCntStatus * 8 + 8,
                          cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "counters copy");
    }
    s.release();
    return SNG_OK;
  }
  rc = read_stats(gb.counters, r, stats, st, &tm);
  note_mapping(gb, stats);
  s.release();
  return rc;
}

sng_status sng_cluster_host(const void *x_host, const sng_params *params, int32_t *labels_host,
                            uint8_t *core_host, sng_stats *stats, void *stream) {
  NvtxRange nvtx_range("sng_cluster_host");
  if (!params || !x_host || !labels_host) return fail(SNG_EINVAL, "NULL argument");
  if (params->n < 2 || params->n > 0x7fffffffLL || params->ld < params->d || params->d < 1)
    return fail(SNG_EINVAL, "bad n / d / ld");
  if (params->dtype != SNG_F32 && params->dtype != SNG_BF16)
    return fail(SNG_EINVAL, "unknown dtype");
  if (params->dtype == SNG_BF16 && !params->x_f32_master)
    return fail(SNG_EINVAL, "BF16 form needs x_f32_master");
  if (params->flags & SNG_FLAG_NO_SYNC)
    return fail(SNG_EINVAL, "the host-buffer call synchronises (no SNG_FLAG_NO_SYNC)");
  device_sms();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = params->n;
  const size_t esize = params->dtype == SNG_F32 ? 4 : 2;
  const size_t xbytes = (size_t)n * (size_t)params->ld * esize;
  const size_t mbytes = params->dtype == SNG_BF16 ? (size_t)n * (size_t)params->ld * 4 : 0;
  Scratch s(st);
  void *xd = nullptr;
  float *md = nullptr;
  int32_t *ld = nullptr;
  uint8_t *cd = nullptr;
  sng_status rc;
  if ((rc = s.alloc(&xd, xbytes, "device points")) ||
      (mbytes && (rc = s.alloc((void **)&md, mbytes, "device FP32 master"))) ||
      (rc = s.alloc((void **)&ld, (size_t)n * 4, "device labels")) ||
      (core_host && (rc = s.alloc((void **)&cd, (size_t)n, "device core mask"))))
    return rc;
  // host -> device in up to four pieces on streams forked from `st`, so
  // several copy engines can take part; the pieces join `st` before use
  struct Piece {
    char *dst;
    const char *src;
    size_t bytes;
  };
  std::vector<Piece> pieces;
  auto split = [&](void *dst, const void *src, size_t bytes) {
    const size_t k = bytes >= ((size_t)64 << 20) ? 4 : 1;
    const size_t step = ((bytes + k - 1) / k + 255) / 256 * 256;
    for (size_t o = 0; o < bytes; o += step)
      pieces.push_back({static_cast<char *>(dst) + o, static_cast<const char *>(src) + o,
                        bytes - o < step ? bytes - o : step});
  };
  split(xd, x_host, xbytes);
  if (mbytes) split(md, params->x_f32_master, mbytes);
  cudaEvent_t fork = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> done;
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(fork, st);
  for (size_t k = 0; e == cudaSuccess && k < pieces.size(); ++k) {
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    side.push_back(cs);
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) break;
    done.push_back(ev);
    if ((e = cudaStreamWaitEvent(cs, fork, 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(pieces[k].dst, pieces[k].src, pieces[k].bytes,
                             cudaMemcpyHostToDevice, cs)) != cudaSuccess)
      break;
    e = cudaEventRecord(ev, cs);
  }
  for (cudaStream_t cs : side) cudaStreamDestroy(cs);   // released once drained
  if (fork) cudaEventDestroy(fork);
  // the stream joins the copies where the clustering first reads the
  // points (after the tiled form's partition); whatever the call did not
  // consume (an error, an early return) is joined here, so no copy from the
  // caller's buffer outlives the call
  auto join_copies = [&]() {
    g_inputs_pending.clear();
    for (cudaEvent_t ev : done) {
      cudaStreamWaitEvent(st, ev, 0);
      cudaEventDestroy(ev);
    }
    done.clear();
  };
  if (e != cudaSuccess) {
    join_copies();
    cudaStreamSynchronize(st);
    return cuda_fail(e, "host to device copy");
  }
  sng_params pd = *params;
  pd.x_f32_master = md;
  g_inputs_pending = done;
  rc = sng_cluster(xd, &pd, ld, cd, stats, stream);
  join_copies();
  if (rc) {
    cudaStreamSynchronize(st);
    return rc;
  }
  e = cudaMemcpyAsync(labels_host, ld, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && core_host)
    e = cudaMemcpyAsync(core_host, cd, (size_t)n, cudaMemcpyDeviceToHost, st);
  s.release();
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "device to host copy");
}

sng_status sng_build_graph(const void *x, const sng_params *params, sng_graph *out,
                           sng_stats *stats, void *stream) {
  NvtxRange nvtx_range("sng_build_graph");
  Resolved r;
  sng_status rc = validate(x, params, &r);
  if (rc) return rc;
  if (!out) return fail(SNG_EINVAL, "out is NULL");
  if (params->flags & SNG_FLAG_NO_SYNC)
    return fail(SNG_EINVAL, "SNG_FLAG_NO_SYNC is for sng_cluster only");
  std::memset(out, 0, sizeof(*out));
  device_sms();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s(st);
  Timer tm((params->flags & SNG_FLAG_TIMING) != 0);
  GraphBufs gb;
  gb.col_owned_by_caller = true;
  rc = run_graph(x, params, r, s, &gb, nullptr, &tm);
  if (rc) {
    if (gb.col) cudaFree(gb.col);
    return rc;
  }
  // library-owned outputs (plain allocations, released by sng_graph_free)
  int64_t *row_ptr = nullptr;
  int32_t *deg = nullptr;
  uint8_t *core = nullptr;
  int32_t *parent = nullptr, *labels = nullptr;
  cudaError_t e = cudaMalloc((void **)&row_ptr, (size_t)(r.n + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc((void **)&deg, (size_t)r.n * 4);
  if (e == cudaSuccess) e = cudaMalloc((void **)&core, (size_t)r.n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(row_ptr);
    cudaFree(deg);
    cudaFree(core);
    cudaFree(gb.col);
    return cuda_fail(e, "graph outputs");
  }
  auto free_all = [&]() {
    cudaFree(row_ptr);
    cudaFree(deg);
    cudaFree(core);
    cudaFree(gb.col);
  };
  if ((rc = s.alloc((void **)&parent, (size_t)r.n * 4, "parent")) ||
      (rc = s.alloc((void **)&labels, (size_t)r.n * 4, "labels"))) {
    cudaStreamSynchronize(st);
    free_all();
    return rc;
  }
  cudaMemcpyAsync(row_ptr, gb.row_ptr, (size_t)(r.n + 1) * 8, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(deg, gb.deg, (size_t)r.n * 4, cudaMemcpyDeviceToDevice, st);
  CoreArgs ca{r.n, params->min_pts, gb.deg, nullptr, core, parent, labels};
  launch_core_init(ca, device_sms(), st);
  rc = read_stats(gb.counters, r, stats, st, &tm);
  note_mapping(gb, stats);
  if (rc) {
    free_all();
    return rc;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    free_all();
    return cuda_fail(e, "build_graph");
  }
  out->n = r.n;
  out->m = r.m;
  out->num_edges = gb.num_edges;
  out->row_ptr = row_ptr;
  out->col = gb.col;
  out->deg = deg;
  out->core = core;
  s.release();
  cudaStreamSynchronize(st);
  return SNG_OK;
}

void sng_graph_free(sng_graph *g) {
  if (!g) return;
  cudaFree(g->row_ptr);
  cudaFree(g->col);
  cudaFree(g->deg);
  cudaFree(g->core);
  std::memset(g, 0, sizeof(*g));
}

}  // extern "C"
