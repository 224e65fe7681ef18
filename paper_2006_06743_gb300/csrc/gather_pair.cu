// gather_pair.cu -- step 2 of Algorithm 1 with the Manhattan (L1) or
// Chebyshev (L-inf) distance as the neighbourhood test.  The method needs
// only similarity queries (Section 1); these two are pair kernels that are
// neither the Euclidean ball nor an inner product, so no norm identity or
// tensor-core form applies.
//
// One warp per source row, stages of 32 draws hashed one per lane; four
// lanes per pair (below) form the distance in FP32 -- the sum of |a_k - b_k|
// or their maximum.  Outside the guard band around eps (validate, api.cu)
// the FP32 value decides; inside it the FP64 value in the oracle's order does
// (recheck_pair_metric, which also counts the reported band).  Keep bits by
// ballot, degrees by atomics, as in the other gathers.  The group's order of
// the additions (four partials per lane, their sum, then two shuffle levels)
// keeps every term's roundings within the (d + 1) u of the guard band.
//
// With a screen flag the same test runs first over a BF16 copy of the
// points (gather_pair16_kernel, below): half the bytes per partner row,
// each decision certified by the rows' copy error bounds, and the pairs it
// cannot certify decided from the FP32 points afterwards (pair_queue_kernel)
// exactly as above.
#include "api_common.cuh"
#include "gather.cuh"
#include "gather_pair.cuh"
#include "screen_queue.cuh"

namespace sng {

// The FP64 distance in the oracle's order (differences, absolute values and
// sums left to right; a NaN difference makes the distance NaN), the band
// count and the decision dist <= eps.
template <int METRIC>
static __device__ __noinline__ bool recheck_pair_metric(const GatherArgs &a, int32_t i,
                                                        int32_t p) {
  const float *xa = a.xm + (int64_t)i * a.ldm, *xb = a.xm + (int64_t)p * a.ldm;
  double s = 0.0;
  for (int k = 0; k < a.d; ++k) {
    const double t = fabs(__dsub_rn((double)xa[k], (double)xb[k]));
    if (METRIC == SNG_METRIC_L1) {
      s = __dadd_rn(s, t);
    } else {
      if (t != t) {
        s = t;
        break;
      }
      if (t > s) s = t;
    }
  }
  atomicAdd(a.counters + kCntRecheck, 1ull);
  if (fabs(__dsub_rn(s, a.tau64)) <= a.band) {
    atomicAdd(a.counters + kCntBandPairs, 1ull);
    a.band_flag[i] = 1;
    a.band_flag[p] = 1;
  }
  return s <= a.tau64;
}

// Partial distance: the sum of |u - v| or their maximum.  The terms are
// non-negative (a NaN's sign cleared by the absolute value too), and for
// such floats the order of the bit patterns as unsigned integers is the
// order of the values with NaN above +inf -- so one integer maximum takes
// the largest term and keeps a NaN (fmaxf would drop it).
template <int METRIC>
__device__ __forceinline__ float pair_combine(float acc, float t) {
  if (METRIC == SNG_METRIC_L1) return acc + t;
  return __uint_as_float(max(__float_as_uint(acc), __float_as_uint(t)));
}

// Group layout (VEC4 rows): four lanes per pair, lane q of a group reading
// the 16-byte chunks q, q + 4, q + 8, ... of the partner row (so the group's
// loads cover consecutive bytes) against the same chunks of the source row,
// kept in registers for rows of up to 64 values; the four partials combine
// in two shuffle levels.  A warp tests 8 pairs per step, 4 steps per stage
// of 32 draws; each distance is handed back to the lane that drew it, which
// decides it, so the stage's keep bits come from one ballot in draw order.
// Rows whose length is not a multiple of 4 (or whose start is not 16-byte
// aligned) take one lane per pair with scalar loads.  FULL: rows of exactly
// 64 values (no bounds tests).
template <int METRIC, bool VEC4, bool FULL>
__global__ void __launch_bounds__(256) gather_pair_kernel(GatherArgs a) {
  constexpr int kSrcChunks = 4;   // source chunks a lane keeps (rows of <= 64 values)
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int nc = a.d >> 2;        // 16-byte chunks per row (VEC4)
  for (int64_t row = a.row_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
       row < a.row_end; row += warps_total) {
    const int32_t i = (int32_t)row;
    const int32_t mi = a.m_row ? a.m_row[i] : a.m;
    const int32_t wi = a.w_row ? a.w_row[i] : 1;
    const uint64_t key = row_key(a.seed, i);
    const float *xa = a.xm + (int64_t)i * a.ldm;
    float4 src[kSrcChunks];
    if (VEC4) {
#pragma unroll
      for (int t = 0; t < kSrcChunks; ++t) {
        const int c = q + 4 * t;
        src[t] = FULL || c < nc ? __ldg(reinterpret_cast<const float4 *>(xa) + c)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    int cnt = 0;
    for (int jb = 0; jb < mi; jb += 32) {
      const int j = jb + lane;
      const bool live = j < mi;
      // draws past the row's count read row 0 and decide nothing
      const int32_t p =
          live ? (a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, a.fm)) : 0;
      float mine = 0.f;   // the distance of this lane's own draw
      if (VEC4) {
#pragma unroll
        for (int step = 0; step < 4; ++step) {
          // group g tests draw 8 step + g
          const int32_t pg = __shfl_sync(kFullMask, p, 8 * step + g);
          const float4 *vb = reinterpret_cast<const float4 *>(a.xm + (int64_t)pg * a.ldm);
          // four independent partials (one per vector component), combined
          // at the end: each term still sees at most d / 16 + 5 roundings
          float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
#pragma unroll
          for (int t = 0; t < kSrcChunks; ++t) {
            const int c = q + 4 * t;
            if (FULL || c < nc) {
              const float4 v = __ldg(vb + c);
              ax = pair_combine<METRIC>(ax, fabsf(src[t].x - v.x));
              ay = pair_combine<METRIC>(ay, fabsf(src[t].y - v.y));
              az = pair_combine<METRIC>(az, fabsf(src[t].z - v.z));
              aw = pair_combine<METRIC>(aw, fabsf(src[t].w - v.w));
            }
          }
          for (int c = q + 4 * kSrcChunks; !FULL && c < nc; c += 4) {
            const float4 u = __ldg(reinterpret_cast<const float4 *>(xa) + c);
            const float4 v = __ldg(vb + c);
            ax = pair_combine<METRIC>(ax, fabsf(u.x - v.x));
            ay = pair_combine<METRIC>(ay, fabsf(u.y - v.y));
            az = pair_combine<METRIC>(az, fabsf(u.z - v.z));
            aw = pair_combine<METRIC>(aw, fabsf(u.w - v.w));
          }
          float acc = pair_combine<METRIC>(pair_combine<METRIC>(ax, ay),
                                           pair_combine<METRIC>(az, aw));
          acc = pair_combine<METRIC>(acc, __shfl_xor_sync(kFullMask, acc, 1));
          acc = pair_combine<METRIC>(acc, __shfl_xor_sync(kFullMask, acc, 2));
          const float got = __shfl_sync(kFullMask, acc, 4 * (lane & 7));
          if ((lane >> 3) == step) mine = got;
        }
      } else {
        const float *xb = a.xm + (int64_t)p * a.ldm;
        for (int k = 0; k < a.d; ++k)
          mine = pair_combine<METRIC>(mine, fabsf(__ldg(xa + k) - __ldg(xb + k)));
      }
      bool keep = false;
      if (live) {
        if (mine < a.lo_thr) {
          keep = true;
        } else if (!(mine > a.hi_thr)) {
          keep = recheck_pair_metric<METRIC>(a, i, p);   // the guard band or NaN
        }
        if (keep && a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) atomicAdd(a.deg + p, wi);
      }
      const uint32_t word = __ballot_sync(kFullMask, keep);
      if (lane == 0) __stcs(a.bitmask + (int64_t)i * a.W + (jb >> 5), word);
      cnt += __popc(word);
    }
    // words past this row's draws (per-row draw counts) are zero
    for (int w = ((mi + 31) >> 5) + lane; w < a.W; w += 32)
      __stcs(a.bitmask + (int64_t)i * a.W + w, 0u);
    if (lane == 0) {
      if (a.out_cnt) a.out_cnt[i] = cnt;
      if (a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) {
        if (cnt) atomicAdd(a.deg + i, cnt * wi);
      } else {
        a.deg[i] = cnt * wi;
      }
    }
  }
}

template <int METRIC, bool VEC4>
static void launch_pm(const GatherArgs &a, int64_t rows, cudaStream_t st) {
  const int64_t need = (rows + 7) / 8;
  int64_t grid = (int64_t)device_sms() * 8;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  if constexpr (VEC4) {
    if (a.d == 64) {
      gather_pair_kernel<METRIC, true, true><<<(int)grid, 256, 0, st>>>(a);
      return;
    }
  }
  gather_pair_kernel<METRIC, VEC4, false><<<(int)grid, 256, 0, st>>>(a);
}

sng_status launch_gather_pair(int metric, const GatherArgs &a, cudaStream_t st) {
  const int64_t rows = a.row_end - a.row_begin;
  const bool vec4 = a.d % 4 == 0 && a.ldm % 4 == 0 &&
                    reinterpret_cast<uintptr_t>(a.xm) % 16 == 0;
  if (metric == SNG_METRIC_L1) {
    vec4 ? launch_pm<SNG_METRIC_L1, true>(a, rows, st) : launch_pm<SNG_METRIC_L1, false>(a, rows, st);
  } else if (metric == SNG_METRIC_LINF) {
    vec4 ? launch_pm<SNG_METRIC_LINF, true>(a, rows, st)
         : launch_pm<SNG_METRIC_LINF, false>(a, rows, st);
  } else {
    return fail(SNG_EINTERNAL, "no pair-kernel gather for metric %d", metric);
  }
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "pair-kernel gather launch");
}


// ------------------------------------------------ the BF16 screen (SCREEN16)
//
// The partner rows come from the BF16 copy of the points (screen.cu): half
// the bytes of the FP32 rows, and a point set that fits L2 twice as easily.
// Rounding the points moves a pair's distance by at most eta = e_a + e_b,
// e_i >= |x_i - x_i'| in the metric's own norm.  The copy carries a bound of
// the Euclidean norm of each row's rounding error; |v|_1 <= sqrt(d) |v|_2
// and |v|_inf <= |v|_2 turn it into the L1 and L-inf bounds (pm_escale:
// sqrt(d) or 1, times 1 + 2^-10, rounded up).  The FP32 value v over the
// copy -- each difference of two BF16 values rounded once, two terms per
// 16-byte chunk into each of four partials, their pairwise combination and
// two shuffle levels -- is within c'' relative of the copy's exact distance
// (c'' = (2 ceil(chunks / 4) + 5) u for L1, u for L-inf: the maximum itself
// is exact).  pm_lo / pm_hi = eps (1 -+ (band_rel + c)) with c = 2 c'' +
// 2^-22, rounded outwards; a pair with v <= pm_lo - eta is then nearer than
// eps (1 - band_rel) and one with v > pm_hi + eta farther than eps (1 +
// band_rel): the FP64 value in the oracle's order decides both the same way
// and neither lies in the reported band.  The row's thresholds against the
// largest partner bound (err_max) decide almost every pair without reading
// the partner's own bound; the rest read it; a pair still open is queued and
// decided from the FP32 points afterwards (pair_queue_kernel), or, past the
// queue's capacity, here (pair_fp32_decide).  A NaN anywhere leaves a pair
// open.

// The pair's keep / drop thresholds for copy error bounds ea, eb.
__device__ __forceinline__ void pm_thresholds(const GatherArgs &a, float ea, float eb,
                                              float &keep_thr, float &drop_thr) {
  const float eta = __fmul_ru(__fadd_ru(ea, eb), a.pm_escale);
  keep_thr = __fsub_rd(a.pm_lo, eta);
  drop_thr = __fadd_ru(a.pm_hi, eta);
}

// Eight BF16 values (one 16-byte chunk) as FP32: value 2k + h is the high
// (h = 1) or low half of word k.
__device__ __forceinline__ void bf16x8_to_f32(const uint4 w, float (&f)[8]) {
  const uint32_t v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    f[2 * k] = __uint_as_float(v[k] << 16);
    f[2 * k + 1] = __uint_as_float(v[k] & 0xffff0000u);
  }
}

// One chunk's eight terms into the four partials: value e goes to e % 4.
template <int METRIC>
__device__ __forceinline__ void pm_chunk(float (&acc)[4], const float (&s)[8], const uint4 w) {
  float b[8];
  bf16x8_to_f32(w, b);
#pragma unroll
  for (int e = 0; e < 8; ++e) acc[e & 3] = pair_combine<METRIC>(acc[e & 3], fabsf(s[e] - b[e]));
}

// An open pair decided in the gather (no room left in the queue): the FP32
// distance in order, its guard band, the FP64 value inside it.
template <int METRIC>
static __device__ __noinline__ bool pair_fp32_decide(const GatherArgs &a, int32_t i, int32_t p) {
  const float *xa = a.xm + (int64_t)i * a.ldm, *xb = a.xm + (int64_t)p * a.ldm;
  float v = 0.f;
  for (int k = 0; k < a.d; ++k) v = pair_combine<METRIC>(v, fabsf(__ldg(xa + k) - __ldg(xb + k)));
  if (v < a.lo_thr) return true;
  if (v > a.hi_thr) return false;
  return recheck_pair_metric<METRIC>(a, i, p);
}

// Group layout as gather_pair_kernel's over 16-byte chunks of 8 BF16
// values: lane q of a group takes chunks q, q + 4, ...; the source row's
// first KC chunks of each lane are held in registers (as FP32 for KC <= 2).
// All 32 partner rows of a stage are fetched before any is tested -- four
// steps of eight rows, KC chunks per lane each -- and the next stage's
// partners are hashed while they are on their way.  FULL: the row has
// exactly 4 KC chunks (no bounds tests).
template <int METRIC, int KC, bool FULL>
__global__ void __launch_bounds__(256, KC <= 2 ? 3 : 2) gather_pair16_kernel(GatherArgs a) {
  constexpr bool kSrcF32 = KC <= 2;
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int nc = (int)(a.ld >> 3);   // 16-byte chunks of a copied row
  const uint16_t *X = static_cast<const uint16_t *>(a.x);
  __shared__ unsigned int s_open;   // open pairs decided here (no room in the queue)
  if (threadIdx.x == 0) s_open = 0;
  __syncthreads();
  const float err_pmax = *a.err_max;   // largest copy error bound of any row
  for (int64_t row = a.row_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
       row < a.row_end; row += warps_total) {
    const int32_t i = (int32_t)row;
    const int32_t mi = a.m_row ? a.m_row[i] : a.m;
    const int32_t wi = a.w_row ? a.w_row[i] : 1;
    const uint64_t key = row_key(a.seed, i);
    const uint4 *xa = reinterpret_cast<const uint4 *>(X + (int64_t)i * a.ld);
    uint4 srcw[KC];
    float srcf[kSrcF32 ? KC : 1][8];
#pragma unroll
    for (int t = 0; t < KC; ++t) {
      const int c = q + 4 * t;
      srcw[t] = c < nc ? __ldg(xa + c) : make_uint4(0u, 0u, 0u, 0u);
      if constexpr (kSrcF32) bf16x8_to_f32(srcw[t], srcf[t]);
    }
    const float ea = __ldg(a.nbe + i).y;
    float keep_row, drop_row;
    pm_thresholds(a, ea, err_pmax, keep_row, drop_row);
    int cnt = 0;
    // draws past the row's count read row 0 and decide nothing
    auto draw = [&](int j) -> int32_t {
      return j < mi ? (a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, a.fm)) : 0;
    };
    int32_t p = draw(lane);
    for (int jb = 0; jb < mi; jb += 32) {
      const int j = jb + lane;
      const bool live = j < mi;
      // the stage's partner rows: step s, group g holds draw 8 s + g
      uint4 buf[4][KC];
#pragma unroll
      for (int step = 0; step < 4; ++step) {
        const int32_t pg = __shfl_sync(kFullMask, p, 8 * step + g);
        const uint4 *vb = reinterpret_cast<const uint4 *>(X + (int64_t)pg * a.ld);
#pragma unroll
        for (int t = 0; t < KC; ++t) {
          const int c = q + 4 * t;
          buf[step][t] = FULL || c < nc ? __ldg(vb + c) : make_uint4(0u, 0u, 0u, 0u);
        }
      }
      // the next stage's partners, hashed while these rows are on their way
      const int32_t p_next = draw(jb + 32 + lane);
      float mine = 0.f;   // the copy's distance of this lane's own draw
#pragma unroll
      for (int step = 0; step < 4; ++step) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < KC; ++t) {
          if (FULL || q + 4 * t < nc) {
            if constexpr (kSrcF32) {
              pm_chunk<METRIC>(acc, srcf[t], buf[step][t]);
            } else {
              float s8[8];
              bf16x8_to_f32(srcw[t], s8);
              pm_chunk<METRIC>(acc, s8, buf[step][t]);
            }
          }
        }
        if (!FULL && nc > 4 * KC) {
          // rows past 32 KC values: the rest of both rows chunk by chunk
          const int32_t pg = __shfl_sync(kFullMask, p, 8 * step + g);
          const uint4 *vb = reinterpret_cast<const uint4 *>(X + (int64_t)pg * a.ld);
          for (int c = q + 4 * KC; c < nc; c += 4) {
            float s8[8];
            bf16x8_to_f32(__ldg(xa + c), s8);
            pm_chunk<METRIC>(acc, s8, __ldg(vb + c));
          }
        }
        float v = pair_combine<METRIC>(pair_combine<METRIC>(acc[0], acc[1]),
                                       pair_combine<METRIC>(acc[2], acc[3]));
        v = pair_combine<METRIC>(v, __shfl_xor_sync(kFullMask, v, 1));
        v = pair_combine<METRIC>(v, __shfl_xor_sync(kFullMask, v, 2));
        const float got = __shfl_sync(kFullMask, v, 4 * (lane & 7));
        if ((lane >> 3) == step) mine = got;
      }
      bool keep = false, open = false;
      if (live) {
        if (mine <= keep_row) {
          keep = true;
        } else if (!(mine > drop_row)) {
          float keep_thr, drop_thr;
          pm_thresholds(a, ea, __ldg(a.nbe + p).y, keep_thr, drop_thr);
          keep = mine <= keep_thr;
          open = !keep && !(mine > drop_thr);
        }
      }
      const uint32_t om = __ballot_sync(kFullMask, open);
      if (om) {
        // open pairs to the queue (one atomic per warp); past its capacity
        // decided here
        unsigned long long base = 0;
        if (lane == 0 && a.openq_cnt)
          base = atomicAdd(a.openq_cnt, (unsigned long long)__popc(om));
        base = __shfl_sync(kFullMask, base, 0);
        if (open) {
          const unsigned long long slot = base + __popc(om & ((1u << lane) - 1u));
          if ((long long)slot < a.openq_cap) {
            a.openq[slot] = make_uint4((uint32_t)i, (uint32_t)p, (uint32_t)j, (uint32_t)wi);
          } else {
            keep = pair_fp32_decide<METRIC>(a, i, p);
            atomicAdd(&s_open, 1u);
          }
        }
      }
      if (keep && a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) atomicAdd(a.deg + p, wi);
      const uint32_t word = __ballot_sync(kFullMask, keep);
      if (lane == 0) __stcs(a.bitmask + (int64_t)i * a.W + (jb >> 5), word);
      cnt += __popc(word);
      p = p_next;
    }
    // words past this row's draws (per-row draw counts) are zero
    for (int w = ((mi + 31) >> 5) + lane; w < a.W; w += 32)
      __stcs(a.bitmask + (int64_t)i * a.W + w, 0u);
    if (lane == 0) {
      if (a.out_cnt) a.out_cnt[i] = cnt;
      if (a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) {
        if (cnt) atomicAdd(a.deg + i, cnt * wi);
      } else {
        a.deg[i] = cnt * wi;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_open) atomicAdd(a.counters + kCntScreen, (unsigned long long)s_open);
}

// The queued open pairs, one group of four lanes per pair (eight per warp):
// the FP32 distance over the FP32 points in gather_pair_kernel's order (its
// guard band lo_thr .. hi_thr), the FP64 value inside the band.  Rows that
// are not float4-aligned are summed in order by the group's first lane.
template <int METRIC>
__global__ void __launch_bounds__(256) pair_queue_kernel(GatherArgs a) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const unsigned long long queued = *a.openq_cnt;
  const int64_t total =
      (long long)queued < a.openq_cap ? (int64_t)queued : (int64_t)a.openq_cap;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nc = a.d >> 2;   // float4 chunks (screen_vec4)
  for (int64_t b0 = warp * 8; b0 < total; b0 += warps * 8) {
    const int64_t t = b0 + g;
    const bool valid = t < total;
    const uint4 e = valid ? a.openq[t] : make_uint4(0u, 0u, 0u, 0u);
    const int32_t i = (int32_t)e.x, p = (int32_t)e.y;
    const float *xa = a.xm + (int64_t)i * a.ldm, *xb = a.xm + (int64_t)p * a.ldm;
    float v = 0.f;
    if (a.screen_vec4) {
      float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
      if (valid) {
        for (int c = q; c < nc; c += 4) {
          const float4 u = __ldg(reinterpret_cast<const float4 *>(xa) + c);
          const float4 w = __ldg(reinterpret_cast<const float4 *>(xb) + c);
          ax = pair_combine<METRIC>(ax, fabsf(u.x - w.x));
          ay = pair_combine<METRIC>(ay, fabsf(u.y - w.y));
          az = pair_combine<METRIC>(az, fabsf(u.z - w.z));
          aw = pair_combine<METRIC>(aw, fabsf(u.w - w.w));
        }
      }
      v = pair_combine<METRIC>(pair_combine<METRIC>(ax, ay), pair_combine<METRIC>(az, aw));
    } else if (valid && q == 0) {
      for (int k = 0; k < a.d; ++k)
        v = pair_combine<METRIC>(v, fabsf(__ldg(xa + k) - __ldg(xb + k)));
    }
    v = pair_combine<METRIC>(v, __shfl_xor_sync(kFullMask, v, 1));
    v = pair_combine<METRIC>(v, __shfl_xor_sync(kFullMask, v, 2));
    if (valid && q == 0) {
      const bool keep = v < a.lo_thr ? true : v > a.hi_thr ? false : recheck_pair_metric<METRIC>(a, i, p);
      if (keep) queue_keep(a, i, p, e.z, (int32_t)e.w);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && total > 0)
    atomicAdd(a.counters + kCntScreen, (unsigned long long)total);
}

template <int METRIC, int KC>
static void launch_pm16(const GatherArgs &a, int64_t rows, cudaStream_t st) {
  const int64_t need = (rows + 7) / 8;
  int64_t grid = (int64_t)device_sms() * (KC <= 2 ? 3 : 2);
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  if (a.ld == 32 * KC)
    gather_pair16_kernel<METRIC, KC, true><<<(int)grid, 256, 0, st>>>(a);
  else
    gather_pair16_kernel<METRIC, KC, false><<<(int)grid, 256, 0, st>>>(a);
}

template <int METRIC>
static void launch_pm16_kc(const GatherArgs &a, int64_t rows, int kc, cudaStream_t st) {
  if (kc <= 1) {
    launch_pm16<METRIC, 1>(a, rows, st);
  } else if (kc == 2) {
    launch_pm16<METRIC, 2>(a, rows, st);
  } else {
    launch_pm16<METRIC, 4>(a, rows, st);
  }
}

sng_status launch_gather_pair16(int metric, const GatherArgs &a, int *kc, cudaStream_t st) {
  const int64_t rows = a.row_end - a.row_begin;
  if (a.ld % 8 != 0 || reinterpret_cast<uintptr_t>(a.x) % 16 != 0)
    return fail(SNG_EINTERNAL, "BF16 copy rows of %lld values", (long long)a.ld);
  const int nc = (int)(a.ld / 8);
  const int per_lane = (nc + 3) / 4;
  const int k = per_lane <= 1 ? 1 : per_lane == 2 ? 2 : 4;
  if (metric == SNG_METRIC_L1) {
    launch_pm16_kc<SNG_METRIC_L1>(a, rows, k, st);
  } else if (metric == SNG_METRIC_LINF) {
    launch_pm16_kc<SNG_METRIC_LINF>(a, rows, k, st);
  } else {
    return fail(SNG_EINTERNAL, "no pair-kernel gather for metric %d", metric);
  }
  note_launch();
  if (kc) *kc = k;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "screened pair-kernel gather launch");
}

sng_status launch_pair_queue(int metric, const GatherArgs &a, cudaStream_t st) {
  if (!a.openq || a.openq_cap <= 0) return SNG_OK;
  const int grid = device_sms() * 8;
  if (metric == SNG_METRIC_L1) {
    pair_queue_kernel<SNG_METRIC_L1><<<grid, 256, 0, st>>>(a);
  } else if (metric == SNG_METRIC_LINF) {
    pair_queue_kernel<SNG_METRIC_LINF><<<grid, 256, 0, st>>>(a);
  } else {
    return fail(SNG_EINTERNAL, "no pair-kernel queue for metric %d", metric);
  }
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "pair-kernel open-pair queue");
}

}  // namespace sng
