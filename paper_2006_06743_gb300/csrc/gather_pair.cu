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
#include "api_common.cuh"
#include "gather.cuh"
#include "gather_pair.cuh"

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
// aligned) take one lane per pair with scalar loads.
template <int METRIC, bool VEC4>
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
        src[t] = c < nc ? __ldg(reinterpret_cast<const float4 *>(xa) + c)
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
            if (c < nc) {
              const float4 v = __ldg(vb + c);
              ax = pair_combine<METRIC>(ax, fabsf(src[t].x - v.x));
              ay = pair_combine<METRIC>(ay, fabsf(src[t].y - v.y));
              az = pair_combine<METRIC>(az, fabsf(src[t].z - v.z));
              aw = pair_combine<METRIC>(aw, fabsf(src[t].w - v.w));
            }
          }
          for (int c = q + 4 * kSrcChunks; c < nc; c += 4) {
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
  gather_pair_kernel<METRIC, VEC4><<<(int)grid, 256, 0, st>>>(a);
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

}  // namespace sng
