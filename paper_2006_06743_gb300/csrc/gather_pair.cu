// gather_pair.cu -- step 2 of Algorithm 1 with the Manhattan (L1) or
// Chebyshev (L-inf) distance as the neighbourhood test.  The method needs
// only similarity queries (Section 1); these two are pair kernels that are
// neither the Euclidean ball nor an inner product, so no norm identity or
// tensor-core form applies.
//
// One warp per source row, one lane per draw, stages of 32 draws: lane r
// hashes draw r, walks its partner row (16-byte loads where rows allow;
// the source row's values are the same address for every lane, a broadcast),
// and forms the distance in FP32 -- the sum of |a_k - b_k| in order, or their
// maximum.  Outside the guard band around eps (validate, api.cu) the FP32
// value decides; inside it the FP64 value in the oracle's order does
// (recheck_pair_metric, which also counts the reported band).  Keep bits by
// ballot, degrees by atomics, as in the other gathers.
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

template <int METRIC>
__device__ __forceinline__ void pair_step(float u, float v, float &acc, bool &nan) {
  const float t = fabsf(u - v);
  if (METRIC == SNG_METRIC_L1) {
    acc += t;
  } else {
    nan |= t != t;   // fmaxf would drop a NaN
    acc = t > acc ? t : acc;
  }
}

template <int METRIC, bool VEC4>
__global__ void __launch_bounds__(256) gather_pair_kernel(GatherArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = a.row_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
       row < a.row_end; row += warps_total) {
    const int32_t i = (int32_t)row;
    const int32_t mi = a.m_row ? a.m_row[i] : a.m;
    const int32_t wi = a.w_row ? a.w_row[i] : 1;
    const uint64_t key = row_key(a.seed, i);
    const float *xa = a.xm + (int64_t)i * a.ldm;
    int cnt = 0;
    for (int jb = 0; jb < mi; jb += 32) {
      const int j = jb + lane;
      const bool live = j < mi;
      // draws past the row's count read row 0 and decide nothing
      const int32_t p =
          live ? (a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, a.fm)) : 0;
      const float *xb = a.xm + (int64_t)p * a.ldm;
      float acc = 0.f;
      bool nan = false;
      if (VEC4) {
        const float4 *ua = reinterpret_cast<const float4 *>(xa);
        const float4 *vb = reinterpret_cast<const float4 *>(xb);
        for (int k = 0; k < (a.d >> 2); ++k) {
          const float4 u = __ldg(ua + k), v = __ldg(vb + k);
          pair_step<METRIC>(u.x, v.x, acc, nan);
          pair_step<METRIC>(u.y, v.y, acc, nan);
          pair_step<METRIC>(u.z, v.z, acc, nan);
          pair_step<METRIC>(u.w, v.w, acc, nan);
        }
      } else {
        for (int k = 0; k < a.d; ++k) pair_step<METRIC>(__ldg(xa + k), __ldg(xb + k), acc, nan);
      }
      if (nan) acc = __int_as_float(0x7fc00000);
      bool keep = false;
      if (live) {
        if (acc < a.lo_thr) {
          keep = true;
        } else if (!(acc > a.hi_thr)) {
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
