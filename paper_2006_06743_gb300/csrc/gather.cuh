// gather.cuh -- the sampled eps-graph kernel (Algorithm 1, step 2).
//
// One warp owns one source point i at a time and walks its m partner draws.
// The warp is split into R = 32/G groups of G lanes; each group tests one
// pair (i, p) per step: lane l of the group loads NCH vector chunks of VEC
// elements of row p (coalesced 16-byte loads for FP32 float4 / BF16 x8),
// accumulates squared differences against the same slice of row i held in
// registers, and the group reduces with xor-shuffles.  Partner indices for
// the next 32*U draws are hashed one per lane and staged in shared memory, so
// U pair-loads per lane are in flight at once.  Keep bits are gathered with a
// warp ballot into 32-bit words (bit j of word w = draw 32w + j), giving a
// compact, deterministic record of the kept draws from which the CSR edge list
// is filled in draw order.
//
// Decision rule: the FP32 value certifies the decision outside a guard band
// [lo_thr, hi_thr] around eps^2 that is wider than the FP32 rounding error;
// inside it the group leader recomputes d2 in FP64 in the oracle's order
// (left to right, no contraction) from the FP32 values, so FP32 inputs give
// the FP64 decision on every pair.  For BF16 inputs the band is a heuristic
// (quantisation error is not bounded by it) and the recheck reads the FP32
// master copy.
//
// Similarity form (SIM = true; inner product or cosine, edge iff sim >= tau):
// the lanes also accumulate the partner's squared norm in the same pass (no
// extra memory traffic; the source row's is summed once per row).  The FP32
// inner product is within gamma_K sum |a_k b_k| <= gamma_K |a| |b| of the
// exact one (K roundings per term: one per fused multiply-add and per shuffle
// level), so each pair gets its own certified band from the two norms;
// cosine scales by the two reciprocal square roots (rsqrtf, within 2 ulp by
// CUDA's documented bound), whose error enters through |cos|.  Norms outside [2^-50, 2^50] (zero, tiny,
// huge or non-finite rows) certify nothing.
#pragma once

#include <type_traits>

#include "sng_internal.cuh"

namespace sng {

struct GatherArgs {
  const void *x;          // n x ld, element type T
  int64_t ld;
  const float *xm;        // FP32 values for the FP64 recheck (x itself for F32)
  int64_t ldm;
  int32_t n, d, m, W;     // W = ceil(m/32) words per bitmask row
  int32_t row_begin, row_end;  // source rows this launch processes
  uint64_t seed;
  FastMod fm;
  float lo_thr, hi_thr;   // d2 < lo_thr: keep; d2 > hi_thr: drop; else FP64
  double eps2;            // (double)eps * (double)eps
  double band;            // band_rel * eps2 (reported band half-width;
                          // band_rel * |tau| in the similarity form)
  // similarity form: keep iff sim >= tau.  Certified outside
  // |sim32 - tau| <= sim_c1 |a| |b| + band_f (inner product) or
  // sim_c1 + sim_c2 |cos32| + band_f (cosine), norms from the FP32 sums.
  int32_t cosine;         // 1: cosine, 0: inner product
  float tau, sim_c1, sim_c2, band_f;
  double tau64;
  int32_t sample_all;
  int32_t deg_mode;
  const int32_t *m_row;   // nullable: draws of row i (<= m)
  const int32_t *w_row;   // nullable: degree weight of each kept draw of row i
                          // (both ends); NULL = weight 1
  int32_t pf_bytes;       // > 0: bulk-prefetch this many bytes of each partner
                          // row into L2 one stage ahead (16-byte rows only)
  // BF16 screen of FP32 points (screen = 1): x holds a BF16 copy of the
  // FP32 points xm.  A pair whose FP32 sum over the BF16 values lies below
  // keep_thr or above drop_thr (per-row thresholds from the rows' norm
  // bounds, screen_thresholds) is decided by it; any other pair is summed
  // again from xm in order, one lane, and decided by lo_thr / hi_thr (set for
  // that sequential sum) and the FP64 recheck, exactly as without the screen.
  int32_t screen;
  int32_t screen_vec4;    // xm rows load as float4 (d and ldm multiples of 4)
  float screen_lo_eps;    // eps sqrt(1 - band_rel), rounded down
  float screen_hi_eps;    // eps sqrt(1 + band_rel), rounded up
  float screen_u;         // BF16 rounding bound per unit of norm (rounded up)
  float screen_abs;       // absolute slack: values below BF16's normal range
  float screen_g;         // relative bound of the FP32 sum, plus margins
  const float *nrm;       // per-row upper bounds of |x_i| (FP32 points)
  const float *nrm_max;   // [0] over all rows; [1 + s] over partner slice s
  // tensor-core form of the screen (gather_mma.cu): squared norms of the
  // BF16 rows (FP32 sums) and the coefficient of its absolute error bound
  const float *nb2;
  float screen_cabs;
  // tensor-core forms: nbe[i] = {|x_i'|^2, bound of |x_i - x_i'|}, err_max
  // -> the largest such bound; FP8 form (gather_mma8.cu): the copy holds
  // x * 2^k, k = *screen_kexp
  const float2 *nbe;
  const float *err_max;
  const int32_t *screen_kexp;
  // pairs the screen left open, queued for screen_queue_kernel: entries
  // {i, p, draw j, weight of i}, openq_cnt counts every open pair (past
  // openq_cap the gather decides them itself); q_lo_thr / q_hi_thr are the
  // guard band of the queue kernel's warp-wide FP32 sum
  uint4 *openq;
  unsigned long long *openq_cnt;
  int64_t openq_cap;
  float q_lo_thr, q_hi_thr;
  // similarity form of the tensor-core screens (sim_screen = 1): keep when
  // the pair's certified interval of the similarity lies at or above
  // sim_keep_thr (tau + band, rounded up), drop when below sim_drop_thr
  // (tau - band, rounded down); sim_cm bounds the MMA's accumulation error
  // relative to |a'| |b'|
  int32_t sim_screen;
  float sim_keep_thr, sim_drop_thr, sim_cm;
  // BF16 screen of the Manhattan / Chebyshev distance (gather_pair.cu): the
  // FP32 value over the copy keeps a pair at or below pm_lo - eta and drops
  // it above pm_hi + eta, eta = (e_a + e_b) pm_escale from the rows' copy
  // error bounds (nbe[i].y) -- directed roundings, NaN leaves it open
  float pm_lo, pm_hi, pm_escale;
  uint32_t *bitmask;      // n x W
  int32_t *out_cnt;       // n, nullable
  int32_t *deg;           // n (zeroed before launch in multigraph mode)
  uint8_t *band_flag;     // n
  unsigned long long *counters;
};

// Similarity in FP64 in the oracle's order: inner product and squared norms
// left to right, unfused; cosine = <a,b> / (sqrt(<a,a>) * sqrt(<b,b>)).
__device__ __forceinline__ bool recheck_sim(const GatherArgs &a, int32_t i, int32_t p) {
  const float *xa = a.xm + (int64_t)i * a.ldm, *xb = a.xm + (int64_t)p * a.ldm;
  double ab = 0.0, aa = 0.0, bb = 0.0;
  for (int k = 0; k < a.d; ++k) {
    const double u = (double)xa[k], v = (double)xb[k];
    ab = __dadd_rn(ab, __dmul_rn(u, v));
    if (a.cosine) {
      aa = __dadd_rn(aa, __dmul_rn(u, u));
      bb = __dadd_rn(bb, __dmul_rn(v, v));
    }
  }
  const double s = a.cosine ? __ddiv_rn(ab, __dmul_rn(__dsqrt_rn(aa), __dsqrt_rn(bb))) : ab;
  atomicAdd(a.counters + kCntRecheck, 1ull);
  if (fabs(__dsub_rn(s, a.tau64)) <= a.band) {
    atomicAdd(a.counters + kCntBandPairs, 1ull);
    a.band_flag[i] = 1;
    a.band_flag[p] = 1;
  }
  return s >= a.tau64;
}

template <typename T>
__device__ __forceinline__ bool recheck_pair(const GatherArgs &a, int32_t i, int32_t p) {
  const double s = dist2_fp64(a.xm + (int64_t)i * a.ldm, a.xm + (int64_t)p * a.ldm, a.d);
  atomicAdd(a.counters + kCntRecheck, 1ull);
  if (fabs(__dsub_rn(s, a.eps2)) <= a.band) {
    atomicAdd(a.counters + kCntBandPairs, 1ull);
    a.band_flag[i] = 1;
    a.band_flag[p] = 1;
  }
  return s <= a.eps2;
}

// Keep / drop thresholds of the BF16 screen for source row norm bound nrm_i
// against partner rows of norm bound at most nrm_p.  With a' = bf16(a) (round
// to nearest: |a'_k - a_k| <= 2^-8 |a_k| in the normal range, and at most
// 2^-134 below it) the triangle inequality gives
// | |a - b| - |a' - b'| | <= |a - a'| + |b - b'| <= eta = 2^-8 (|a| + |b|) +
// slack.  The kernel's FP32 sum s of (a'_k - b'_k)^2 is within a relative
// delta of |a' - b'|^2, so s <= (eps - eta)^2 (1 - g) proves |a - b| <= eps
// (the pair is kept) and s > (eps + eta)^2 (1 + g) proves |a - b| > eps
// (dropped), with g = delta plus margins for the rounding of these
// thresholds and of the FP64 reference decision.  eps is taken as
// eps sqrt(1 -/+ band_rel) on the two sides, so that no pair of the reported
// band is decided here (those are all rechecked and counted as without the
// screen).  NaN and infinite bounds certify nothing.
__device__ __forceinline__ void screen_thresholds(const GatherArgs &a, float nrm_i, float nrm_p,
                                                  float &keep_thr, float &drop_thr) {
  const float eta = fmaf(a.screen_u, nrm_i + nrm_p, a.screen_abs);
  const float lo = a.screen_lo_eps - eta;
  const float hi = a.screen_hi_eps + eta;
  keep_thr = lo > 0x1p-10f * a.screen_lo_eps ? (lo * lo) * (1.f - a.screen_g) : -1.f;
  drop_thr = (hi * hi) * (1.f + a.screen_g);
}

// Keep / drop thresholds of a pair (or of a row against every partner) whose
// distance the copy's rounding moves by at most eta (the sum of the two
// rows' own error bounds, by the triangle inequality), widened by the
// evaluation bound e_abs of |a'|^2 + |b'|^2 - 2 a'.b' (gather_mma.cu,
// gather_mma8.cu).
__device__ __forceinline__ void pair_thresholds(const GatherArgs &a, float eta, float e_abs,
                                                float &keep_thr, float &drop_thr) {
  const float lo = a.screen_lo_eps - eta;
  const float hi = a.screen_hi_eps + eta;
  keep_thr = lo > 0x1p-10f * a.screen_lo_eps ? fmaf(lo * lo, 1.f - a.screen_g, -e_abs) : -1.f;
  drop_thr = fmaf(hi * hi, 1.f + a.screen_g, e_abs);
}

// Similarity form of the tensor-core screens: the pair's decision from the
// copy's inner product `dot` (in the units of x) of rows a', b' with squared
// norms na2, nb2 (FP32 sums of exact squares) and rounding-error bounds
// ea >= |a - a'|, eb >= |b - b'|.  <a,b> - <a',b'> = <a - a', b> +
// <a', b - b'>, so |<a,b> - <a',b'>| <= ea (|b'| + eb) + |a'| eb; the MMA
// adds at most sim_cm |a'| |b'|, and 2^-24 |a'| |b'| covers the rounding of
// these terms and of the FP64 reference value.  For cosine the interval of
// <a,b> is divided by the interval of |a| |b| (|a| within ea of |a'|);
// norms outside [2^-60, 2^60] certify nothing.  Returns 1 (keep), 0 (drop)
// or -1 (open: FP64 decides); NaN anywhere leaves the pair open.
static __device__ __noinline__ int sim_screen_decide(const GatherArgs &a, float dot, float na2,
                                                     float ea, float nb2, float eb) {
  const float ra = sqrtf(na2), rb = sqrtf(nb2);   // correctly rounded
  const float na = ra * (1.f + 0x1p-12f), nb = rb * (1.f + 0x1p-12f);   // >= |a'|, |b'|
  float eta = fmaf(ea, nb + eb, na * eb);
  eta = fmaf((a.sim_cm + 0x1p-24f) * na, nb, eta);
  eta = fmaf(eta, 0x1p-20f, eta) + 0x1p-100f;
  const float w = 0x1p-22f * fabsf(dot);
  float lo = dot - eta - w, hi = dot + eta + w;
  if (a.cosine) {
    const float al = fmaf(ra, -0x1p-12f, ra) - ea, bl = fmaf(rb, -0x1p-12f, rb) - eb;
    const float ah = na + ea, bh = nb + eb;
    if (!(al >= 0x1p-60f && bl >= 0x1p-60f && ah <= 0x1p60f && bh <= 0x1p60f)) return -1;
    const float pl = (al * bl) * (1.f - 0x1p-22f), ph = (ah * bh) * (1.f + 0x1p-22f);
    const float cl = lo >= 0.f ? lo / ph : lo / pl;
    const float ch = hi >= 0.f ? hi / pl : hi / ph;
    lo = cl - 0x1p-22f * fabsf(cl);
    hi = ch + 0x1p-22f * fabsf(ch);
  }
  if (lo >= a.sim_keep_thr) return 1;
  if (hi < a.sim_drop_thr) return 0;
  return -1;
}

// The FP64 similarity recheck as a call of its own (the tensor-core gathers
// reach it only for pairs they cannot queue).
static __device__ __noinline__ bool sim_pair(const GatherArgs &a, int32_t i, int32_t p) {
  return recheck_sim(a, i, p);
}

// A pair the BF16 screen left open: the FP32 squared distance of the FP32
// rows, summed in order with one fused multiply-add per element (the bound
// behind lo_thr / hi_thr), then the FP64 recheck inside the guard band --
// the decision of the plain FP32 path, so of the FP64 oracle.
static __device__ __noinline__ bool screen_pair(const GatherArgs &a, int32_t i, int32_t p) {
  const float *xa = a.xm + (int64_t)i * a.ldm, *xb = a.xm + (int64_t)p * a.ldm;
  float acc = 0.f;
  if (a.screen_vec4) {
    // eight 16-byte chunks of each row in flight, then their terms in order
    constexpr int B = 8;
    int k = 0;
    for (; k + 4 * B <= a.d; k += 4 * B) {
      float4 u[B], v[B];
#pragma unroll
      for (int c = 0; c < B; ++c) {
        u[c] = __ldg(reinterpret_cast<const float4 *>(xa + k) + c);
        v[c] = __ldg(reinterpret_cast<const float4 *>(xb + k) + c);
      }
#pragma unroll
      for (int c = 0; c < B; ++c) {
        float t = u[c].x - v[c].x;
        acc = fmaf(t, t, acc);
        t = u[c].y - v[c].y;
        acc = fmaf(t, t, acc);
        t = u[c].z - v[c].z;
        acc = fmaf(t, t, acc);
        t = u[c].w - v[c].w;
        acc = fmaf(t, t, acc);
      }
    }
    for (; k < a.d; k += 4) {
      const float4 u = __ldg(reinterpret_cast<const float4 *>(xa + k));
      const float4 v = __ldg(reinterpret_cast<const float4 *>(xb + k));
      float t = u.x - v.x;
      acc = fmaf(t, t, acc);
      t = u.y - v.y;
      acc = fmaf(t, t, acc);
      t = u.z - v.z;
      acc = fmaf(t, t, acc);
      t = u.w - v.w;
      acc = fmaf(t, t, acc);
    }
  } else {
    for (int k = 0; k < a.d; ++k) {
      const float t = __ldg(xa + k) - __ldg(xb + k);
      acc = fmaf(t, t, acc);
    }
  }
  if (acc < a.lo_thr) return true;
  if (acc > a.hi_thr) return false;
  return recheck_pair<float>(a, i, p);
}

// Bulk prefetch of the start of partner row p into L2 (the copy engine
// fetches it while the warp works on the current stage).  Only for rows that
// start on 16 bytes (16-byte vector mappings); the size is a multiple of 16.
template <typename T, int VEC>
__device__ __forceinline__ void prefetch_row(const GatherArgs &a, int32_t p) {
  if constexpr (VEC * sizeof(T) == 16) {
    const T *row = static_cast<const T *>(a.x) + (int64_t)p * a.ld;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(row), "r"(a.pf_bytes)
                 : "memory");
  }
}

// Partners of draws j0 .. j0+32U-1 of row i into buf (one hash per lane per
// batch of 32; -1 past the row's draws), prefetching their rows if enabled.
template <typename T, int VEC, int U>
__device__ __forceinline__ void stage_partners(const GatherArgs &a, int32_t i, uint64_t key,
                                               int64_t j0, int32_t mi, int32_t *buf, int lane) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t j = j0 + u * 32 + lane;
    int32_t p = -1;
    if (j < mi) p = a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, a.fm);
    buf[u * 32 + lane] = p;
    if (a.pf_bytes > 0 && p >= 0) prefetch_row<T, VEC>(a, p);
  }
}

// One source row: draws 0..mi-1 of point i, keep bits into bitmask row i,
// in-degree atomics; returns the row's kept count (same value on all lanes).
// `sp` is this warp's 2*32*U-entry shared-memory partner buffer: the stage
// being tested and the next one, hashed (and prefetched) one stage ahead.
template <typename T, int VEC, int G, int NCH, int U, bool SIM = false, bool FULL = false>
__device__ __forceinline__ int gather_row(const GatherArgs &a, int32_t i, int32_t mi,
                                          int32_t *sp, int lane, unsigned int *screen_cnt = nullptr) {
  constexpr int R = 32 / G;      // pairs per warp step
  constexpr int S = 32 * U;      // draws per stage
  constexpr int STEPS = S / R;   // warp steps per stage
  const int grp = lane / G;
  const int gl = lane % G;
  const T *X = static_cast<const T *>(a.x);
  const int d = a.d;
  const uint64_t key = row_key(a.seed, i);
  const int32_t wi = a.w_row ? a.w_row[i] : 1;
  constexpr bool kScreenable = std::is_same<T, uint16_t>::value && !SIM;
  float keep_thr = 0.f, drop_thr = 0.f;
  if constexpr (kScreenable) {
    if (a.screen) screen_thresholds(a, a.nrm[i], a.nrm_max[0], keep_thr, drop_thr);
  }

  // this lane's slice of row i; elements at or past d read as zero
  float xi[NCH][VEC];
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int off = (c * G + gl) * VEC;
    if (FULL || off < d) {
      Chunk<T, VEC>::load(X + (int64_t)i * a.ld + off, xi[c]);
#pragma unroll
      for (int k = 0; k < VEC; ++k)
        if (!FULL && off + k >= d) xi[c][k] = 0.f;
    } else {
#pragma unroll
      for (int k = 0; k < VEC; ++k) xi[c][k] = 0.f;
    }
  }

  // similarity form: the row's scale, from its squared norm summed like a
  // pair (group reduction): 1/|x_i| for cosine, |x_i| for the inner
  // product; NaN when the norm is outside [2^-50, 2^50] (zero, tiny, huge or
  // non-finite row), which then certifies none of the row's pairs
  float scale_i = 1.f;
  if constexpr (SIM) {
    float nn = 0.f;
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
      for (int k = 0; k < VEC; ++k) nn = fmaf(xi[c][k], xi[c][k], nn);
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) nn += __shfl_xor_sync(kFullMask, nn, o);
    const float r = rsqrtf(nn);   // within 2 ulp (CUDA's documented bound)
    scale_i = a.cosine ? r : nn * r;
    if (!(nn >= 0x1p-100f && nn <= 0x1p100f)) scale_i = __int_as_float(0x7fc00000);
  }

  int cnt = 0;
  int jb = 0;
  int32_t *cur = sp, *nxt = sp + S;
  if (mi > 0) stage_partners<T, VEC, U>(a, i, key, 0, mi, cur, lane);
  for (; jb < mi; jb += S) {
    if (jb + S < mi) stage_partners<T, VEC, U>(a, i, key, (int64_t)jb + S, mi, nxt, lane);
    __syncwarp();
    uint32_t myword = 0;
#pragma unroll 1
    for (int t0 = 0; t0 < STEPS; t0 += U) {
      typename Raw<T, VEC>::type v[U][NCH];
      int32_t pv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int t = t0 + u;
        const int32_t p = cur[t * R + grp];
        pv[u] = p;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          const int off = (c * G + gl) * VEC;
          v[u][c] = (p >= 0 && (FULL || off < d)) ? Raw<T, VEC>::load(X + (int64_t)p * a.ld + off)
                                        : Raw<T, VEC>::zero();
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int t = t0 + u;
        float acc = 0.f;
        float bb = 0.f;     // similarity form: partner's squared norm
        // full-row instantiations: even and odd elements in the two halves of
        // packed FP32x2 accumulators (one instruction per element pair)
        F32x2 acc2 = f32x2_zero(), bb2 = f32x2_zero();
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          const int off = (c * G + gl) * VEC;
          if (FULL && VEC % 2 == 0) {
#pragma unroll
            for (int k = 0; k < VEC; k += 2) {
              const F32x2 a2 = f32x2_pack(xi[c][k], xi[c][k + 1]);
              const F32x2 b2 = f32x2_pack(Raw<T, VEC>::get(v[u][c], k),
                                          Raw<T, VEC>::get(v[u][c], k + 1));
              if constexpr (SIM) {
                acc2 = f32x2_fma(a2, b2, acc2);
                bb2 = f32x2_fma(b2, b2, bb2);
              } else {
                const F32x2 d2 = f32x2_sub(a2, b2);
                acc2 = f32x2_fma(d2, d2, acc2);
              }
            }
          } else if (FULL || off + VEC <= d) {
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
              if constexpr (SIM) {
                const float b = Raw<T, VEC>::get(v[u][c], k);
                acc = fmaf(xi[c][k], b, acc);
                bb = fmaf(b, b, bb);
              } else {
                const float diff = xi[c][k] - Raw<T, VEC>::get(v[u][c], k);
                acc = fmaf(diff, diff, acc);
              }
            }
          } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
              if constexpr (SIM) {
                float b = Raw<T, VEC>::get(v[u][c], k);
                if (off + k >= d) b = 0.f;   // row padding may hold anything
                acc = fmaf(xi[c][k], b, acc);
                bb = fmaf(b, b, bb);
              } else {
                float diff = xi[c][k] - Raw<T, VEC>::get(v[u][c], k);
                if (off + k >= d) diff = 0.f;
                acc = fmaf(diff, diff, acc);
              }
            }
          }
        }
        if constexpr (FULL && VEC % 2 == 0) {
          acc = f32x2_sum(acc2);
          if constexpr (SIM) bb = f32x2_sum(bb2);
        }
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) {
          acc += __shfl_xor_sync(kFullMask, acc, o);
          if constexpr (SIM) bb += __shfl_xor_sync(kFullMask, bb, o);
        }
        bool keep = false;
        const int32_t p = pv[u];
        if (gl == 0 && p >= 0) {
          if constexpr (SIM) {
            const float inv_p = rsqrtf(bb);
            float sim, err;
            if (a.cosine) {
              sim = (acc * scale_i) * inv_p;
              err = a.sim_c1 + a.sim_c2 * fabsf(sim);
            } else {
              sim = acc;
              err = a.sim_c1 * (scale_i * (bb * inv_p));   // c1 |a| |b|
            }
            // zero, tiny, huge or non-finite norms certify nothing (a NaN
            // scale_i has already made err NaN)
            const bool ok = bb >= 0x1p-100f && bb <= 0x1p100f;
            err = ok ? err + a.band_f : __int_as_float(0x7fc00000);
            // NaN (zero or non-finite rows) certifies nothing: FP64 decides
            if (sim - err >= a.tau) {
              keep = true;
            } else if (!(sim + err < a.tau)) {
              keep = recheck_sim(a, i, p);
            }
          } else {
            bool screened = false;
            if constexpr (kScreenable) {
              if (a.screen) {
                screened = true;
                if (acc < keep_thr) {
                  keep = true;
                } else if (!(acc > drop_thr)) {
                  keep = screen_pair(a, i, p);
                  if (screen_cnt) atomicAdd(screen_cnt, 1u);   // shared-memory tally
                }
              }
            }
            if (!screened) {
              if (acc < a.lo_thr) {
                keep = true;
              } else if (!(acc > a.hi_thr)) {
                keep = recheck_pair<T>(a, i, p);
              }
            }
          }
          if (keep && a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) atomicAdd(a.deg + p, wi);
        }
        // R keep flags (held by the group leaders, lanes g*G) -> R low bits
        uint32_t bits;
        if (G == 1) {
          bits = __ballot_sync(kFullMask, keep);
        } else {
          const int src = (lane < R ? lane : 0) * G;
          const bool kg = __shfl_sync(kFullMask, keep ? 1 : 0, src) != 0;
          bits = __ballot_sync(kFullMask, lane < R && kg);
        }
        const int first = t * R;  // draw index within the stage
        if (lane == (first >> 5)) myword |= bits << (first & 31);
      }
    }
    // keep-bit words are written once and read back only by later kernels:
    // streaming (evict-first) stores leave L2 to the partner rows
    const int w = (jb >> 5) + lane;
    if (lane < U && w < a.W) __stcs(a.bitmask + (int64_t)i * a.W + w, myword);
    cnt += __popc(myword);
    __syncwarp();
    int32_t *t = cur;
    cur = nxt;
    nxt = t;
  }
  // words past this row's draws (per-row draw counts) are zero
  for (int w = (jb >> 5) + lane; w < a.W; w += 32) __stcs(a.bitmask + (int64_t)i * a.W + w, 0u);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(kFullMask, cnt, o);
  if (lane == 0) {
    if (a.out_cnt) a.out_cnt[i] = cnt;
    if (a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) {
      if (cnt) atomicAdd(a.deg + i, cnt * wi);
    } else {
      a.deg[i] = cnt * wi;
    }
  }
  return cnt;
}

// One lane per source row, for rows of at most NCH vectors of VEC elements
// (the mappings with one lane per pair): each lane hashes its own row's
// draws, keeps U partner rows in flight and assembles the keep-bit words in
// a register -- no shared-memory staging, no ballots, no idle slots in a
// row's last stage.  Rows [r0, r1) are taken 32 at a time by warps
// first_warp, first_warp + warp_stride, ...  Decisions, keep bits, row
// counts and degrees are those of gather_row.  Returns this lane's kept
// draws.
template <typename T, int VEC, int NCH, int U>
__device__ __forceinline__ unsigned long long gather_rows_lanes(const GatherArgs &a, int64_t r0,
                                                                int64_t r1, int lane,
                                                                int64_t first_warp,
                                                                int64_t warp_stride) {
  const T *X = static_cast<const T *>(a.x);
  const int d = a.d;
  unsigned long long kept = 0;
  for (int64_t base = r0 + first_warp * 32; base < r1; base += warp_stride * 32) {
    const int64_t row = base + lane;
    if (row >= r1) continue;
    const int32_t i = (int32_t)row;
    const int32_t mi = a.m_row ? a.m_row[i] : a.m;
    const int32_t wi = a.w_row ? a.w_row[i] : 1;
    const uint64_t key = row_key(a.seed, i);
    float xi[NCH][VEC];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const int off = c * VEC;
      if (off < d) {
        Chunk<T, VEC>::load(X + (int64_t)i * a.ld + off, xi[c]);
#pragma unroll
        for (int k = 0; k < VEC; ++k)
          if (off + k >= d) xi[c][k] = 0.f;
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) xi[c][k] = 0.f;
      }
    }
    int cnt = 0;
    for (int jb = 0; jb < mi; jb += 32) {
      const int jn = min(32, mi - jb);
      uint32_t word = 0;
      for (int j0 = 0; j0 < jn; j0 += U) {
        int32_t p[U];
        typename Raw<T, VEC>::type v[U][NCH];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t j = (int64_t)jb + j0 + u;
          p[u] = -1;
          if (j0 + u < jn) p[u] = a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, a.fm);
#pragma unroll
          for (int c = 0; c < NCH; ++c)
            v[u][c] = (p[u] >= 0 && c * VEC < d)
                          ? Raw<T, VEC>::load(X + (int64_t)p[u] * a.ld + c * VEC)
                          : Raw<T, VEC>::zero();
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (p[u] < 0) continue;
          float acc = 0.f;
#pragma unroll
          for (int c = 0; c < NCH; ++c) {
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
              float diff = xi[c][k] - Raw<T, VEC>::get(v[u][c], k);
              if (c * VEC + k >= d) diff = 0.f;   // row padding may hold anything
              acc = fmaf(diff, diff, acc);
            }
          }
          bool keep = false;
          if (acc < a.lo_thr) {
            keep = true;
          } else if (!(acc > a.hi_thr)) {
            keep = recheck_pair<T>(a, i, p[u]);
          }
          if (keep) {
            word |= 1u << (j0 + u);
            if (a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) atomicAdd(a.deg + p[u], wi);
          }
        }
      }
      __stcs(a.bitmask + (int64_t)i * a.W + (jb >> 5), word);
      cnt += __popc(word);
    }
    // words past this row's draws (per-row draw counts) are zero
    for (int w = (mi + 31) >> 5; w < a.W; ++w) __stcs(a.bitmask + (int64_t)i * a.W + w, 0u);
    if (a.out_cnt) a.out_cnt[i] = cnt;
    if (a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) {
      if (cnt) atomicAdd(a.deg + i, cnt * wi);
    } else {
      a.deg[i] = cnt * wi;
    }
    kept += (unsigned long long)cnt;
  }
  return kept;
}

// Resident 256-thread blocks per SM the compiler must allow for: mappings
// with few registers of row data get 4 (32 warps), wider ones 3 or 2.
template <typename T, int VEC, int NCH, int U, bool SIM = false>
struct MinBlocks {
  // 32-bit registers per lane of row data: partner chunks in flight (raw
  // bits) plus this lane's slice of the source row (FP32); the similarity
  // form carries a second accumulator per pair and the row's norms besides
  static constexpr int words = U * NCH * (VEC * (int)sizeof(T) / 4 > 0 ? VEC * (int)sizeof(T) / 4 : 1) +
                               NCH * VEC + (SIM ? 2 * U + 4 : 0);
  static constexpr int value = words <= 32 ? 4 : (words <= 56 ? 3 : 2);
};

// FULL: every row is exactly G * NCH * VEC elements wide (no partial or
// empty chunk), so the per-chunk bounds tests drop out of the pair loop.
// LANES: one lane per source row (G == 1 only; see gather_rows_lanes).
template <typename T, int VEC, int G, int NCH, int U, bool SIM = false, bool FULL = false,
          bool LANES = false>
__global__ void __launch_bounds__(256, MinBlocks<T, VEC, NCH, U, SIM>::value)
    gather_kernel(GatherArgs a) {
  extern __shared__ int32_t smem_partner[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  if constexpr (LANES) {
    static_assert(G == 1 && !SIM, "one lane per row: Euclidean form, one lane per pair");
    gather_rows_lanes<T, VEC, NCH, U>(a, a.row_begin, a.row_end, lane,
                                      (int64_t)blockIdx.x * (blockDim.x >> 5) + warp,
                                      (int64_t)gridDim.x * (blockDim.x >> 5));
    return;
  }
  int32_t *sp = smem_partner + warp * 64 * U;   // two stages of 32*U partners
  __shared__ unsigned int s_screen;               // pairs the BF16 screen left open
  if (threadIdx.x == 0) s_screen = 0;
  __syncthreads();
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = a.row_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
       row < a.row_end; row += warps_total) {
    const int32_t i = (int32_t)row;
    const int32_t mi = a.m_row ? a.m_row[i] : a.m;
    gather_row<T, VEC, G, NCH, U, SIM, FULL>(a, i, mi, sp, lane, &s_screen);
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_screen) atomicAdd(a.counters + kCntScreen, (unsigned long long)s_screen);
}

// L2-blocked form: one launch per slice [lo, hi) of partner indices.  Each
// warp re-derives all m draws of its row, keeps the ones whose partner lies
// in the slice (warp-ballot compaction into a shared-memory list of (draw,
// partner)), and tests only those, so a launch touches one slice of X that
// stays resident in L2 while every source row streams past it once.  Kept
// draws set their bit with atomicOr (the bitmask is zeroed before the first
// slice) and add to the row count; degrees as in gather_row.
template <typename T, int VEC, int G, int NCH, int U>
__device__ __forceinline__ void gather_row_blocked(const GatherArgs &a, int32_t i, int32_t mi,
                                                   int32_t lo, int32_t hi, int32_t *sp,
                                                   int32_t *sj, int lane) {
  constexpr int R = 32 / G;
  constexpr int S = 32 * U;   // list capacity
  const int grp = lane / G;
  const int gl = lane % G;
  const T *X = static_cast<const T *>(a.x);
  const int d = a.d;
  const uint64_t key = row_key(a.seed, i);
  const int32_t wi = a.w_row ? a.w_row[i] : 1;
  float xi[NCH][VEC];
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int off = (c * G + gl) * VEC;
    if (off < d) {
      Chunk<T, VEC>::load(X + (int64_t)i * a.ld + off, xi[c]);
#pragma unroll
      for (int k = 0; k < VEC; ++k)
        if (off + k >= d) xi[c][k] = 0.f;
    } else {
#pragma unroll
      for (int k = 0; k < VEC; ++k) xi[c][k] = 0.f;
    }
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
  int cnt = 0;
  int64_t j = 0;
  while (j < mi) {
    int nlist = 0;
    while (nlist <= S - 32 && j < mi) {
      const int64_t jj = j + lane;
      int32_t p = -1;
      if (jj < mi) p = a.sample_all ? partner_all(i, jj) : partner_from_key(key, i, jj, a.fm);
      const bool in = p >= lo && p < hi;
      const uint32_t b = __ballot_sync(kFullMask, in);
      if (in) {
        const int pos = nlist + __popc(b & lt_mask);
        sp[pos] = p;
        sj[pos] = (int32_t)jj;
      }
      nlist += __popc(b);
      j += 32;
    }
    __syncwarp();
    const int steps = (nlist + R - 1) / R;
#pragma unroll 1
    for (int t0 = 0; t0 < steps; t0 += U) {
      typename Raw<T, VEC>::type v[U][NCH];
      int32_t pv[U], jv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = (t0 + u) * R + grp;
        const int32_t p = e < nlist ? sp[e] : -1;
        pv[u] = p;
        jv[u] = e < nlist ? sj[e] : 0;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          const int off = (c * G + gl) * VEC;
          v[u][c] = (p >= 0 && off < d) ? Raw<T, VEC>::load(X + (int64_t)p * a.ld + off)
                                        : Raw<T, VEC>::zero();
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          const int off = (c * G + gl) * VEC;
#pragma unroll
          for (int k = 0; k < VEC; ++k) {
            float diff = xi[c][k] - Raw<T, VEC>::get(v[u][c], k);
            if (off + VEC > d && off + k >= d) diff = 0.f;
            acc = fmaf(diff, diff, acc);
          }
        }
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) acc += __shfl_xor_sync(kFullMask, acc, o);
        const int32_t p = pv[u];
        if (gl == 0 && p >= 0) {
          bool keep = false;
          if (acc < a.lo_thr) {
            keep = true;
          } else if (!(acc > a.hi_thr)) {
            keep = recheck_pair<T>(a, i, p);
          }
          if (keep) {
            const int32_t jj = jv[u];
            atomicOr(a.bitmask + (int64_t)i * a.W + (jj >> 5), 1u << (jj & 31));
            if (a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) atomicAdd(a.deg + p, wi);
            ++cnt;
          }
        }
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(kFullMask, cnt, o);
  if (lane == 0 && cnt) {
    if (a.out_cnt) atomicAdd(a.out_cnt + i, cnt);
    atomicAdd(a.deg + i, cnt * wi);
  }
}

template <typename T, int VEC, int G, int NCH, int U>
__global__ void __launch_bounds__(256, MinBlocks<T, VEC, NCH, U>::value)
    gather_blocked_kernel(GatherArgs a, int32_t lo, int32_t hi) {
  extern __shared__ int32_t smem_list[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  int32_t *sp = smem_list + warp * 64 * U;
  int32_t *sj = sp + 32 * U;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = a.row_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
       row < a.row_end; row += warps_total) {
    const int32_t i = (int32_t)row;
    const int32_t mi = a.m_row ? a.m_row[i] : a.m;
    gather_row_blocked<T, VEC, G, NCH, U>(a, i, mi, lo, hi, sp, sj, lane);
  }
}

// Mapping of the gather: lanes per pair, chunks per lane, vector width,
// batches in flight, block size.
struct GatherMap {
  int vec, group, nch, unroll, block;
  int passes;   // 1: single pass; > 1: L2-blocked slices of the partner range
  int sim;      // 1: similarity form (inner product / cosine) of the kernel
  int full;     // 1: d == group * nch * vec (a FULL instantiation may serve)
  int lanes;    // 1: one lane per source row (a LANES instantiation may serve)
};

// Host-side launcher; returns false if no compiled variant matches `map`.
bool launch_gather(int dtype, const GatherMap &map, const GatherArgs &args, int grid,
                   cudaStream_t stream);
bool launch_gather_blocked(int dtype, const GatherMap &map, const GatherArgs &args, int grid,
                           int32_t lo, int32_t hi, cudaStream_t stream);
int gather_blocked_max_blocks_per_sm(int dtype, const GatherMap &map);
// Whether a mapping has a compiled kernel (host-only check, no CUDA call).
bool gather_is_compiled(int dtype, const GatherMap &map);
bool gather_blocked_is_compiled(int dtype, const GatherMap &map);
size_t gather_smem_bytes(const GatherMap &map);
int gather_max_blocks_per_sm(int dtype, const GatherMap &map);

}  // namespace sng
