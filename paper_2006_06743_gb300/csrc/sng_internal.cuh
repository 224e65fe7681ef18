// sng_internal.cuh -- device helpers shared by the SNG-DBSCAN kernels.
//
// Partner draws of Algorithm 1, step 2 (Jiang, Jang & Lacki 2020, Section 3):
// each point i draws m partners with replacement, never itself.  The draw is a
// counter-based hash so that every implementation sees the same pairs:
//   mix(z)  = SplitMix64 output function (Steele, Lea & Flood 2014)
//   k_i     = mix(seed ^ mix(i)),  h = mix(k_i ^ j)
//   r       = h mod (n - 1),       partner = r + (r >= i)
// The remainder is computed without a 64-bit divide by the direct-remainder
// method of Lemire, Kaser & Kurz (2019): for a < 2^N and d < 2^L, with
// c = ceil(2^F / d) and F >= N + L, a mod d = ((c * a mod 2^F) * d) >> F.
// Here N = 64, d = n - 1 < 2^31 and F = 96.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sng.h"

namespace sng {

constexpr uint32_t kFullMask = 0xffffffffu;
constexpr int32_t kNoLabel = 0x7fffffff;
// Largest draw count per point: the gather loops step a 32-bit draw index by
// up to 256 draws, which must not overflow.
constexpr int64_t kMaxDraws = 0x7fffffffLL - 1024;

// Device status word bits (written by kernels, read back by the host).
constexpr uint32_t kErrUnionLimit = 1u << 0;   // union-find retry bound hit
constexpr uint32_t kErrFindLimit = 1u << 1;    // find walked more than n steps
constexpr uint32_t kErrBatchLimit = 1u << 2;   // batched scheduler bound hit
constexpr uint32_t kErrIndex = 1u << 3;        // an index fell outside its array
constexpr uint32_t kErrDeviceWait = 1u << 6;   // a bounded wait on tensor-core / TMA completion gave up

// Counters kept on the device for sng_stats (unsigned long long each).
enum CounterSlot : int {
  kCntKept = 0,
  kCntBandPairs = 1,
  kCntRecheck = 2,
  kCntBandPoints = 3,
  kCntCores = 4,
  kCntClusters = 5,
  kCntNoise = 6,
  kCntEdges = 7,      // scan total
  kCntStatus = 8,     // error bits (uint32 stored in a 64-bit slot)
  kCntScreen = 9,     // pairs the BF16 screen of FP32 points left open
  kCntSlots = 16
};

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Constants for r = a mod dv, dv = n - 1 in [1, 2^31 - 2].
struct FastMod {
  uint64_t c_lo;   // low 64 bits of c = ceil(2^96 / dv)
  uint32_t c_hi;   // bits 64..95 of c
  uint32_t dv;     // divisor; dv == 1 is handled directly (r = 0)
};

// a mod dv by direct computation (Lemire, Kaser & Kurz 2019, F = 96).
__device__ __forceinline__ uint32_t fast_mod(uint64_t a, const FastMod &f) {
  if (f.dv == 1u) return 0u;
  // L = c * a mod 2^96, kept as (l_hi:32, l_lo:64)
  const uint64_t l_lo = f.c_lo * a;
  const uint64_t p_hi = __umul64hi(f.c_lo, a);
  const uint32_t l_hi = (uint32_t)p_hi + f.c_hi * (uint32_t)a;
  // (L * dv) >> 96 = (l_hi*dv + umulhi(l_lo, dv)) >> 32
  const uint64_t acc = (uint64_t)l_hi * f.dv + __umul64hi(l_lo, (uint64_t)f.dv);
  return (uint32_t)(acc >> 32);
}

__device__ __forceinline__ uint64_t row_key(uint64_t seed, int64_t i) {
  return mix64(seed ^ mix64((uint64_t)i));
}

// Partner j of point i given its key (hash mode).
__device__ __forceinline__ int32_t partner_from_key(uint64_t key, int32_t i, int64_t j,
                                                    const FastMod &f) {
  const uint32_t r = fast_mod(mix64(key ^ (uint64_t)j), f);
  return (int32_t)r + ((int32_t)r >= i ? 1 : 0);
}

__device__ __forceinline__ int32_t partner_all(int32_t i, int64_t j) {
  return (int32_t)j + ((int32_t)j >= i ? 1 : 0);
}

// Host: build the remainder constants for dv = n - 1.
inline FastMod make_fastmod(int64_t n) {
  FastMod f;
  const uint64_t dv = (uint64_t)(n - 1);
  f.dv = (uint32_t)dv;
  if (dv <= 1) {
    f.c_lo = 0;
    f.c_hi = 0;
    return f;
  }
  const unsigned __int128 two96 = (unsigned __int128)1 << 96;
  unsigned __int128 c = two96 / dv + ((two96 % dv) != 0 ? 1 : 0);
  f.c_lo = (uint64_t)c;
  f.c_hi = (uint32_t)(c >> 64);
  return f;
}

// ---------------------------------------------------------------- loads

__device__ __forceinline__ float bf16_bits_to_f32(uint16_t b) {
  return __uint_as_float(((uint32_t)b) << 16);
}

// Read-only vector loads of one chunk of VEC elements, converted to FP32.
// Packed FP32 pairs (Blackwell's two-wide FP32 add / fused multiply-add):
// each half is rounded exactly as the scalar operation on that half.
typedef unsigned long long F32x2;
__device__ __forceinline__ F32x2 f32x2_zero() { return 0ull; }
__device__ __forceinline__ F32x2 f32x2_pack(float lo, float hi) {
  F32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ F32x2 f32x2_sub(F32x2 a, F32x2 b) {
  F32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ F32x2 f32x2_fma(F32x2 a, F32x2 b, F32x2 c) {
  F32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// lo + hi, one rounding
__device__ __forceinline__ float f32x2_sum(F32x2 v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return lo + hi;
}

template <typename T, int VEC>
struct Chunk;

template <>
struct Chunk<float, 4> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <>
struct Chunk<float, 2> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[2]) {
    const float2 q = __ldg(reinterpret_cast<const float2 *>(p));
    v[0] = q.x; v[1] = q.y;
  }
};
template <>
struct Chunk<float, 1> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[1]) { v[0] = __ldg(p); }
};
template <>
struct Chunk<uint16_t, 8> {
  static __device__ __forceinline__ void load(const uint16_t *p, float (&v)[8]) {
    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = __uint_as_float(w[k] << 16);
      v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
};
template <>
struct Chunk<uint16_t, 4> {
  static __device__ __forceinline__ void load(const uint16_t *p, float (&v)[4]) {
    const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
    v[0] = __uint_as_float(q.x << 16);
    v[1] = __uint_as_float(q.x & 0xffff0000u);
    v[2] = __uint_as_float(q.y << 16);
    v[3] = __uint_as_float(q.y & 0xffff0000u);
  }
};
template <>
struct Chunk<uint16_t, 2> {
  static __device__ __forceinline__ void load(const uint16_t *p, float (&v)[2]) {
    const uint32_t q = __ldg(reinterpret_cast<const unsigned int *>(p));
    v[0] = __uint_as_float(q << 16);
    v[1] = __uint_as_float(q & 0xffff0000u);
  }
};
template <>
struct Chunk<uint16_t, 1> {
  static __device__ __forceinline__ void load(const uint16_t *p, float (&v)[1]) {
    v[0] = bf16_bits_to_f32(__ldg(reinterpret_cast<const unsigned short *>(p)));
  }
};

// Raw vector registers of one chunk (the loaded bits, widened to FP32 only
// where an element is used): float4/float2/float for FP32, uint4/uint2/uint
// of packed bfloat16 pairs for BF16.
template <typename T, int VEC>
struct Raw;

template <>
struct Raw<float, 4> {
  using type = float4;
  static __device__ __forceinline__ type load(const float *p) {
    return __ldg(reinterpret_cast<const float4 *>(p));
  }
  static __device__ __forceinline__ float get(const type &v, int k) {
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
  }
  static __device__ __forceinline__ type zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <>
struct Raw<float, 2> {
  using type = float2;
  static __device__ __forceinline__ type load(const float *p) {
    return __ldg(reinterpret_cast<const float2 *>(p));
  }
  static __device__ __forceinline__ float get(const type &v, int k) { return k == 0 ? v.x : v.y; }
  static __device__ __forceinline__ type zero() { return make_float2(0.f, 0.f); }
};
template <>
struct Raw<float, 1> {
  using type = float;
  static __device__ __forceinline__ type load(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ float get(const type &v, int) { return v; }
  static __device__ __forceinline__ type zero() { return 0.f; }
};
template <>
struct Raw<uint16_t, 8> {
  using type = uint4;
  static __device__ __forceinline__ type load(const uint16_t *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
  }
  static __device__ __forceinline__ float get(const type &v, int k) {
    const uint32_t w = (k >> 1) == 0 ? v.x : (k >> 1) == 1 ? v.y : (k >> 1) == 2 ? v.z : v.w;
    return __uint_as_float((k & 1) ? (w & 0xffff0000u) : (w << 16));
  }
  static __device__ __forceinline__ type zero() { return make_uint4(0u, 0u, 0u, 0u); }
};
template <>
struct Raw<uint16_t, 4> {
  using type = uint2;
  static __device__ __forceinline__ type load(const uint16_t *p) {
    return __ldg(reinterpret_cast<const uint2 *>(p));
  }
  static __device__ __forceinline__ float get(const type &v, int k) {
    const uint32_t w = (k >> 1) == 0 ? v.x : v.y;
    return __uint_as_float((k & 1) ? (w & 0xffff0000u) : (w << 16));
  }
  static __device__ __forceinline__ type zero() { return make_uint2(0u, 0u); }
};
template <>
struct Raw<uint16_t, 2> {
  using type = uint32_t;
  static __device__ __forceinline__ type load(const uint16_t *p) {
    return __ldg(reinterpret_cast<const unsigned int *>(p));
  }
  static __device__ __forceinline__ float get(const type &v, int k) {
    return __uint_as_float(k ? (v & 0xffff0000u) : (v << 16));
  }
  static __device__ __forceinline__ type zero() { return 0u; }
};
template <>
struct Raw<uint16_t, 1> {
  using type = uint32_t;
  static __device__ __forceinline__ type load(const uint16_t *p) {
    return (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(p));
  }
  static __device__ __forceinline__ float get(const type &v, int) {
    return __uint_as_float(v << 16);
  }
  static __device__ __forceinline__ type zero() { return 0u; }
};

// FP64 squared distance in the oracle's order: left to right, each operation
// rounded on its own (explicit _rn intrinsics forbid contraction into FMA).
__device__ __forceinline__ double dist2_fp64(const float *a, const float *b, int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    const double t = __dsub_rn((double)__ldg(a + k), (double)__ldg(b + k));
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}

// ------------------------------------------------------------ union-find

// Every union-find loop below stops after `limit` steps, records the
// overrun in the status word and returns, so a corrupted forest can never
// spin; with the default limit (2^30, above any tree depth for n < 2^31) it
// is never reached.

// Root of x with path halving.  Parent links only ever point to smaller
// indices and only ever move towards the root, so concurrent halving writes
// keep every link an ancestor.  Loads bypass L1 (cg) to see other SMs' links.
__device__ __forceinline__ int32_t uf_find(int32_t *parent, int32_t x, uint32_t *status,
                                           int32_t limit) {
  for (int32_t it = 0; it < limit; ++it) {
    const int32_t p = __ldcg(parent + x);
    if (p == x) return x;
    const int32_t gp = __ldcg(parent + p);
    if (gp != p) parent[x] = gp;
    x = gp;
  }
  atomicOr(status, kErrFindLimit);
  return x;
}

// Read-only root lookup (no writes), used once components are final.
__device__ __forceinline__ int32_t uf_root(const int32_t *parent, int32_t x, uint32_t *status,
                                           int32_t limit) {
  for (int32_t it = 0; it < limit; ++it) {
    const int32_t p = __ldcg(parent + x);
    if (p == x) return x;
    x = p;
  }
  atomicOr(status, kErrFindLimit);
  return x;
}

// Join the components of a and b: the larger root is linked under the
// smaller with a compare-and-swap, so the surviving root of every component
// is its smallest index.  A failed swap means another thread linked that
// root first; retry from the new parent (bounded).
__device__ __forceinline__ void uf_unite(int32_t *parent, int32_t a, int32_t b, uint32_t *status,
                                         int32_t limit) {
  for (int32_t it = 0; it < limit; ++it) {
    a = uf_find(parent, a, status, limit);
    b = uf_find(parent, b, status, limit);
    if (a == b) return;
    const int32_t hi = a > b ? a : b;
    const int32_t lo = a > b ? b : a;
    const int32_t old = atomicCAS(parent + hi, hi, lo);
    if (old == hi) return;
    a = old;
    b = lo;
  }
  atomicOr(status, kErrUnionLimit);
}

constexpr int32_t kLoopLimit = 1 << 30;

// ---------------------------------------------------------- launch count

void note_launch(int count = 1);

}  // namespace sng
