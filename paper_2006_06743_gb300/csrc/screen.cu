// screen.cu -- the BF16 copy behind the certified screen of FP32 points
// (SNG_FLAG_SCREEN16; Algorithm 1, step 2).
//
// The gather of FP32 points reads d * 4 bytes of every partner row; with the
// screen it reads a BF16 copy (half the bytes, and a point set that fits in
// L2 twice as easily) and decides each pair from it wherever the rounding of
// the copy cannot change the decision (screen_thresholds in gather.cuh).
// This file makes the copy, rounding each value to the nearest BF16, an
// upper bound of every row's Euclidean norm, with the maximum over all rows
// (and, for the tiled form, over each slice of rows), and the squared norm
// of every copied row (for the tensor-core form).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "api_common.cuh"
#include "screen.cuh"

namespace sng {

// Largest bits of non-negative floats (or NaN, whose bits order above +inf,
// so that a NaN norm certifies nothing) over a block, one atomic per block.
__device__ __forceinline__ void block_max_bits(unsigned int v, unsigned int *out) {
  __shared__ unsigned int s_max;
  if (threadIdx.x == 0) s_max = 0u;
  __syncthreads();
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v = max(v, __shfl_xor_sync(kFullMask, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&s_max, v);
  __syncthreads();
  if (threadIdx.x == 0 && s_max) atomicMax(out, s_max);
}

// One warp per row: the BF16 copy (round to nearest even; the padding of
// each copied row up to ldb is zero) and the row's norm bound.  The FP32 sum
// of squares (per-lane fused multiply-adds, then a 5-level butterfly) is
// within (d/32 + 6) 2^-24 relative of the exact one; the correctly rounded
// square root times (1 + 2^-11) is then an upper bound of |x_i| for every
// supported d.  Sums that overflow give +inf (no certificate); values too
// small to square in FP32 are covered by the screen's absolute slack.  The
// same sum over the differences x - bf16(x) (exact in FP32: they are the
// low bits of x) bounds the copy's rounding error |x_i - x_i'|, with 2^-60
// for squares below FP32's range.
__global__ void __launch_bounds__(256) shadow_kernel(const float *x, int64_t ld, int32_t d,
                                                     int64_t n, uint16_t *xb, int64_t ldb,
                                                     float *nrm, float *nb2, float2 *nbe,
                                                     unsigned int *nmax_all) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned int mx = 0u, ex = 0u;
  for (int64_t i = warp; i < n; i += warps) {
    const float *row = x + i * ld;
    uint16_t *out = xb + i * ldb;
    float ss = 0.f, sb = 0.f, se = 0.f;
    for (int64_t k = lane; k < ldb; k += 32) {
      const float v = k < d ? __ldg(row + k) : 0.f;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      out[k] = __bfloat16_as_ushort(h);
      ss = fmaf(v, v, ss);
      const float vb = __bfloat162float(h);
      sb = fmaf(vb, vb, sb);   // the square of a BF16 value is exact in FP32
      const float e = v - vb;
      se = fmaf(e, e, se);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      ss += __shfl_xor_sync(kFullMask, ss, o);
      sb += __shfl_xor_sync(kFullMask, sb, o);
      se += __shfl_xor_sync(kFullMask, se, o);
    }
    const float bound = sqrtf(ss) * (1.f + 0x1p-11f);
    const float err = fmaf(sqrtf(se), 1.f + 0x1p-11f, 0x1p-60f);
    if (lane == 0) {
      nrm[i] = bound;
      nb2[i] = sb;
      nbe[i] = make_float2(sb, err);
    }
    mx = max(mx, __float_as_uint(bound));
    ex = max(ex, __float_as_uint(err));
  }
  block_max_bits(mx, nmax_all);
  block_max_bits(ex, nmax_all + kErrMaxSlot);
}

// Maximum norm bound over each slice of `slice` consecutive rows, into
// nmax[1 + s] (the tiled form's partner slices).
__global__ void __launch_bounds__(256) slice_max_kernel(const float *nrm, int64_t n,
                                                        int64_t slice, int32_t k,
                                                        unsigned int *nmax) {
  for (int s = 0; s < k; ++s) {
    const int64_t lo = (int64_t)s * slice;
    const int64_t hi = lo + slice < n ? lo + slice : n;
    unsigned int mx = 0u;
    for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi;
         i += (int64_t)gridDim.x * blockDim.x)
      mx = max(mx, __float_as_uint(__ldg(nrm + i)));
    block_max_bits(mx, nmax + 1 + s);
  }
}

sng_status make_shadow(const float *x, int64_t ld, int32_t d, int64_t n, int64_t ldb, Scratch &s,
                       Shadow *out) {
  cudaStream_t st = s.stream;
  out->ldb = ldb > 0 ? ldb : ((int64_t)d + 7) / 8 * 8;
  sng_status rc;
  if ((rc = s.alloc((void **)&out->xb, (size_t)n * out->ldb * 2, "BF16 screen copy")) ||
      (rc = s.alloc((void **)&out->nrm, (size_t)n * 4, "row norm bounds")) ||
      (rc = s.alloc((void **)&out->nb2, (size_t)n * 4, "squared norms of the copy")) ||
      (rc = s.alloc((void **)&out->nbe, (size_t)n * 8, "squared norms and errors of the copy")) ||
      (rc = s.alloc((void **)&out->nmax, (size_t)(1 + kErrMaxSlot) * 4, "norm maxima")))
    return rc;
  cudaMemsetAsync(out->nmax, 0, (size_t)(1 + kErrMaxSlot) * 4, st);
  const int64_t blocks_needed = (n + 7) / 8;
  const int64_t cap = (int64_t)device_sms() * 8;
  const int grid = (int)(blocks_needed < cap ? blocks_needed : cap);
  shadow_kernel<<<grid, 256, 0, st>>>(x, ld, d, n, out->xb, out->ldb, out->nrm, out->nb2,
                                      out->nbe, reinterpret_cast<unsigned int *>(out->nmax));
  note_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "BF16 screen copy");
}

// Largest finite |x| over the point set, as float bits, into *amax.
__global__ void __launch_bounds__(256) amax_kernel(const float *x, int64_t ld, int32_t d,
                                                   int64_t n, unsigned int *amax) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned int mx = 0u;
  for (int64_t i = warp; i < n; i += warps)
    for (int64_t k = lane; k < d; k += 32) {
      const float v = fabsf(__ldg(x + i * ld + k));
      if (v <= 3.4028235e38f) mx = max(mx, __float_as_uint(v));   // skips inf and NaN
    }
  block_max_bits(mx, amax);
}

// The copy's scale exponent k from the largest |x|: |x| < 2^e with e the
// exponent of frexp, so 2^(8 - e) puts every scaled value below 256 (E4M3
// reaches 448).  k stays within [-60, 60] so that 2^-2k is a normal FP32
// number; a point set whose largest value needs k < -60 has values above
// 2^68, whose squares overflow FP32, so its norm bounds certify nothing.
__device__ __forceinline__ int32_t fp8_scale_exp(unsigned int amax_bits) {
  const float amax = __uint_as_float(amax_bits);
  if (!(amax > 0.f)) return 0;
  int e;
  frexpf(amax, &e);
  int32_t k = 8 - e;
  return k < -60 ? -60 : k > 60 ? 60 : k;
}

// One warp per row: the E4M3 copy of x * 2^k (round to nearest even), the
// row's norm bound (as the BF16 copy's), the copy's squared norm (the
// squares of E4M3 values are exact in FP32, their FP32 sum is scaled back
// by 2^-2k exactly) and a bound of |x_i - x_i'| with x_i' = copy * 2^-k:
// each difference x - x' is exact where x' is within a factor two of x
// (Sterbenz) and otherwise rounded once, and the FP32 sum of their squares
// is bounded as the norms' sums are, so sqrt of the sum times (1 + 2^-11),
// plus 2^-60 for squares below FP32's range, bounds the rounding error of
// the copy.  A non-finite value makes the bound inf or NaN: no certificate.
__global__ void __launch_bounds__(256) shadow8_kernel(const float *x, int64_t ld, int32_t d,
                                                      int64_t n, uint8_t *xq, int64_t ldb,
                                                      float *nrm, float2 *nbe,
                                                      unsigned int *nmax_all,
                                                      const unsigned int *amax, int32_t *kexp) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t k = fp8_scale_exp(*amax);
  if (blockIdx.x == 0 && threadIdx.x == 0) *kexp = k;
  const float scale = ldexpf(1.f, k), back = ldexpf(1.f, -k), back2 = ldexpf(1.f, -2 * k);
  unsigned int mx = 0u, ex = 0u;
  for (int64_t i = warp; i < n; i += warps) {
    const float *row = x + i * ld;
    uint8_t *out = xq + i * ldb;
    float ss = 0.f, sq = 0.f, se = 0.f;
    for (int64_t c = lane; c < ldb; c += 32) {
      const float v = c < d ? __ldg(row + c) : 0.f;
      const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(v * scale, __NV_SATFINITE, __NV_E4M3);
      out[c] = q;
      ss = fmaf(v, v, ss);
      const __half_raw hr = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
      const float vq = __half2float(__half(hr));
      sq = fmaf(vq, vq, sq);
      const float e = v - vq * back;
      se = fmaf(e, e, se);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      ss += __shfl_xor_sync(kFullMask, ss, o);
      sq += __shfl_xor_sync(kFullMask, sq, o);
      se += __shfl_xor_sync(kFullMask, se, o);
    }
    const float bound = sqrtf(ss) * (1.f + 0x1p-11f);
    const float err = fmaf(sqrtf(se), 1.f + 0x1p-11f, 0x1p-60f);
    if (lane == 0) {
      nrm[i] = bound;
      nbe[i] = make_float2(sq * back2, err);
    }
    mx = max(mx, __float_as_uint(bound));
    ex = max(ex, __float_as_uint(err));
  }
  block_max_bits(mx, nmax_all);
  block_max_bits(ex, nmax_all + kErrMaxSlot);
}

sng_status make_shadow8(const float *x, int64_t ld, int32_t d, int64_t n, int64_t ldb,
                        Scratch &s, Shadow *out) {
  cudaStream_t st = s.stream;
  if (ldb != 64 && ldb != 128) return fail(SNG_EINTERNAL, "FP8 copy rows of %lld bytes",
                                           (long long)ldb);
  out->ldb = ldb;
  sng_status rc;
  unsigned int *amax = nullptr;
  if ((rc = s.alloc((void **)&out->xb, (size_t)n * ldb, "FP8 screen copy")) ||
      (rc = s.alloc((void **)&out->nrm, (size_t)n * 4, "row norm bounds")) ||
      (rc = s.alloc((void **)&out->nbe, (size_t)n * 8, "squared norms and errors of the copy")) ||
      (rc = s.alloc((void **)&out->nmax, (size_t)(1 + kErrMaxSlot) * 4, "norm maxima")) ||
      (rc = s.alloc((void **)&amax, 8, "largest value")))
    return rc;
  out->kexp = reinterpret_cast<int32_t *>(amax) + 1;
  cudaMemsetAsync(out->nmax, 0, (size_t)(1 + kErrMaxSlot) * 4, st);
  cudaMemsetAsync(amax, 0, 4, st);
  const int64_t blocks_needed = (n + 7) / 8;
  const int64_t cap = (int64_t)device_sms() * 8;
  const int grid = (int)(blocks_needed < cap ? blocks_needed : cap);
  amax_kernel<<<grid, 256, 0, st>>>(x, ld, d, n, amax);
  note_launch();
  shadow8_kernel<<<grid, 256, 0, st>>>(x, ld, d, n, reinterpret_cast<uint8_t *>(out->xb), ldb,
                                       out->nrm, out->nbe,
                                       reinterpret_cast<unsigned int *>(out->nmax), amax,
                                       out->kexp);
  note_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "FP8 screen copy");
}

sng_status shadow_slice_max(const Shadow &sh, int64_t n, int64_t slice, int k, cudaStream_t st) {
  if (k < 1 || k > kShadowSlices) return fail(SNG_EINTERNAL, "slice count %d out of range", k);
  const int grid = device_sms();
  slice_max_kernel<<<grid, 256, 0, st>>>(sh.nrm, n, slice, k,
                                         reinterpret_cast<unsigned int *>(sh.nmax));
  note_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "norm maxima per slice");
}

}  // namespace sng
