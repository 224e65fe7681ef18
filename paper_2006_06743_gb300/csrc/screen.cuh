// screen.cuh -- the BF16 copy of FP32 points for the certified screen
// (screen.cu; SNG_FLAG_SCREEN16).
#pragma once

#include "api_common.cuh"

namespace sng {

constexpr int kShadowSlices = 32;   // the tiled form's largest slice count
// nmax[kErrMaxSlot]: the largest |x_i - x_i'| bound of the copy
constexpr int kErrMaxSlot = 1 + kShadowSlices;

struct Shadow {
  uint16_t *xb = nullptr;   // n x ldb BF16 bit patterns (ldb = d rounded up to 8)
  int64_t ldb = 0;
  float *nrm = nullptr;     // n: upper bounds of the rows' Euclidean norms
  float *nmax = nullptr;    // [0] max over all rows, [1 + s] over slice s,
                            // [kErrMaxSlot] the largest bound in nbe[].y
  float *nb2 = nullptr;     // n: squared norms of the copied rows (FP32 sums)
  float2 *nbe = nullptr;    // n: {|x_i'|^2, an upper bound of |x_i - x_i'|}
  // FP8 copy (make_shadow8): xb holds n x ldb bytes of E4M3 values of
  // x * 2^k, k = *kexp on the device; nbe in the units of x (nb2 unused)
  int32_t *kexp = nullptr;
};

// BF16 copy (row stride ldb, 0 = d rounded up to 8), norm bounds, their
// maximum, the copy's squared norms, and per row {squared norm, bound of the
// copy's rounding error} with the largest bound (stream-ordered; scratch
// from s).
sng_status make_shadow(const float *x, int64_t ld, int32_t d, int64_t n, int64_t ldb, Scratch &s,
                       Shadow *out);
// FP8 (E4M3) copy of x * 2^k, one power of two k for the whole point set
// (the largest finite |x| times 2^k below 256), rows of ldb = 64 or 128
// bytes (zero past d); norm bounds, their maximum (nmax[0]), and per row the
// copy's squared norm and a bound of its rounding error, in the units of x,
// with the largest error bound in nmax[kErrMaxSlot].
sng_status make_shadow8(const float *x, int64_t ld, int32_t d, int64_t n, int64_t ldb,
                        Scratch &s, Shadow *out);
// Maxima of the norm bounds over k slices of `slice` rows into nmax[1..k].
sng_status shadow_slice_max(const Shadow &sh, int64_t n, int64_t slice, int k, cudaStream_t st);

}  // namespace sng
