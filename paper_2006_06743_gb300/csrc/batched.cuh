// batched.cuh -- structures of the persistent per-cloud kernel (batched.cu).
#pragma once

#include "api_common.cuh"

namespace sng {

struct CloudInfo {
  int64_t off;      // first row of the cloud in x_concat / labels
  int64_t bm_off;   // first keep-bit word of the cloud
  uint64_t seed;    // base seed + cloud index
  FastMod fm;       // remainder constants for n - 1
  int32_t n, m, W, ntiles;
};

struct BatchArgs {
  const float *x;
  int64_t ld;
  int32_t d;
  int32_t n_items;
  int32_t tile_rows;
  int32_t min_pts, deg_mode, sample_all;
  float lo_thr, hi_thr;
  double eps2, band;
  const CloudInfo *clouds;
  const int2 *items;  // (cloud, tile)
  uint32_t *bitmask;
  int32_t *deg;
  int32_t *parent;
  uint8_t *core;
  uint8_t *band_flag;
  int32_t *labels;
  unsigned int *next_item;
  unsigned int *done;
  unsigned long long *counters;
  int32_t loop_limit;   // union-find loop bound
};

struct BatchMap {
  int vec, group, nch, unroll;
  int lanes;   // 1: one lane per source row (rows of one float4)
};

// Launch the persistent kernel for mapping m (occ != NULL: only report the
// resident blocks per SM).  Returns false if the mapping is not compiled.
bool launch_batched_kernel(const BatchMap &m, const BatchArgs &a, int grid, int block,
                           cudaStream_t st, int *occ);

}  // namespace sng
