// gather_pair.cuh -- step 2 with the Manhattan or Chebyshev distance
// (gather_pair.cu).
#pragma once

#include "gather.cuh"

namespace sng {

// Launch over rows a.row_begin .. a.row_end of the FP32 points a.xm (row
// stride a.ldm) for metric SNG_METRIC_L1 or SNG_METRIC_LINF, with the guard
// band a.lo_thr .. a.hi_thr of the FP32 distance; SNG_EINTERNAL for another
// metric.
sng_status launch_gather_pair(int metric, const GatherArgs &a, cudaStream_t st);

}  // namespace sng
