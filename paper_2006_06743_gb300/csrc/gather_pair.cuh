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

// The same over the BF16 copy a.x (row stride a.ld values, a multiple of 8,
// zero past d) with the copy's error bounds a.nbe / a.err_max and the
// thresholds a.pm_lo, a.pm_hi, a.pm_escale; open pairs to the queue a.openq
// (past its capacity decided from a.xm in the gather).  *kc receives the
// 16-byte chunks of the source row each lane keeps in registers.
sng_status launch_gather_pair16(int metric, const GatherArgs &a, int *kc, cudaStream_t st);

// Decide the queued open pairs from the FP32 points as launch_gather_pair
// would (its group order, guard band a.lo_thr .. a.hi_thr, FP64 recheck) and
// fold the kept ones into a.bitmask, a.out_cnt and a.deg.
sng_status launch_pair_queue(int metric, const GatherArgs &a, cudaStream_t st);

}  // namespace sng
