// screen_queue.cuh -- deciding the pairs a tensor-core screen queued
// (screen_queue.cu).
#pragma once

#include "gather.cuh"

namespace sng {

// Decide the a.openq entries (as many as *a.openq_cnt, at most a.openq_cap)
// from the FP32 points a.xm and fold the kept ones into a.bitmask,
// a.out_cnt and a.deg; adds the count to the screen counter.  Nothing to do
// without a queue.
sng_status launch_screen_queue(const GatherArgs &a, cudaStream_t st);

}  // namespace sng
