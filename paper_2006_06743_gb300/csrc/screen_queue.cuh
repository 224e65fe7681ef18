// screen_queue.cuh -- deciding the pairs a tensor-core screen queued
// (screen_queue.cu).
#pragma once

#include "gather.cuh"

namespace sng {

// A kept pair into the gather's results: its keep bit, its row's count, the
// degrees.
__device__ __forceinline__ void queue_keep(const GatherArgs &a, int32_t i, int32_t p, uint32_t j,
                                           int32_t wi) {
  atomicOr(a.bitmask + (int64_t)i * a.W + (j >> 5), 1u << (j & 31));
  if (a.out_cnt) atomicAdd(a.out_cnt + i, 1);
  atomicAdd(a.deg + i, wi);
  if (a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) atomicAdd(a.deg + p, wi);
}

// Decide the a.openq entries (as many as *a.openq_cnt, at most a.openq_cap)
// from the FP32 points a.xm and fold the kept ones into a.bitmask,
// a.out_cnt and a.deg; adds the count to the screen counter.  Nothing to do
// without a queue.
sng_status launch_screen_queue(const GatherArgs &a, cudaStream_t st);

}  // namespace sng
