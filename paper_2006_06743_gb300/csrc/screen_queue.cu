// screen_queue.cu -- the pairs a tensor-core screen left open (Algorithm 1,
// step 2), decided from the FP32 points after the gather.
//
// The FP8 gather (gather_mma8.cu) certifies most pairs from its copy and
// queues the rest as {i, p, draw j, weight of i}.  (Similarity pairs go
// straight to the FP64 recheck, one per thread.)  Deciding them inside the
// gather would stall a whole warp on two FP32 row fetches per open pair;
// here one warp takes one pair, its lanes read the two rows with coalesced
// loads, and the pair is decided as the plain FP32 path decides it: the FP32
// squared distance (per-lane fused multiply-adds, then a five-level tree, so
// its own guard band q_lo_thr / q_hi_thr), and inside that band the FP64
// recheck with its band count.  A kept pair sets its bit in the keep mask
// and adds to the counts and degrees the gather wrote for its row.
#include "api_common.cuh"
#include "gather.cuh"
#include "screen_queue.cuh"

namespace sng {

__global__ void __launch_bounds__(256) screen_queue_kernel(GatherArgs a) {
  const int lane = threadIdx.x & 31;
  const unsigned long long queued = *a.openq_cnt;
  const int64_t total =
      (long long)queued < a.openq_cap ? (int64_t)queued : (int64_t)a.openq_cap;
  if (a.sim_screen) {
    // inner product / cosine: every open pair straight to the FP64 value in
    // the oracle's order (the similarity form's recheck, with its band
    // count), one pair per thread
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t t = t0; t < total; t += (int64_t)gridDim.x * blockDim.x) {
      const uint4 e = a.openq[t];
      if (recheck_sim(a, (int32_t)e.x, (int32_t)e.y))
        queue_keep(a, (int32_t)e.x, (int32_t)e.y, e.z, (int32_t)e.w);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && total > 0)
      atomicAdd(a.counters + kCntScreen, (unsigned long long)total);
    return;
  }
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = warp; t < total; t += warps) {
    const uint4 e = a.openq[t];
    const int32_t i = (int32_t)e.x, p = (int32_t)e.y, wi = (int32_t)e.w;
    const uint32_t j = e.z;
    const float *xa = a.xm + (int64_t)i * a.ldm, *xb = a.xm + (int64_t)p * a.ldm;
    float acc = 0.f;
    for (int k = lane; k < a.d; k += 32) {
      const float u = __ldg(xa + k) - __ldg(xb + k);
      acc = fmaf(u, u, acc);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_down_sync(kFullMask, acc, o);
    if (lane == 0) {
      const bool keep =
          acc < a.q_lo_thr ? true : acc > a.q_hi_thr ? false : recheck_pair<float>(a, i, p);
      if (keep) queue_keep(a, i, p, j, wi);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && total > 0)
    atomicAdd(a.counters + kCntScreen, (unsigned long long)total);
}

sng_status launch_screen_queue(const GatherArgs &a, cudaStream_t st) {
  if (!a.openq || a.openq_cap <= 0) return SNG_OK;
  const int grid = device_sms() * 8;
  screen_queue_kernel<<<grid, 256, 0, st>>>(a);
  note_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "open-pair queue");
}

}  // namespace sng
