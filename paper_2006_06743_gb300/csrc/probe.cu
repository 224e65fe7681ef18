// probe.cu -- a measurement aid: the read bandwidth from L2 into the SMs.
//
// The gather's tiled and screened forms keep their working set in L2, so
// their roofline is the rate at which the SMs can pull data out of L2, not
// the HBM copy rate.  This kernel measures that rate on the device it runs
// on: a buffer small enough to stay resident in L2 is read over and over
// with 16-byte loads that bypass L1 (ld.global.cg), by every SM, with
// several loads in flight per thread; the bytes read divided by the time
// between two CUDA events is the peak a kernel bound by L2 reads can reach.
#include <cuda_runtime.h>

#include "api_common.cuh"

namespace sng {

constexpr int kProbeLoads = 8;   // independent 16-byte loads in flight per thread

__device__ __forceinline__ uint4 ld_cg_v4(const uint4 *p) {
  uint4 v;
  asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// Every thread reads words tid, tid + T, ... (T = threads in the grid) of
// the buffer, kProbeLoads at a time, `passes` times; each pass starts one
// block further along so that no SM reads the same lines twice in a row.
__global__ void __launch_bounds__(512) l2_read_kernel(const uint4 *buf, int64_t words,
                                                      int32_t passes, unsigned int *sink) {
  const int64_t threads = (int64_t)gridDim.x * blockDim.x;
  uint32_t acc = 0;
  for (int32_t r = 0; r < passes; ++r) {
    const int64_t tid = ((int64_t)((blockIdx.x + r) % gridDim.x)) * blockDim.x + threadIdx.x;
    for (int64_t i = tid; i < words; i += threads * kProbeLoads) {
      uint4 v[kProbeLoads];
#pragma unroll
      for (int k = 0; k < kProbeLoads; ++k) {
        const int64_t j = i + (int64_t)k * threads;
        v[k] = j < words ? ld_cg_v4(buf + j) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int k = 0; k < kProbeLoads; ++k) acc ^= v[k].x ^ v[k].y ^ v[k].z ^ v[k].w;
    }
  }
  // one word per block keeps the loads alive
  if (threadIdx.x == 0) sink[blockIdx.x] = acc;
}

}  // namespace sng

using namespace sng;

extern "C" {

sng_status sng_measure_l2_read(int64_t bytes, int32_t passes, double *gbs, void *stream) {
  if (!gbs) return fail(SNG_EINVAL, "gbs is NULL");
  if (bytes < (1 << 20) || bytes > (int64_t(1) << 30) || passes < 1 || passes > 100000)
    return fail(SNG_EINVAL, "need 1 MiB <= bytes <= 1 GiB and 1 <= passes <= 100000");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int sms = device_sms();
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, l2_read_kernel, 512, 0);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  const int64_t words = bytes / 16;
  uint4 *buf = nullptr;
  unsigned int *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&buf, (size_t)words * 16);
  if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)grid * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0x5a, (size_t)words * 16, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    l2_read_kernel<<<grid, 512, 0, st>>>(buf, words, 2, sink);   // warm L2
    note_launch();
    cudaEventRecord(e0, st);
    l2_read_kernel<<<grid, 512, 0, st>>>(buf, words, passes, sink);
    note_launch();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "L2 read probe");
  *gbs = (double)words * 16.0 * (double)passes / ((double)ms * 1e-3) / 1e9;
  return SNG_OK;
}

}  // extern "C"
