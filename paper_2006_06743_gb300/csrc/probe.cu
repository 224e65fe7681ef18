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

// Random rows (the tensor-core gather's access pattern without its work):
// each warp takes stages of 32 rows, one 32-bit xorshift index per lane,
// and four lanes read each row in RB / 4-byte pieces with 32-byte (or
// 16-byte) loads that bypass L1, eight rows per load instruction -- the
// load layout of gather_mma_kernel -- folding the words into a checksum.
template <int RB>
__global__ void __launch_bounds__(256) random_rows_kernel(const uint8_t *buf, uint32_t n_rows,
                                                          int64_t stages, uint32_t seed,
                                                          unsigned int *sink) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint32_t h = (seed ^ (wid * 0x9E3779B9u) ^ ((uint32_t)lane * 0x85EBCA6Bu)) | 1u;
  uint32_t acc = 0;
  for (int64_t s = 0; s < stages; ++s) {
    h ^= h << 13;
    h ^= h >> 17;
    h ^= h << 5;
    const uint32_t r = __umulhi(h, n_rows);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t rt = __shfl_sync(0xffffffffu, r, 8 * t + g);
      const uint8_t *row = buf + (int64_t)rt * RB + q * (RB / 4);
      if constexpr (RB == 64) {
        uint4 v;
        asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(row));
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
      } else {
#pragma unroll
        for (int k = 0; k < RB / 128; ++k) {
          uint32_t w[8];
          asm volatile("ld.global.cg.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                       : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]),
                         "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                       : "l"(row + 32 * k));
          acc ^= w[0] ^ w[1] ^ w[2] ^ w[3] ^ w[4] ^ w[5] ^ w[6] ^ w[7];
        }
      }
    }
  }
  if (lane == 0) sink[wid] = acc;
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

sng_status sng_measure_random_rows(int64_t n_rows, int32_t row_bytes, int64_t fetches,
                                   int32_t blocks_per_sm, double *rows_per_s, void *stream) {
  if (!rows_per_s) return fail(SNG_EINVAL, "rows_per_s is NULL");
  if (row_bytes != 64 && row_bytes != 128 && row_bytes != 256)
    return fail(SNG_EINVAL, "row_bytes must be 64, 128 or 256");
  if (n_rows < 1024 || n_rows > (int64_t)1 << 31 || n_rows * row_bytes > (int64_t)1 << 33)
    return fail(SNG_EINVAL, "need 1024 <= n_rows <= 2^31 and at most 8 GiB of rows");
  if (fetches < (1 << 20) || fetches > (int64_t)1 << 40)
    return fail(SNG_EINVAL, "need 2^20 <= fetches <= 2^40");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int sms = device_sms();
  int per_sm = 0;
  const void *k64 = (const void *)random_rows_kernel<64>;
  const void *k128 = (const void *)random_rows_kernel<128>;
  const void *k256 = (const void *)random_rows_kernel<256>;
  const void *kern = row_bytes == 64 ? k64 : row_bytes == 128 ? k128 : k256;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
  if (per_sm < 1) per_sm = 1;
  if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
  const int grid = sms * per_sm;
  const int64_t warps = (int64_t)grid * 8;
  const int64_t stages = (fetches + 32 * warps - 1) / (32 * warps);
  uint8_t *buf = nullptr;
  unsigned int *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&buf, (size_t)(n_rows * row_bytes));
  if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)warps * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0x5a, (size_t)(n_rows * row_bytes), st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto launch = [&](int64_t stg, uint32_t seed) {
    if (row_bytes == 64)
      random_rows_kernel<64><<<grid, 256, 0, st>>>(buf, (uint32_t)n_rows, stg, seed, sink);
    else if (row_bytes == 128)
      random_rows_kernel<128><<<grid, 256, 0, st>>>(buf, (uint32_t)n_rows, stg, seed, sink);
    else
      random_rows_kernel<256><<<grid, 256, 0, st>>>(buf, (uint32_t)n_rows, stg, seed, sink);
    note_launch();
  };
  if (e == cudaSuccess) {
    launch(stages > 4 ? stages / 4 : 1, 7u);   // warm-up
    cudaEventRecord(e0, st);
    launch(stages, 12345u);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "random-row probe");
  *rows_per_s = (double)(32 * warps) * (double)stages / ((double)ms * 1e-3);
  return SNG_OK;
}

}  // extern "C"
