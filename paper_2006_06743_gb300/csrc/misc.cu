// misc.cu -- gather dispatch and partner materialisation.
#include "api_common.cuh"

namespace sng {

#define SNG_UNIT(tag)                                                      \
  bool launch_##tag(const GatherMap &, const GatherArgs &, int, cudaStream_t); \
  int occ_##tag(const GatherMap &);
SNG_UNIT(f32_a) SNG_UNIT(f32_b) SNG_UNIT(f32_c) SNG_UNIT(bf16_a) SNG_UNIT(bf16_b) SNG_UNIT(bf16_c)
SNG_UNIT(sim_f32_a) SNG_UNIT(sim_f32_b) SNG_UNIT(sim_bf16_a) SNG_UNIT(sim_bf16_b)
SNG_UNIT(full_f32) SNG_UNIT(full_bf16) SNG_UNIT(full_sim_f32) SNG_UNIT(full_sim_bf16)
SNG_UNIT(lanes_f32) SNG_UNIT(lanes_bf16)
#undef SNG_UNIT
bool has_sim_f32_a(const GatherMap &);
bool has_sim_f32_b(const GatherMap &);
bool has_sim_bf16_a(const GatherMap &);
bool has_sim_bf16_b(const GatherMap &);
bool has_f32_a(const GatherMap &);
bool has_f32_b(const GatherMap &);
bool has_f32_c(const GatherMap &);
bool has_bf16_a(const GatherMap &);
bool has_bf16_b(const GatherMap &);
bool has_bf16_c(const GatherMap &);
bool has_gather_blocked_f32(const GatherMap &);
bool has_gather_blocked_bf16(const GatherMap &);

bool gather_is_compiled(int dtype, const GatherMap &map) {
  if (map.sim) {
    if (dtype == SNG_F32) return has_sim_f32_a(map) || has_sim_f32_b(map);
    return has_sim_bf16_a(map) || has_sim_bf16_b(map);
  }
  if (dtype == SNG_F32) return has_f32_a(map) || has_f32_b(map) || has_f32_c(map);
  return has_bf16_a(map) || has_bf16_b(map) || has_bf16_c(map);
}

bool gather_blocked_is_compiled(int dtype, const GatherMap &map) {
  return dtype == SNG_F32 ? has_gather_blocked_f32(map) : has_gather_blocked_bf16(map);
}
bool launch_gather_blocked_f32(const GatherMap &, const GatherArgs &, int, int32_t, int32_t,
                               cudaStream_t);
bool launch_gather_blocked_bf16(const GatherMap &, const GatherArgs &, int, int32_t, int32_t,
                                cudaStream_t);
int occ_gather_blocked_f32(const GatherMap &);
int occ_gather_blocked_bf16(const GatherMap &);

bool launch_gather(int dtype, const GatherMap &map, const GatherArgs &args, int grid,
                   cudaStream_t stream) {
  if (map.sim) {
    if (map.full && (dtype == SNG_F32 ? launch_full_sim_f32(map, args, grid, stream)
                                       : launch_full_sim_bf16(map, args, grid, stream)))
      return true;
    if (dtype == SNG_F32)
      return launch_sim_f32_a(map, args, grid, stream) || launch_sim_f32_b(map, args, grid, stream);
    return launch_sim_bf16_a(map, args, grid, stream) || launch_sim_bf16_b(map, args, grid, stream);
  }
  if (map.lanes && (dtype == SNG_F32 ? launch_lanes_f32(map, args, grid, stream)
                                      : launch_lanes_bf16(map, args, grid, stream)))
    return true;
  if (map.full && (dtype == SNG_F32 ? launch_full_f32(map, args, grid, stream)
                                     : launch_full_bf16(map, args, grid, stream)))
    return true;
  if (dtype == SNG_F32)
    return launch_f32_a(map, args, grid, stream) || launch_f32_b(map, args, grid, stream) ||
           launch_f32_c(map, args, grid, stream);
  return launch_bf16_a(map, args, grid, stream) || launch_bf16_b(map, args, grid, stream) ||
         launch_bf16_c(map, args, grid, stream);
}

int gather_max_blocks_per_sm(int dtype, const GatherMap &map) {
  int b;
  if (map.sim) {
    if (map.full &&
        (b = dtype == SNG_F32 ? occ_full_sim_f32(map) : occ_full_sim_bf16(map)) >= 0)
      return b;
    if (dtype == SNG_F32) {
      if ((b = occ_sim_f32_a(map)) >= 0 || (b = occ_sim_f32_b(map)) >= 0) return b;
    } else {
      if ((b = occ_sim_bf16_a(map)) >= 0 || (b = occ_sim_bf16_b(map)) >= 0) return b;
    }
    return 0;
  }
  if (map.lanes && (b = dtype == SNG_F32 ? occ_lanes_f32(map) : occ_lanes_bf16(map)) >= 0)
    return b;
  if (map.full && (b = dtype == SNG_F32 ? occ_full_f32(map) : occ_full_bf16(map)) >= 0) return b;
  if (dtype == SNG_F32) {
    if ((b = occ_f32_a(map)) >= 0 || (b = occ_f32_b(map)) >= 0 || (b = occ_f32_c(map)) >= 0)
      return b;
  } else {
    if ((b = occ_bf16_a(map)) >= 0 || (b = occ_bf16_b(map)) >= 0 || (b = occ_bf16_c(map)) >= 0)
      return b;
  }
  return 0;
}

bool launch_gather_blocked(int dtype, const GatherMap &map, const GatherArgs &args, int grid,
                           int32_t lo, int32_t hi, cudaStream_t stream) {
  return dtype == SNG_F32 ? launch_gather_blocked_f32(map, args, grid, lo, hi, stream)
                          : launch_gather_blocked_bf16(map, args, grid, lo, hi, stream);
}

int gather_blocked_max_blocks_per_sm(int dtype, const GatherMap &map) {
  return dtype == SNG_F32 ? occ_gather_blocked_f32(map) : occ_gather_blocked_bf16(map);
}

size_t gather_smem_bytes(const GatherMap &map) {
  return (size_t)(map.block / 32) * 64 * map.unroll * sizeof(int32_t);
}

// ------------------------------------------------------------ partners

__global__ void partners_kernel(int64_t n, uint64_t seed, int64_t i0, int64_t rows, int64_t m,
                                int32_t sample_all, FastMod fm, int32_t *out) {
  const int64_t total = rows * m;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t r = t / m, j = t - r * m;
    const int32_t i = (int32_t)(i0 + r);
    out[t] = sample_all ? partner_all(i, j) : partner_from_key(row_key(seed, i), i, j, fm);
  }
}

}  // namespace sng

using namespace sng;

extern "C" {

sng_status sng_sample_partners(int64_t n, uint64_t seed, int64_t i0, int64_t rows, int64_t m,
                               int32_t sample_mode, int32_t *out, void *stream) {
  if (n < 2 || n > 0x7fffffffLL) return fail(SNG_EINVAL, "n must be in [2, 2^31-1]");
  if (rows < 0 || i0 < 0 || i0 + rows > n) return fail(SNG_EINVAL, "rows out of range");
  if (m < 0 || (sample_mode == SNG_SAMPLE_ALL && m > n - 1))
    return fail(SNG_EINVAL, "bad m");
  if (!out && rows * m > 0) return fail(SNG_EINVAL, "out is NULL");
  if (rows * m == 0) return SNG_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int sms = device_sms();
  int64_t blocks = (rows * m + 255) / 256;
  if (blocks > sms * 32) blocks = sms * 32;
  partners_kernel<<<(int)blocks, 256, 0, st>>>(n, seed, i0, rows, m,
                                               sample_mode == SNG_SAMPLE_ALL, make_fastmod(n),
                                               out);
  note_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "partners launch");
}

}  // extern "C"
