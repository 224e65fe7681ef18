// misc.cu -- gather dispatch, partner materialisation and the ARI.
#include "api_common.cuh"

namespace sng {

#define SNG_UNIT(tag)                                                      \
  bool launch_##tag(const GatherMap &, const GatherArgs &, int, cudaStream_t); \
  int occ_##tag(const GatherMap &);
SNG_UNIT(f32_a) SNG_UNIT(f32_b) SNG_UNIT(f32_c) SNG_UNIT(bf16_a) SNG_UNIT(bf16_b) SNG_UNIT(bf16_c)
#undef SNG_UNIT
bool has_f32_a(const GatherMap &);
bool has_f32_b(const GatherMap &);
bool has_f32_c(const GatherMap &);
bool has_bf16_a(const GatherMap &);
bool has_bf16_b(const GatherMap &);
bool has_bf16_c(const GatherMap &);
bool has_gather_blocked_f32(const GatherMap &);
bool has_gather_blocked_bf16(const GatherMap &);

bool gather_is_compiled(int dtype, const GatherMap &map) {
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
  if (dtype == SNG_F32)
    return launch_f32_a(map, args, grid, stream) || launch_f32_b(map, args, grid, stream) ||
           launch_f32_c(map, args, grid, stream);
  return launch_bf16_a(map, args, grid, stream) || launch_bf16_b(map, args, grid, stream) ||
         launch_bf16_c(map, args, grid, stream);
}

int gather_max_blocks_per_sm(int dtype, const GatherMap &map) {
  int b;
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

// ------------------------------------------------------------------ ARI

// Open-addressing table of (a, b) label pairs -> count, plus per-label
// counts of a and b (labels are in [-1, n), indexed by label + 1).
__global__ void ari_count_kernel(const int32_t *a, const int32_t *b, int64_t n,
                                 unsigned long long *keys, unsigned long long *cnt,
                                 uint64_t cap_mask, unsigned long long *ca,
                                 unsigned long long *cb, unsigned long long *counters) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t *status = reinterpret_cast<uint32_t *>(counters + kCntStatus);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t la = (int64_t)a[i] + 1, lb = (int64_t)b[i] + 1;
    if (la < 0 || la > n || lb < 0 || lb > n) {
      atomicOr(status, kErrIndex);
      continue;
    }
    atomicAdd(ca + la, 1ull);
    atomicAdd(cb + lb, 1ull);
    const unsigned long long key = ((unsigned long long)la << 32) | (unsigned long long)lb;
    uint64_t h = mix64(key) & cap_mask;
    bool done = false;
    for (uint64_t probe = 0; probe <= cap_mask; ++probe) {
      const unsigned long long old = atomicCAS(keys + h, ~0ull, key);
      if (old == ~0ull || old == key) {
        atomicAdd(cnt + h, 1ull);
        done = true;
        break;
      }
      h = (h + 1) & cap_mask;
    }
    if (!done) atomicOr(status, kErrIndex);
  }
}

// sum over entries of c*(c-1)/2 for three count arrays
__global__ void ari_pairs_kernel(const unsigned long long *cnt, int64_t len,
                                 unsigned long long *out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
    const unsigned long long c = cnt[i];
    s += c * (c - (c ? 1ull : 0ull)) / 2ull;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(kFullMask, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
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

sng_status sng_ari(const int32_t *a, const int32_t *b, int64_t n, double *ari, void *stream) {
  if (!a || !b || !ari) return fail(SNG_EINVAL, "NULL argument");
  if (n < 0 || n > 0x7fffffffLL) return fail(SNG_EINVAL, "n out of range");
  if (n < 2) {
    *ari = 1.0;
    return SNG_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s(st);
  uint64_t cap = 1;
  while (cap < (uint64_t)(2 * n)) cap <<= 1;
  unsigned long long *keys, *cnt, *ca, *cb, *counters;
  sng_status rc;
  if ((rc = s.alloc((void **)&keys, cap * 8, "ari keys")) ||
      (rc = s.alloc((void **)&cnt, cap * 8, "ari counts")) ||
      (rc = s.alloc((void **)&ca, (size_t)(n + 1) * 8, "ari a")) ||
      (rc = s.alloc((void **)&cb, (size_t)(n + 1) * 8, "ari b")) ||
      (rc = s.alloc((void **)&counters, kCntSlots * 8, "ari sums")))
    return rc;
  cudaMemsetAsync(keys, 0xff, cap * 8, st);
  cudaMemsetAsync(cnt, 0, cap * 8, st);
  cudaMemsetAsync(ca, 0, (size_t)(n + 1) * 8, st);
  cudaMemsetAsync(cb, 0, (size_t)(n + 1) * 8, st);
  cudaMemsetAsync(counters, 0, kCntSlots * 8, st);
  const int sms = device_sms();
  ari_count_kernel<<<sms * 8, 256, 0, st>>>(a, b, n, keys, cnt, cap - 1, ca, cb, counters);
  ari_pairs_kernel<<<sms * 8, 256, 0, st>>>(cnt, (int64_t)cap, counters + 0);
  ari_pairs_kernel<<<sms * 8, 256, 0, st>>>(ca, n + 1, counters + 1);
  ari_pairs_kernel<<<sms * 8, 256, 0, st>>>(cb, n + 1, counters + 2);
  note_launch(4);
  unsigned long long h[kCntSlots];
  cudaError_t e = cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ari");
  if ((uint32_t)h[kCntStatus]) return fail(SNG_EINVAL, "labels outside [-1, n)");
  const double index = (double)h[0], sa = (double)h[1], sb = (double)h[2];
  const double total = (double)n * (double)(n - 1) / 2.0;
  const double expected = sa * sb / total;
  const double maxi = 0.5 * (sa + sb);
  *ari = (maxi == expected) ? 1.0 : (index - expected) / (maxi - expected);
  return SNG_OK;
}

}  // extern "C"
