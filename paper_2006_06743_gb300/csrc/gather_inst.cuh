// gather_inst.cuh -- compiled mappings of the gather kernel and their dispatch.
// Each translation unit that includes this defines SNG_GATHER_T / SNG_GATHER_VEC_MAX
// and instantiates the kernel for the (group, chunks, unroll) combinations the
// mapping policy and the autotuner choose from.
#pragma once
#include "gather.cuh"

namespace sng {

// A FULL instantiation serves only maps with m.full; the general one serves
// either.
template <typename T, int VEC, int G, int NCH, int U, bool SIM = false, bool FULL = false>
static bool try_launch(const GatherMap &m, const GatherArgs &args, int grid, cudaStream_t st) {
  if (m.vec != VEC || m.group != G || m.nch != NCH || m.unroll != U || (m.sim != 0) != SIM ||
      (FULL && !m.full))
    return false;
  const size_t smem = (size_t)(m.block / 32) * 64 * U * sizeof(int32_t);
  gather_kernel<T, VEC, G, NCH, U, SIM, FULL><<<grid, m.block, smem, st>>>(args);
  return true;
}

template <typename T, int VEC, int G, int NCH, int U, bool SIM = false, bool FULL = false>
static int occ_blocks(const GatherMap &m) {
  if (m.vec != VEC || m.group != G || m.nch != NCH || m.unroll != U || (m.sim != 0) != SIM ||
      (FULL && !m.full))
    return -1;
  int blocks = 0;
  const size_t smem = (size_t)(m.block / 32) * 64 * U * sizeof(int32_t);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &blocks, gather_kernel<T, VEC, G, NCH, U, SIM, FULL>, m.block, smem) != cudaSuccess)
    return 0;
  return blocks;
}

template <typename T, int VEC, int G, int NCH, int U>
static bool try_launch_blocked(const GatherMap &m, const GatherArgs &args, int grid, int32_t lo,
                               int32_t hi, cudaStream_t st) {
  if (m.vec != VEC || m.group != G || m.nch != NCH || m.unroll != U || m.sim) return false;
  const size_t smem = (size_t)(m.block / 32) * 64 * U * sizeof(int32_t);
  gather_blocked_kernel<T, VEC, G, NCH, U><<<grid, m.block, smem, st>>>(args, lo, hi);
  return true;
}

template <typename T, int VEC, int G, int NCH, int U>
static int occ_blocks_blocked(const GatherMap &m) {
  if (m.vec != VEC || m.group != G || m.nch != NCH || m.unroll != U || m.sim) return -1;
  int blocks = 0;
  const size_t smem = (size_t)(m.block / 32) * 64 * U * sizeof(int32_t);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &blocks, gather_blocked_kernel<T, VEC, G, NCH, U>, m.block, smem) != cudaSuccess)
    return 0;
  return blocks;
}

// L2-blocked mappings: the row widths of the large workloads
#define SNG_BLOCKED_SHAPES(T, V, X)                                                         \
  X(T, V, 8, 1, 4) X(T, V, 16, 1, 4) X(T, V, 16, 1, 8) X(T, V, 32, 1, 4) X(T, V, 16, 2, 4) \
  X(T, V, 32, 2, 4) X(T, V, 2, 4, 2) X(T, V, 4, 4, 2) X(T, V, 8, 4, 2) X(T, V, 16, 4, 2)   \
  X(T, V, 32, 4, 2) X(T, V, 4, 4, 4) X(T, V, 1, 4, 4) X(T, V, 1, 2, 4) X(T, V, 1, 1, 4)

#define SNG_TRY_B(T, V, G, N, U) \
  if (try_launch_blocked<T, V, G, N, U>(map, args, grid, lo, hi, stream)) return true;
#define SNG_OCC_B(T, V, G, N, U)                       \
  {                                                    \
    int b = occ_blocks_blocked<T, V, G, N, U>(map);    \
    if (b >= 0) return b;                              \
  }

// (group, chunks) shapes: thread-per-pair for tiny rows, sub-warp groups for
// medium rows, whole warps (several chunks per lane) for wide rows.
#define SNG_SHAPES_U(T, V, U, X)                                                         \
  X(T, V, 1, 1, U) X(T, V, 2, 1, U) X(T, V, 4, 1, U) X(T, V, 8, 1, U) X(T, V, 16, 1, U) \
  X(T, V, 32, 1, U) X(T, V, 16, 2, U) X(T, V, 32, 2, U) X(T, V, 32, 4, U)                \
  X(T, V, 32, 8, U) X(T, V, 1, 2, U) X(T, V, 1, 4, U) X(T, V, 8, 2, U) X(T, V, 4, 4, U)  \
  X(T, V, 2, 8, U) X(T, V, 4, 2, U) X(T, V, 8, 4, U) X(T, V, 16, 4, U) X(T, V, 4, 8, U)  \
  X(T, V, 2, 4, U)

template <int VEC, int G, int NCH, int U, bool SIM = false>
static bool matches(const GatherMap &m) {
  return m.vec == VEC && m.group == G && m.nch == NCH && m.unroll == U && (m.sim != 0) == SIM;
}
#define SNG_HAS(T, V, G, N, U) \
  if (matches<V, G, N, U>(map)) return true;

#define SNG_TRY(T, V, G, N, U) \
  if (try_launch<T, V, G, N, U>(map, args, grid, stream)) return true;
#define SNG_OCC(T, V, G, N, U)                 \
  {                                            \
    int b = occ_blocks<T, V, G, N, U>(map);    \
    if (b >= 0) return b;                      \
  }

// one lane per source row (group 1, Euclidean form): no shared memory
template <typename T, int VEC, int NCH, int U>
static bool try_launch_lanes(const GatherMap &m, const GatherArgs &args, int grid,
                             cudaStream_t st) {
  if (m.vec != VEC || m.group != 1 || m.nch != NCH || m.unroll != U || m.sim || !m.lanes)
    return false;
  gather_kernel<T, VEC, 1, NCH, U, false, false, true><<<grid, m.block, 0, st>>>(args);
  return true;
}

template <typename T, int VEC, int NCH, int U>
static int occ_blocks_lanes(const GatherMap &m) {
  if (m.vec != VEC || m.group != 1 || m.nch != NCH || m.unroll != U || m.sim || !m.lanes)
    return -1;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &blocks, gather_kernel<T, VEC, 1, NCH, U, false, false, true>, m.block, 0) !=
      cudaSuccess)
    return 0;
  return blocks;
}

#define SNG_LANE_SHAPES(T, V, X) \
  X(T, V, 1, 2) X(T, V, 1, 4) X(T, V, 2, 2) X(T, V, 2, 4) X(T, V, 4, 2) X(T, V, 4, 4)
#define SNG_TRY_L(T, V, N, U) \
  if (try_launch_lanes<T, V, N, U>(map, args, grid, stream)) return true;
#define SNG_OCC_L(T, V, N, U)                        \
  {                                                  \
    int b = occ_blocks_lanes<T, V, N, U>(map);       \
    if (b >= 0) return b;                            \
  }

// full rows (d == group * nch * vec), Euclidean form
#define SNG_TRY_F(T, V, G, N, U) \
  if (try_launch<T, V, G, N, U, false, true>(map, args, grid, stream)) return true;
#define SNG_OCC_F(T, V, G, N, U)                          \
  {                                                       \
    int b = occ_blocks<T, V, G, N, U, false, true>(map);  \
    if (b >= 0) return b;                                 \
  }

// full rows, similarity form
#define SNG_TRY_SF(T, V, G, N, U) \
  if (try_launch<T, V, G, N, U, true, true>(map, args, grid, stream)) return true;
#define SNG_OCC_SF(T, V, G, N, U)                        \
  {                                                      \
    int b = occ_blocks<T, V, G, N, U, true, true>(map);  \
    if (b >= 0) return b;                                \
  }

// similarity form (inner product / cosine)
#define SNG_HAS_S(T, V, G, N, U) \
  if (matches<V, G, N, U, true>(map)) return true;
#define SNG_TRY_S(T, V, G, N, U) \
  if (try_launch<T, V, G, N, U, true>(map, args, grid, stream)) return true;
#define SNG_OCC_S(T, V, G, N, U)                    \
  {                                                 \
    int b = occ_blocks<T, V, G, N, U, true>(map);   \
    if (b >= 0) return b;                           \
  }

}  // namespace sng
