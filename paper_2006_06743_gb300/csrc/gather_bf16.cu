// gather_bf16.cu -- BF16 gather mappings (8 x bf16 = 16-byte loads, narrower
// for unaligned rows); values are widened to FP32 before the arithmetic.
#include "gather_inst.cuh"

namespace sng {

bool launch_gather_bf16(const GatherMap &map, const GatherArgs &args, int grid,
                        cudaStream_t stream) {
  SNG_SHAPES_U(uint16_t, 8, 2, SNG_TRY)
  SNG_SHAPES_U(uint16_t, 8, 4, SNG_TRY)
  SNG_SHAPES_U(uint16_t, 8, 8, SNG_TRY)
  SNG_SHAPES_U(uint16_t, 4, 4, SNG_TRY)
  SNG_SHAPES_U(uint16_t, 2, 4, SNG_TRY)
  SNG_SHAPES_U(uint16_t, 1, 4, SNG_TRY)
  return false;
}

int occ_gather_bf16(const GatherMap &map) {
  SNG_SHAPES_U(uint16_t, 8, 2, SNG_OCC)
  SNG_SHAPES_U(uint16_t, 8, 4, SNG_OCC)
  SNG_SHAPES_U(uint16_t, 8, 8, SNG_OCC)
  SNG_SHAPES_U(uint16_t, 4, 4, SNG_OCC)
  SNG_SHAPES_U(uint16_t, 2, 4, SNG_OCC)
  SNG_SHAPES_U(uint16_t, 1, 4, SNG_OCC)
  return 0;
}

bool launch_gather_blocked_bf16(const GatherMap &map, const GatherArgs &args, int grid,
                                int32_t lo, int32_t hi, cudaStream_t stream) {
  SNG_BLOCKED_SHAPES(uint16_t, 8, SNG_TRY_B)
  return false;
}

int occ_gather_blocked_bf16(const GatherMap &map) {
  SNG_BLOCKED_SHAPES(uint16_t, 8, SNG_OCC_B)
  return 0;
}

}  // namespace sng
