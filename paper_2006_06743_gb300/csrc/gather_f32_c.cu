// gather_f32_c.cu -- compiled FP32 gather mappings: vec 2 x unroll 4, vec 1 x unroll 4.
// (Split across translation units so the library builds in parallel.)
#include "gather_inst.cuh"

namespace sng {

bool launch_f32_c(const GatherMap &map, const GatherArgs &args, int grid, cudaStream_t stream) {
  SNG_SHAPES_U(float, 2, 4, SNG_TRY)
  SNG_SHAPES_U(float, 1, 4, SNG_TRY)
  return false;
}

int occ_f32_c(const GatherMap &map) {
  SNG_SHAPES_U(float, 2, 4, SNG_OCC)
  SNG_SHAPES_U(float, 1, 4, SNG_OCC)
  return -1;
}

bool launch_gather_blocked_f32(const GatherMap &map, const GatherArgs &args, int grid,
                               int32_t lo, int32_t hi, cudaStream_t stream) {
  SNG_BLOCKED_SHAPES(float, 4, SNG_TRY_B)
  return false;
}

int occ_gather_blocked_f32(const GatherMap &map) {
  SNG_BLOCKED_SHAPES(float, 4, SNG_OCC_B)
  return 0;
}

bool has_f32_c(const GatherMap &map) {
  SNG_SHAPES_U(float, 2, 4, SNG_HAS)
  SNG_SHAPES_U(float, 1, 4, SNG_HAS)
  return false;
}

bool has_gather_blocked_f32(const GatherMap &map) {
  SNG_BLOCKED_SHAPES(float, 4, SNG_HAS)
  return false;
}

}  // namespace sng
