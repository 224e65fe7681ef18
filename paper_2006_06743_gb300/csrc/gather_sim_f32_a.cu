// gather_sim_f32_a.cu -- compiled FP32 similarity-form gather mappings: vec 4 x unroll 2, vec 4 x unroll 4
// (the default mapping rule's vector widths and unrolls; split across
// translation units so the library builds in parallel).
#include "gather_inst.cuh"

namespace sng {

bool launch_sim_f32_a(const GatherMap &map, const GatherArgs &args, int grid, cudaStream_t stream) {
  SNG_SHAPES_U(float, 4, 2, SNG_TRY_S)
  SNG_SHAPES_U(float, 4, 4, SNG_TRY_S)
  return false;
}

int occ_sim_f32_a(const GatherMap &map) {
  SNG_SHAPES_U(float, 4, 2, SNG_OCC_S)
  SNG_SHAPES_U(float, 4, 4, SNG_OCC_S)
  return -1;
}

bool has_sim_f32_a(const GatherMap &map) {
  SNG_SHAPES_U(float, 4, 2, SNG_HAS_S)
  SNG_SHAPES_U(float, 4, 4, SNG_HAS_S)
  return false;
}

}  // namespace sng
