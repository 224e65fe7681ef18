// gather_f32_a.cu -- compiled FP32 gather mappings: vec 4 x unroll 1, vec 4 x unroll 2.
// (Split across translation units so the library builds in parallel.)
#include "gather_inst.cuh"

namespace sng {

bool launch_f32_a(const GatherMap &map, const GatherArgs &args, int grid, cudaStream_t stream) {
  SNG_SHAPES_U(float, 4, 1, SNG_TRY)
  SNG_SHAPES_U(float, 4, 2, SNG_TRY)
  return false;
}

int occ_f32_a(const GatherMap &map) {
  SNG_SHAPES_U(float, 4, 1, SNG_OCC)
  SNG_SHAPES_U(float, 4, 2, SNG_OCC)
  return -1;
}

bool has_f32_a(const GatherMap &map) {
  SNG_SHAPES_U(float, 4, 1, SNG_HAS)
  SNG_SHAPES_U(float, 4, 2, SNG_HAS)
  return false;
}

}  // namespace sng
