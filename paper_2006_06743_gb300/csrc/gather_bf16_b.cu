// gather_bf16_b.cu -- compiled BF16 (values widened to FP32) gather mappings: vec 8 x unroll 4, vec 8 x unroll 8.
// (Split across translation units so the library builds in parallel.)
#include "gather_inst.cuh"

namespace sng {

bool launch_bf16_b(const GatherMap &map, const GatherArgs &args, int grid, cudaStream_t stream) {
  SNG_SHAPES_U(uint16_t, 8, 4, SNG_TRY)
  SNG_SHAPES_U(uint16_t, 8, 8, SNG_TRY)
  return false;
}

int occ_bf16_b(const GatherMap &map) {
  SNG_SHAPES_U(uint16_t, 8, 4, SNG_OCC)
  SNG_SHAPES_U(uint16_t, 8, 8, SNG_OCC)
  return -1;
}

bool has_bf16_b(const GatherMap &map) {
  SNG_SHAPES_U(uint16_t, 8, 4, SNG_HAS)
  SNG_SHAPES_U(uint16_t, 8, 8, SNG_HAS)
  return false;
}

}  // namespace sng
