// gather_full_f32.cu -- FP32 gather mappings for rows exactly group * nch * vec wide
// (16-byte vectors, unroll 2 and 4: the default rule's choices for such
// widths), without per-chunk bounds tests.  The general instantiations serve
// every other row width.
#include "gather_inst.cuh"

namespace sng {

bool launch_full_f32(const GatherMap &map, const GatherArgs &args, int grid, cudaStream_t stream) {
  SNG_SHAPES_U(float, 4, 2, SNG_TRY_F)
  SNG_SHAPES_U(float, 4, 4, SNG_TRY_F)
  return false;
}

int occ_full_f32(const GatherMap &map) {
  SNG_SHAPES_U(float, 4, 2, SNG_OCC_F)
  SNG_SHAPES_U(float, 4, 4, SNG_OCC_F)
  return -1;
}

}  // namespace sng
