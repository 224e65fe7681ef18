// gather_full_sim_bf16.cu -- BF16 similarity-form gather mappings for rows exactly
// group * nch * vec wide, without per-chunk bounds tests.
#include "gather_inst.cuh"

namespace sng {

bool launch_full_sim_bf16(const GatherMap &map, const GatherArgs &args, int grid, cudaStream_t stream) {
  SNG_SHAPES_U(uint16_t, 8, 2, SNG_TRY_SF)
  SNG_SHAPES_U(uint16_t, 8, 4, SNG_TRY_SF)
  return false;
}

int occ_full_sim_bf16(const GatherMap &map) {
  SNG_SHAPES_U(uint16_t, 8, 2, SNG_OCC_SF)
  SNG_SHAPES_U(uint16_t, 8, 4, SNG_OCC_SF)
  return -1;
}

}  // namespace sng
