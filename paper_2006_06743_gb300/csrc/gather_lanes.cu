// gather_lanes.cu -- one-lane-per-source-row gather mappings (rows of at
// most 4 vectors: the mappings with one lane per pair), FP32 and BF16, 2 and
// 4 partner rows in flight per lane.
#include "gather_inst.cuh"

namespace sng {

bool launch_lanes_f32(const GatherMap &map, const GatherArgs &args, int grid,
                      cudaStream_t stream) {
  SNG_LANE_SHAPES(float, 4, SNG_TRY_L)
  SNG_LANE_SHAPES(float, 2, SNG_TRY_L)
  SNG_LANE_SHAPES(float, 1, SNG_TRY_L)
  return false;
}

bool launch_lanes_bf16(const GatherMap &map, const GatherArgs &args, int grid,
                       cudaStream_t stream) {
  SNG_LANE_SHAPES(uint16_t, 8, SNG_TRY_L)
  SNG_LANE_SHAPES(uint16_t, 4, SNG_TRY_L)
  SNG_LANE_SHAPES(uint16_t, 2, SNG_TRY_L)
  SNG_LANE_SHAPES(uint16_t, 1, SNG_TRY_L)
  return false;
}

int occ_lanes_f32(const GatherMap &map) {
  SNG_LANE_SHAPES(float, 4, SNG_OCC_L)
  SNG_LANE_SHAPES(float, 2, SNG_OCC_L)
  SNG_LANE_SHAPES(float, 1, SNG_OCC_L)
  return -1;
}

int occ_lanes_bf16(const GatherMap &map) {
  SNG_LANE_SHAPES(uint16_t, 8, SNG_OCC_L)
  SNG_LANE_SHAPES(uint16_t, 4, SNG_OCC_L)
  SNG_LANE_SHAPES(uint16_t, 2, SNG_OCC_L)
  SNG_LANE_SHAPES(uint16_t, 1, SNG_OCC_L)
  return -1;
}

}  // namespace sng
