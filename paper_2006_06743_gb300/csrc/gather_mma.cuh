// gather_mma.cuh -- the screened gather with tensor-core dot products
// (gather_mma.cu).
#pragma once

#include "gather.cuh"

namespace sng {

// k-tiles of 16 BF16 values per row for d (0: d > 128, not compiled); the
// BF16 copy's rows are then 16 * tiles values wide.
int mma_tiles_for(int d);
// Launch over rows a.row_begin .. a.row_end (a.x: the BF16 copy, a.ld its
// row stride = 16 * kt) with registers budgeted for minb resident blocks per
// SM (0: the default); false if that variant is not compiled.
bool launch_gather_mma(int kt, int minb, const GatherArgs &a, int64_t rows, cudaStream_t st);

}  // namespace sng
