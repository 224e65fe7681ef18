// gather_mma8.cuh -- the screened gather on an FP8 copy with tensor-core dot
// products (gather_mma8.cu).
#pragma once

#include "gather.cuh"

namespace sng {

// Launch over rows a.row_begin .. a.row_end (a.x: the FP8 copy, a.ld its row
// stride in bytes, 32 ks = 64 or 128) with registers budgeted for minb
// resident blocks per SM (0: the default); false if that variant is not
// compiled.
bool launch_gather_mma8(int ks, int minb, const GatherArgs &a, int64_t rows, cudaStream_t st);

}  // namespace sng
