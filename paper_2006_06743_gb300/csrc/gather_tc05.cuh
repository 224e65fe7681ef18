// gather_tc05.cuh -- the screened gather with TMA row gathers and tcgen05
// dot products (gather_tc05.cu).
#pragma once

#include "gather.cuh"

namespace sng {

// Ring stages when map_unroll is 0.
constexpr int kTc05DefaultStages = 2;

// Launch over rows a.row_begin .. a.row_end of the BF16 copy a.x (n rows of
// ldb = 64 values) with a ring of `stages` shared-memory stages (2..5; 0:
// the default), the count used stored in *used; SNG_EINVAL for other row
// widths or stage counts, SNG_ECUDA if the tensor map cannot be made.
sng_status launch_gather_tc05(const GatherArgs &a, int64_t n, int64_t ldb, int stages,
                              int *used, cudaStream_t st);

}  // namespace sng
