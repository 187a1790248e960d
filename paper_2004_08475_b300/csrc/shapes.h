// Shapes of the dual cells (see shapes.cu). Internal to the library; the C
// ABI is include/amriso.h.
#pragma once

#include <cuda_runtime.h>

namespace amriso {

// counts[d] (may be NULL): the number of distinct cells among dual d's 8
// vertex slots; hist[0..8] (zeroed by the caller) accumulates the counts.
cudaError_t launch_dual_shapes(const uint4* duals, long long nd, unsigned char* counts, unsigned long long* hist,
                               int grid, cudaStream_t st);

}  // namespace amriso
