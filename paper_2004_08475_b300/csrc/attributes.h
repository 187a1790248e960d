// Attribute interpolation at the vertices of an indexed face set (see
// attributes.cu). Internal to the library; the C ABI is include/amriso.h.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace amriso {

// out[v]: the per-cell field attr interpolated between the input cells
// vkeys[v][0..1] along the same t as the vertex position at iso; a cell
// index outside [0, n) sets ERR_RANGE in sc->err (and gives 0).
cudaError_t launch_interpolate(const int* xyz, const float* s, const float* attr, long long n, const int* vkeys,
                               long long nv, float iso, float* out, Scratch* sc, int grid, cudaStream_t st);

}  // namespace amriso
