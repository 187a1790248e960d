// Shapes of the dual cells (sm_103a): snapping turns a dual hexahedron into
// a wedge, pyramid, tetrahedron or a flatter shape when some of its 8
// vertices resolve to the same cell (Sec. 4.1, Sec. 5). The number of
// distinct cells among the 8 vertices classifies it: 8 hexahedron, 6 wedge,
// 5 pyramid, 4 tetrahedron.
#include "shapes.h"

namespace amriso {
namespace {

constexpr unsigned kDistinctFlag = 0x80000000u;   // bit 31 of a dual's first slot: 8 different cells

__global__ void __launch_bounds__(256) k_dual_shapes(const uint4* __restrict__ duals, long long nd,
                                                     unsigned char* __restrict__ counts,
                                                     unsigned long long* __restrict__ hist) {
  __shared__ unsigned h_sh[9];
  if (threadIdx.x < 9) h_sh[threadIdx.x] = 0;
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x; d < nd; d += stride) {
    const uint4 a = __ldcs(duals + 2 * d), b = __ldcs(duals + 2 * d + 1);
    int k = 8;
    if (!(a.x & kDistinctFlag)) {
      const unsigned v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      k = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        bool seen = false;
#pragma unroll
        for (int f = 0; f < e; ++f) seen = seen || v[f] == v[e];
        k += seen ? 0 : 1;
      }
    }
    if (counts) counts[d] = (unsigned char)k;
    atomicAdd(&h_sh[k], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 9 && h_sh[threadIdx.x]) atomicAdd(hist + threadIdx.x, (unsigned long long)h_sh[threadIdx.x]);
}

}  // namespace

cudaError_t launch_dual_shapes(const uint4* duals, long long nd, unsigned char* counts, unsigned long long* hist,
                               int grid, cudaStream_t st) {
  if (nd <= 0) return cudaSuccess;
  k_dual_shapes<<<grid, 256, 0, st>>>(duals, nd, counts, hist);
  return cudaGetLastError();
}

}  // namespace amriso
