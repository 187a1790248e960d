// Attribute interpolation (sm_103a): a second per-cell field evaluated at the
// vertices of an indexed face set, along the same edges and with the same t
// as the vertex positions (the attribute mapping of the paper's introduction,
// Sec. 1; the vertex formula of Sec. 5).
#include "attributes.h"

namespace amriso {
namespace {

// Per vertex: cells a, b as input indices, taken from the one with the lower
// (z,y,x) corner (as the vertex position is); t = (iso - s_a) / (s_b - s_a)
// and f = f_a + t (f_b - f_a), each operation rounded on its own.
__global__ void __launch_bounds__(256) k_interpolate(const int* __restrict__ xyz, const float* __restrict__ s,
                                                     const float* __restrict__ attr, long long n,
                                                     const int* __restrict__ vkeys, long long nv, float iso,
                                                     float* __restrict__ out, Scratch* sc) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
    int a = __ldg(vkeys + 2 * v), b = __ldg(vkeys + 2 * v + 1);
    if (a < 0 || b < 0 || a >= n || b >= n) {
      atomicOr(&sc->err, (unsigned)ERR_RANGE);   // rare: only on invalid keys
      out[v] = 0.f;
      continue;
    }
    const int az = __ldg(xyz + 3ll * a + 2), ay = __ldg(xyz + 3ll * a + 1), ax = __ldg(xyz + 3ll * a);
    const int bz = __ldg(xyz + 3ll * b + 2), by = __ldg(xyz + 3ll * b + 1), bx = __ldg(xyz + 3ll * b);
    if (bz < az || (bz == az && (by < ay || (by == ay && bx < ax)))) {
      const int tmp = a;
      a = b;
      b = tmp;
    }
    const float sa = __ldg(s + a), sb = __ldg(s + b);
    const float t = __fdiv_rn(__fsub_rn(iso, sa), __fsub_rn(sb, sa));
    const float fa = __ldg(attr + a), fb = __ldg(attr + b);
    out[v] = __fadd_rn(fa, __fmul_rn(t, __fsub_rn(fb, fa)));
  }
}

}  // namespace

cudaError_t launch_interpolate(const int* xyz, const float* s, const float* attr, long long n, const int* vkeys,
                               long long nv, float iso, float* out, Scratch* sc, int grid, cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  k_interpolate<<<grid, 256, 0, st>>>(xyz, s, attr, n, vkeys, nv, iso, out, sc);
  return cudaGetLastError();
}

}  // namespace amriso
