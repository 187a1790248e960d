// Spatial processing order of the bricks: a counting sort of the bricks by
// the Morton index of the bucket that holds their lower corner.
#include "order.h"

namespace amriso {
namespace {

// Bits 0..4 of v moved to bits 0, 3, 6, 9, 12.
__device__ __forceinline__ unsigned spread5(unsigned v) {
  v &= 31u;
  v = (v | (v << 8)) & 0x0000F00Fu;
  v = (v | (v << 4)) & 0x000C30C3u;
  v = (v | (v << 2)) & 0x00009249u;
  return v;
}

__device__ __forceinline__ unsigned bucket_of(const int4 b, const OrderFrame& f) {
  const int c[3] = {b.x, b.y, b.z};
  unsigned code = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int r = (c[a] - f.lo[a]) >> f.shift;   // arithmetic shift: below lo stays negative
    code |= spread5((unsigned)min(max(r, 0), (1 << kOrderAxisBits) - 1)) << a;
  }
  return code;
}

__global__ void __launch_bounds__(256) k_order_count(const int4* __restrict__ bricks, long long n, OrderFrame f,
                                                     unsigned* __restrict__ count) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    atomicAdd(count + bucket_of(__ldg(bricks + i), f), 1u);
}

// One CTA of 1024 threads; each thread owns 32 consecutive counters.
constexpr int kScanThreads = 1024;
constexpr int kPerScanThread = kOrderBuckets / kScanThreads;
static_assert(kPerScanThread % 4 == 0, "counters are read as uint4");

__global__ void __launch_bounds__(kScanThreads) k_order_scan(unsigned* __restrict__ count) {
  __shared__ unsigned wsum[kScanThreads / 32];
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  uint4* mine = reinterpret_cast<uint4*>(count) + t * (kPerScanThread / 4);
  uint4 v[kPerScanThread / 4];
  unsigned sum = 0;
#pragma unroll
  for (int k = 0; k < kPerScanThread / 4; ++k) {
    v[k] = mine[k];
    sum += v[k].x + v[k].y + v[k].z + v[k].w;
  }
  unsigned incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[wp] = incl;
  __syncthreads();
  if (wp == 0) {
    const unsigned w = wsum[lane];
    unsigned wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += y;
    }
    wsum[lane] = wi - w;
  }
  __syncthreads();
  unsigned run = wsum[wp] + incl - sum;
#pragma unroll
  for (int k = 0; k < kPerScanThread / 4; ++k) {
    uint4 o;
    o.x = run; run += v[k].x;
    o.y = run; run += v[k].y;
    o.z = run; run += v[k].z;
    o.w = run; run += v[k].w;
    mine[k] = o;
  }
}

__global__ void __launch_bounds__(256) k_order_scatter(const int4* __restrict__ bricks, long long n, OrderFrame f,
                                                       unsigned* __restrict__ offset, int* __restrict__ order) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    order[atomicAdd(offset + bucket_of(__ldg(bricks + i), f), 1u)] = (int)i;
}

}  // namespace

OrderFrame order_frame(const int lo[3], const int hi[3]) {
  OrderFrame f;
  long long ext = 1;
  for (int a = 0; a < 3; ++a) {
    f.lo[a] = lo[a];
    const long long e = (long long)hi[a] - (long long)lo[a];
    if (e > ext) ext = e;
  }
  f.shift = 0;
  while ((ext - 1) >> f.shift >= (1ll << kOrderAxisBits)) ++f.shift;
  return f;
}

cudaError_t launch_brick_order_count(const int4* bricks, long long n_bricks, OrderFrame f, unsigned* count,
                                     int grid, cudaStream_t st) {
  if (n_bricks <= 0) return cudaSuccess;
  k_order_count<<<grid, 256, 0, st>>>(bricks, n_bricks, f, count);
  return cudaGetLastError();
}

cudaError_t launch_brick_order_scan(unsigned* count, cudaStream_t st) {
  k_order_scan<<<1, kScanThreads, 0, st>>>(count);
  return cudaGetLastError();
}

cudaError_t launch_brick_order_scatter(const int4* bricks, long long n_bricks, OrderFrame f, unsigned* offset,
                                       int* order, int grid, cudaStream_t st) {
  if (n_bricks <= 0) return cudaSuccess;
  k_order_scatter<<<grid, 256, 0, st>>>(bricks, n_bricks, f, offset, order);
  return cudaGetLastError();
}

}  // namespace amriso
