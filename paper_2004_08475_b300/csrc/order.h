// Spatial processing order of the bricks (sm_103a).
//
// The insert pass numbers bricks in the order their first cell arrives, which
// for unordered input is a random order in space. The dual-cell kernel runs
// one CTA per brick and reads a one-cell halo from the 26 neighbouring
// bricks; in random order those neighbours were read long ago or will be read
// much later, so their halo sectors come from DRAM. Visiting the bricks
// bucket by bucket along a Morton curve over the bounding box (a counting
// sort of their lower corners, 5 bits per axis) keeps the neighbours of the
// bricks in flight in L2. Any permutation gives the same set of dual cells;
// only the order of the output list and the traffic change.
#pragma once

#include <cuda_runtime.h>

namespace amriso {

constexpr int kOrderAxisBits = 5;
constexpr int kOrderBuckets = 1 << (3 * kOrderAxisBits);   // 32768

// Bucket frame: bucket coordinate = clamp((corner - lo) >> shift, 0, 31).
struct OrderFrame {
  int lo[3];
  int shift;
};

// Host: the frame for a bounding box [lo, hi) (finest units).
OrderFrame order_frame(const int lo[3], const int hi[3]);

// count[kOrderBuckets] must be zeroed by the caller; order[n_bricks] receives
// a permutation of 0..n_bricks-1. Three launches on `st`: histogram, scan
// (count becomes the exclusive offsets), scatter.
cudaError_t launch_brick_order_count(const int4* bricks, long long n_bricks, OrderFrame f, unsigned* count,
                                     int grid, cudaStream_t st);
cudaError_t launch_brick_order_scan(unsigned* count, cudaStream_t st);
cudaError_t launch_brick_order_scatter(const int4* bricks, long long n_bricks, OrderFrame f, unsigned* offset,
                                       int* order, int grid, cudaStream_t st);

}  // namespace amriso
