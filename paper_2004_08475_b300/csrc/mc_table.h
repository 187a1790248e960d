// Host-generated Marching Cubes table (see mc_table.cpp).
#pragma once
#include <cstdint>

namespace amriso {

struct McTable {
  uint8_t count[256];        // triangles per case, 0..5
  uint8_t edges[256][15];    // 3 edge indices per triangle, 255 = unused
  uint64_t packed[256];      // edge index of vertex i of the case at bits 4i..4i+3
  uint8_t edge_a[12], edge_b[12];
};

void make_mc_table(McTable* t);

}  // namespace amriso
