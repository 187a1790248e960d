// Marching Cubes triangle table for the dual-cell kernels (Sec. 5, Sec. 5.1).
//
// The paper feeds every (possibly degenerate) dual hexahedron to standard MC
// case tables. This library generates its own table once, on the host, from
// a face rule, instead of copying one:
//   * corner e of the hexahedron sits at (e&1, (e>>1)&1, e>>2); a corner is
//     inside when its scalar is > iso;
//   * every face is walked counter-clockwise as seen from outside the cube;
//     each maximal run of inside corners is entered through one crossed edge
//     and left through another, and the run contributes the directed segment
//     entry -> exit. On a face with two separate inside corners this cuts off
//     each inside corner on its own (the two duals sharing a face see the same
//     four cells and therefore the same segments: no cracks, Sec. 5);
//   * the segments chain into closed loops; each loop is fanned from its
//     smallest edge index that has no fan diagonal lying in one cube face.
// Walking counter-clockwise with the inside run on the left makes the
// triangle normals point away from the inside corners, i.e. toward
// decreasing s.

#include <cstdint>
#include <cstring>

#include "mc_table.h"

namespace amriso {
namespace {

struct Cube {
  int ea[12], eb[12];   // edge k joins corners ea[k] < eb[k]
  int edge_of[8][8];    // corner pair -> edge index or -1
  int face_mask[12];    // bit f set when edge k lies on face f = 2*axis+side
};

Cube make_cube() {
  Cube c;
  std::memset(c.edge_of, -1, sizeof(c.edge_of));
  int k = 0;
  for (int a = 0; a < 8; ++a)
    for (int b = a + 1; b < 8; ++b) {
      const int d = a ^ b;
      if (d != 1 && d != 2 && d != 4) continue;
      c.ea[k] = a;
      c.eb[k] = b;
      c.edge_of[a][b] = c.edge_of[b][a] = k;
      int mask = 0;
      for (int axis = 0; axis < 3; ++axis) {
        if ((d >> axis) & 1) continue;                 // edge runs along axis
        mask |= 1 << (2 * axis + ((a >> axis) & 1));   // both ends on this side
      }
      c.face_mask[k] = mask;
      ++k;
    }
  return c;
}

// Corners of face (axis, side) counter-clockwise seen from outside.
void face_ring_ccw(int axis, int side, int ring[4]) {
  const int u = (axis + 1) % 3, v = (axis + 2) % 3;   // (u, v, axis) right-handed
  const int uv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};  // ccw seen from +axis
  for (int r = 0; r < 4; ++r) {
    const int rr = side ? r : (4 - r) % 4;   // seen from -axis: reverse
    ring[r] = (uv[rr][0] << u) | (uv[rr][1] << v) | (side << axis);
  }
}

int build_case(const Cube& c, int cas, uint8_t out[15]) {
  int next[12];
  for (int k = 0; k < 12; ++k) next[k] = -1;
  auto in = [cas](int corner) { return (cas >> corner) & 1; };
  for (int axis = 0; axis < 3; ++axis)
    for (int side = 0; side < 2; ++side) {
      int ring[4];
      face_ring_ccw(axis, side, ring);
      int entry = -1;
      // start the walk just after an outside corner so runs are not split
      int start = -1;
      for (int r = 0; r < 4; ++r)
        if (!in(ring[r])) start = r;
      if (start < 0) continue;  // all four inside: nothing crosses
      for (int s = 1; s <= 4; ++s) {
        const int p = ring[(start + s - 1) % 4], q = ring[(start + s) % 4];
        if (!in(p) && in(q)) entry = c.edge_of[p][q];
        if (in(p) && !in(q)) next[entry] = c.edge_of[p][q];
      }
    }
  int n = 0;
  bool used[12] = {false};
  for (int k = 0; k < 12; ++k) {
    if (next[k] < 0 || used[k]) continue;
    int loop[12], len = 0;
    for (int e = k; !used[e]; e = next[e]) {
      used[e] = true;
      loop[len++] = e;
    }
    // apex: smallest edge index whose fan diagonals leave the cube faces
    int best = -1;
    for (int p = 0; p < len; ++p) {
      bool flat = false;
      for (int q = 2; q + 1 < len; ++q)
        if (c.face_mask[loop[p]] & c.face_mask[loop[(p + q) % len]]) flat = true;
      if (!flat && (best < 0 || loop[p] < loop[best])) best = p;
    }
    if (best < 0) best = 0;
    for (int t = 1; t + 1 < len; ++t) {
      out[3 * n + 0] = uint8_t(loop[best]);
      out[3 * n + 1] = uint8_t(loop[(best + t) % len]);
      out[3 * n + 2] = uint8_t(loop[(best + t + 1) % len]);
      ++n;
    }
  }
  return n;
}

}  // namespace

void make_mc_table(McTable* t) {
  const Cube c = make_cube();
  for (int cas = 0; cas < 256; ++cas) {
    uint8_t tri[15];
    std::memset(tri, 255, sizeof(tri));
    const int n = build_case(c, cas, tri);
    t->count[cas] = uint8_t(n);
    uint64_t packed = 0;
    for (int i = 0; i < 15; ++i) {
      t->edges[cas][i] = tri[i];
      if (i < 3 * n) packed |= uint64_t(tri[i]) << (4 * i);
    }
    t->packed[cas] = packed;
  }
  for (int k = 0; k < 12; ++k) {
    t->edge_a[k] = uint8_t(c.ea[k]);
    t->edge_b[k] = uint8_t(c.eb[k]);
  }
}

}  // namespace amriso
