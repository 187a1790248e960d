// Oracle for the AMR dual-mesh and iso-surface method (Wald, "A Simple,
// General, and GPU Friendly Method for Computing Dual Mesh and Iso-Surfaces
// of AMR Data").
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow, single-threaded CPU
// restatement of what the method computes. Only the test suite, the smoke
// check and the benchmark's CPU-baseline leg may load it. The CUDA library
// shares no code, header, table or helper with it.
//
// What it computes, in the paper's order and notation:
//   * the set of actual cells and the snap() cell-location operator (Sec. 3.1,
//     Sec. 3.2): an ordered map from the integer label (i,j,k;l) to the cell,
//     probed finest level first after zeroing the low l bits of the query;
//   * for every actual cell its 8 logical duals and the three rejection rules
//     that make each dual cell come out exactly once (Sec. 4.2, Sec. 4.3,
//     the doCell/doDualCell pseudo-code of Sec. 4.4);
//   * Marching Cubes on the possibly degenerate dual hexahedra, with vertices
//     interpolated between the snapped cell centres and triangles that do not
//     have three different vertices dropped (Sec. 5, Sec. 5.1, Sec. 5.2).
//
// Readings where the paper is silent or garbled (each is listed in the design
// notes of the repository):
//   * the 8 duals of cell C^(l)_{i,j,k} are D^(l)_{i+d} with d in {-1,0}^3 in
//     level units (the duals whose vertex sets contain the cell; Sec. 3.1
//     defines D_i as spanning centre C_i to centre C_{i+1});
//   * "v < self" in rule 3 is lexicographic on the lower corner (z, y, x);
//   * a cell centre is lower corner + 2^l / 2;
//   * inside bit of a MC corner: s > iso (strict); a crossed edge is
//     interpolated from its endpoint with the smaller (z, y, x) lower corner;
//     fp32 in the fixed order d = sb - sa, t = (iso - sa) / d,
//     P = ca + t * (cb - ca), no fused multiply-add (built with
//     -ffp-contract=off); the same in fp64 as a cross-check;
//   * triangulation by a run-time face walk: on every face of the hexahedron
//     the crossed edges are paired so that inside corners are cut off, the
//     pairs are oriented with the inside corner on a fixed side (normals point
//     toward decreasing s), chained into loops, and each loop is fanned from
//     its smallest edge index;
//   * "three different vertices" means three different edge keys, the
//     unordered pair of cells an interpolated vertex lies between.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Cells and cell location (Sec. 3.1, Sec. 3.2)
// ---------------------------------------------------------------------------

// Integer label (i,j,k;l) of a logical cell; ordered by level, then z, y, x.
struct Label {
  int l;
  int32_t k, j, i;
  bool operator<(const Label& o) const {
    return std::tie(l, k, j, i) < std::tie(o.l, o.k, o.j, o.i);
  }
};

struct Mesh {
  const int32_t* xyz;      // [n][3] lower corners, finest-level units
  const uint8_t* level;    // [n]
  int64_t n;
  int L;                   // number of levels present: max level + 1
  std::map<Label, int64_t> actual;  // the set of actual cells -> local index
};

// Zero the low l bits (two's complement, so negative coordinates floor).
inline int32_t project(int32_t c, int l) {
  return c & ~((int32_t(1) << l) - 1);
}

// snap(i,j,k): the actual cell containing the integer point (i,j,k), probing
// the levels finest to coarsest (Sec. 3.2); -1 stands for "does not exist".
int64_t snap(const Mesh& m, int32_t i, int32_t j, int32_t k) {
  for (int l = 0; l < m.L; ++l) {
    auto it = m.actual.find(Label{l, project(k, l), project(j, l), project(i, l)});
    if (it != m.actual.end()) return it->second;
  }
  return -1;
}

// "v < self" of rule 3: lexicographic on the lower corner, z first.
bool lower_than(const Mesh& m, int64_t a, int64_t b) {
  const int32_t* pa = m.xyz + 3 * a;
  const int32_t* pb = m.xyz + 3 * b;
  return std::tie(pa[2], pa[1], pa[0]) < std::tie(pb[2], pb[1], pb[0]);
}

// Builds the cell set; returns 0, or a negative code for invalid input
// (-2 unaligned corner, -3 level out of range, -5 duplicate label).
int build_mesh(Mesh& m, const int32_t* xyz, const uint8_t* level, int64_t n) {
  m.xyz = xyz;
  m.level = level;
  m.n = n;
  m.L = 0;
  m.actual.clear();
  for (int64_t c = 0; c < n; ++c) {
    int l = level[c];
    if (l > 20) return -3;
    const int32_t* p = xyz + 3 * c;
    for (int a = 0; a < 3; ++a)
      if (project(p[a], l) != p[a]) return -2;
    if (!m.actual.emplace(Label{l, p[2], p[1], p[0]}, c).second) return -5;
    if (l + 1 > m.L) m.L = l + 1;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Dual cells (Sec. 4.2 - 4.4)
// ---------------------------------------------------------------------------

// doDualCell: the logical level-l dual whose lowest vertex is the logical cell
// with lower corner (i,j,k). Returns true and fills vertex[ex + 2ey + 4ez] when
// the dual is emitted by cell `self`.
bool do_dual_cell(const Mesh& m, int64_t self, int32_t i, int32_t j, int32_t k,
                  int l, int64_t vertex[8]) {
  const int32_t w = int32_t(1) << l;
  for (int ez = 0; ez < 2; ++ez)
    for (int ey = 0; ey < 2; ++ey)
      for (int ex = 0; ex < 2; ++ex) {
        int64_t v = snap(m, i + ex * w, j + ey * w, k + ez * w);
        if (v < 0) return false;                       // rule #1: outside / hole
        if (m.level[v] < l) return false;              // rule #2: finer level
        if (m.level[v] == l && lower_than(m, v, self))
          return false;                                // rule #3: smaller owner
        vertex[ex + 2 * ey + 4 * ez] = v;
      }
  return true;
}

// doCell: the 8 logical duals that cover cell `self` (offsets -1,0).
int do_cell(const Mesh& m, int64_t self, int64_t out[8][8]) {
  const int l = m.level[self];
  const int32_t w = int32_t(1) << l;
  const int32_t* p = m.xyz + 3 * self;
  int emitted = 0;
  for (int dk = -1; dk <= 0; ++dk)
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        int64_t vertex[8];
        if (do_dual_cell(m, self, p[0] + di * w, p[1] + dj * w, p[2] + dk * w, l,
                         vertex)) {
          for (int e = 0; e < 8; ++e) out[emitted][e] = vertex[e];
          ++emitted;
        }
      }
  return emitted;
}

// ---------------------------------------------------------------------------
// Marching Cubes on a (possibly degenerate) dual hexahedron (Sec. 5)
// ---------------------------------------------------------------------------

// Hexahedron corner e = ex + 2 ey + 4 ez sits at unit-cube position (ex,ey,ez).
// The 12 edges are the corner pairs (a,b), a < b, differing in one bit, listed
// in increasing (a,b) order.
struct Edges {
  int a[12], b[12];
  int id[8][8];
  Edges() {
    int n = 0;
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < 8; ++j) id[i][j] = -1;
    for (int i = 0; i < 8; ++i)
      for (int j = i + 1; j < 8; ++j) {
        int d = i ^ j;
        if (d == 1 || d == 2 || d == 4) {
          a[n] = i;
          b[n] = j;
          id[i][j] = id[j][i] = n;
          ++n;
        }
      }
  }
};
const Edges kEdges;

void corner_pos(int v, double p[3]) {
  p[0] = v & 1;
  p[1] = (v >> 1) & 1;
  p[2] = (v >> 2) & 1;
}

// True when hexahedron edges e and f lie on a common face of the unit cube
// (the face is the axis along which both endpoints of both edges agree).
bool share_face(int e, int f) {
  double a0[3], a1[3], b0[3], b1[3];
  corner_pos(kEdges.a[e], a0);
  corner_pos(kEdges.b[e], a1);
  corner_pos(kEdges.a[f], b0);
  corner_pos(kEdges.b[f], b1);
  for (int x = 0; x < 3; ++x)
    if (a0[x] == a1[x] && b0[x] == b1[x] && a0[x] == b0[x]) return true;
  return false;
}

// Run-time face walk for one case: returns the triangles (as edge-index
// triples) in fan order, loops taken in order of their smallest edge index.
int face_walk(int cas, int tri[16][3]) {
  bool inside[8];
  for (int v = 0; v < 8; ++v) inside[v] = (cas >> v) & 1;
  int next[12];
  for (int e = 0; e < 12; ++e) next[e] = -1;
  // The 6 faces: fixed axis and side; corners listed around the face.
  for (int axis = 0; axis < 3; ++axis)
    for (int side = 0; side < 2; ++side) {
      const int u = (axis + 1) % 3, w = (axis + 2) % 3;
      int ring[4];
      const int uv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
      for (int r = 0; r < 4; ++r) {
        int c[3];
        c[axis] = side;
        c[u] = uv[r][0];
        c[w] = uv[r][1];
        ring[r] = c[0] + 2 * c[1] + 4 * c[2];
      }
      double normal[3] = {0, 0, 0};
      normal[axis] = side ? 1.0 : -1.0;  // outward
      // crossed ring edges: ring[r] -- ring[r+1]
      int crossed[4], nc = 0;
      for (int r = 0; r < 4; ++r)
        if (inside[ring[r]] != inside[ring[(r + 1) % 4]]) crossed[nc++] = r;
      // pairs of ring-edge slots, each with the inside corner it cuts off
      int pr[2][2], pc[2], np = 0;
      if (nc == 2) {
        pr[0][0] = crossed[0];
        pr[0][1] = crossed[1];
        // any inside corner of the face lies on the cut-off side
        int cin = -1;
        for (int r = 0; r < 4; ++r)
          if (inside[ring[r]]) cin = ring[r];
        pc[0] = cin;
        np = 1;
      } else if (nc == 4) {
        // ambiguous face: pair the two edges meeting at each inside corner
        for (int r = 0; r < 4; ++r)
          if (inside[ring[r]]) {
            pr[np][0] = (r + 3) % 4;
            pr[np][1] = r;
            pc[np] = ring[r];
            ++np;
          }
      }
      for (int q = 0; q < np; ++q) {
        int s0 = pr[q][0], s1 = pr[q][1];
        int e0 = kEdges.id[ring[s0]][ring[(s0 + 1) % 4]];
        int e1 = kEdges.id[ring[s1]][ring[(s1 + 1) % 4]];
        double p0[3], p1[3], ca[3], cb[3], c[3];
        corner_pos(kEdges.a[e0], ca);
        corner_pos(kEdges.b[e0], cb);
        for (int x = 0; x < 3; ++x) p0[x] = 0.5 * (ca[x] + cb[x]);
        corner_pos(kEdges.a[e1], ca);
        corner_pos(kEdges.b[e1], cb);
        for (int x = 0; x < 3; ++x) p1[x] = 0.5 * (ca[x] + cb[x]);
        corner_pos(pc[q], c);
        double d[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
        double g[3] = {c[0] - p0[0], c[1] - p0[1], c[2] - p0[2]};
        double x[3] = {d[1] * g[2] - d[2] * g[1], d[2] * g[0] - d[0] * g[2],
                       d[0] * g[1] - d[1] * g[0]};
        double side_sign = x[0] * normal[0] + x[1] * normal[1] + x[2] * normal[2];
        // orientation: run P0 -> P1 when ((P1 - P0) x (c - P0)) . n_out < 0,
        // with c the inside corner the segment cuts off; this makes the
        // loop normals point away from the inside corners (decreasing s)
        if (side_sign < 0) next[e0] = e1;
        else next[e1] = e0;
      }
    }
  int ntri = 0;
  bool seen[12] = {false};
  for (int e = 0; e < 12; ++e) {
    if (next[e] < 0 || seen[e]) continue;
    int loop[12], len = 0;
    int cur = e;
    do {
      seen[cur] = true;
      loop[len++] = cur;
      cur = next[cur];
    } while (cur != e && len < 12);
    // Fan apex: the smallest edge index none of whose fan diagonals joins
    // two edges of one cube face (such a diagonal would put a flat triangle
    // into a face that the neighbouring dual also fills).
    int apex = -1;
    for (int cand = 0; cand < 12 && apex < 0; ++cand) {
      int pos = -1;
      for (int q = 0; q < len; ++q)
        if (loop[q] == cand) pos = q;
      if (pos < 0) continue;
      bool ok = true;
      for (int q = 0; q < len; ++q) {
        if (q == pos || q == (pos + 1) % len || q == (pos + len - 1) % len) continue;
        if (share_face(loop[pos], loop[q])) ok = false;
      }
      if (ok) apex = pos;
    }
    if (apex < 0) apex = 0;  // not reached: every loop has such an apex
    for (int t = 1; t + 1 < len; ++t) {
      tri[ntri][0] = loop[apex];
      tri[ntri][1] = loop[(apex + t) % len];
      tri[ntri][2] = loop[(apex + t + 1) % len];
      ++ntri;
    }
  }
  return ntri;
}

struct Vtx {
  float p32[3];
  double p64[3];
  int64_t key_lo, key_hi;  // edge key: the two cells (local indices), sorted
};

// Interpolated vertex on hexahedron edge (va, vb) at `iso`.
Vtx edge_vertex(const Mesh& m, const float* s, int64_t va, int64_t vb, float iso) {
  // canonical orientation: smaller (z,y,x) lower corner first
  if (lower_than(m, vb, va)) std::swap(va, vb);
  const int32_t* pa = m.xyz + 3 * va;
  const int32_t* pb = m.xyz + 3 * vb;
  const float ha = float(int32_t(1) << m.level[va]) * 0.5f;
  const float hb = float(int32_t(1) << m.level[vb]) * 0.5f;
  Vtx out;
  const float sa = s[va], sb = s[vb];
  const float d = sb - sa;
  const float t = (iso - sa) / d;
  const double d64 = double(sb) - double(sa);
  const double t64 = (double(iso) - double(sa)) / d64;
  for (int x = 0; x < 3; ++x) {
    const float ca = float(pa[x]) + ha;  // cell centre (exact)
    const float cb = float(pb[x]) + hb;
    const float dc = cb - ca;
    const float tdc = t * dc;
    out.p32[x] = ca + tdc;
    out.p64[x] = double(ca) + t64 * (double(cb) - double(ca));
  }
  out.key_lo = va < vb ? va : vb;
  out.key_hi = va < vb ? vb : va;
  return out;
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (called through ctypes by the tests and the CPU baseline)
// ---------------------------------------------------------------------------

struct OracleMesh {
  Mesh m;
};

extern "C" {

// Builds the actual-cell set. Returns a handle, or nullptr with *err set.
void* oracle_mesh_create(const int32_t* xyz, const uint8_t* level, int64_t n,
                         int* err) {
  OracleMesh* om = new OracleMesh();
  int rc = build_mesh(om->m, xyz, level, n);
  if (err) *err = rc;
  if (rc != 0) {
    delete om;
    return nullptr;
  }
  return om;
}

void oracle_mesh_destroy(void* h) { delete static_cast<OracleMesh*>(h); }

int oracle_num_levels(void* h) { return static_cast<OracleMesh*>(h)->m.L; }

// snap() of Sec. 3.2 at one integer point; -1 when no actual cell contains it.
int64_t oracle_snap(void* h, int32_t i, int32_t j, int32_t k) {
  return snap(static_cast<OracleMesh*>(h)->m, i, j, k);
}

// Dual cells emitted by the cells `owners[0..n_owners)` (all cells when owners
// is null). Writes local cell indices, 8 per dual in vertex order
// e = ex + 2 ey + 4 ez, into out[cap][8] and the owner of each dual into
// out_owner (optional). Returns the number of duals (which may exceed cap;
// nothing past cap is written).
int64_t oracle_duals(void* h, const int64_t* owners, int64_t n_owners,
                     int64_t* out, int64_t* out_owner, int64_t cap) {
  const Mesh& m = static_cast<OracleMesh*>(h)->m;
  int64_t nd = 0;
  const int64_t count = owners ? n_owners : m.n;
  for (int64_t q = 0; q < count; ++q) {
    const int64_t self = owners ? owners[q] : q;
    int64_t duals[8][8];
    const int k = do_cell(m, self, duals);
    for (int d = 0; d < k; ++d) {
      if (nd < cap) {
        for (int e = 0; e < 8; ++e) out[8 * nd + e] = duals[d][e];
        if (out_owner) out_owner[nd] = self;
      }
      ++nd;
    }
  }
  return nd;
}

// Triangles of one MC case by the run-time face walk: tri[16][3] edge
// indices; returns the count (before any degenerate-triangle filtering).
int oracle_case_triangles(int cas, int32_t* tri) {
  int t[16][3];
  int n = face_walk(cas & 255, t);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) tri[3 * i + c] = t[i][c];
  return n;
}

// Marching Cubes over the given dual cells at `iso`.
//   duals [nd][8] local cell indices; s [n] scalars.
//   cases [nd] (optional) case index; ntri [nd] (optional) kept triangles;
//   tris [cap][3][3] fp32 vertices; keys [cap][3][2] (optional) edge keys as
//   local cell indices; tri_dual [cap] (optional) dual index of each triangle.
//   *max_err (optional): max |P32 - P64| over all written vertices.
// Returns the number of kept triangles (may exceed cap; nothing past cap is
// written).
int64_t oracle_iso(void* h, const float* s, const int64_t* duals, int64_t nd,
                   float iso, uint8_t* cases, uint8_t* ntri, float* tris,
                   int64_t* keys, int64_t* tri_dual, int64_t cap,
                   double* max_err) {
  const Mesh& m = static_cast<OracleMesh*>(h)->m;
  int64_t nt = 0;
  double err = 0.0;
  for (int64_t d = 0; d < nd; ++d) {
    const int64_t* v = duals + 8 * d;
    int cas = 0;
    for (int e = 0; e < 8; ++e)
      if (s[v[e]] > iso) cas |= 1 << e;
    if (cases) cases[d] = uint8_t(cas);
    int t[16][3];
    const int n = face_walk(cas, t);
    int kept = 0;
    for (int i = 0; i < n; ++i) {
      Vtx vt[3];
      for (int c = 0; c < 3; ++c) {
        const int e = t[i][c];
        vt[c] = edge_vertex(m, s, v[kEdges.a[e]], v[kEdges.b[e]], iso);
      }
      auto same = [](const Vtx& a, const Vtx& b) {
        return a.key_lo == b.key_lo && a.key_hi == b.key_hi;
      };
      if (same(vt[0], vt[1]) || same(vt[1], vt[2]) || same(vt[0], vt[2]))
        continue;  // fewer than three different vertices
      if (nt < cap) {
        for (int c = 0; c < 3; ++c)
          for (int x = 0; x < 3; ++x) {
            tris[9 * nt + 3 * c + x] = vt[c].p32[x];
            double e64 = std::fabs(double(vt[c].p32[x]) - vt[c].p64[x]);
            if (e64 > err) err = e64;
          }
        if (keys)
          for (int c = 0; c < 3; ++c) {
            keys[6 * nt + 2 * c] = vt[c].key_lo;
            keys[6 * nt + 2 * c + 1] = vt[c].key_hi;
          }
        if (tri_dual) tri_dual[nt] = d;
      }
      ++nt;
      ++kept;
    }
    if (ntri) ntri[d] = uint8_t(kept);
  }
  if (max_err) *max_err = err;
  return nt;
}

}  // extern "C"
