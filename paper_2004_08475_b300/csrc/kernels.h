// Declarations shared by the CUDA kernels (kernels.cu) and the C ABI
// (api.cu). Nothing here is part of the public interface.
#pragma once

#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

namespace amriso {

constexpr uint32_t kReject = 0xFFFFFFFFu;          // "does not exist" in a view
constexpr unsigned long long kEmptyKey = ~0ull;     // free hash slot
constexpr unsigned long long kEmptyRec = ~0ull;     // free brick slot
constexpr int kMaxLevel = 14;                       // levels 0..14
constexpr int kMaxIso = 64;                         // iso-values per batch

enum ErrBits : uint32_t {
  ERR_UNALIGNED = 1u,
  ERR_RANGE = 2u,
  ERR_NONFINITE = 4u,
  ERR_DUPLICATE = 8u,
  ERR_OVERLAP = 16u,
  ERR_HASH_FULL = 32u,
};

// Small device-resident counters, one allocation per context.
struct Scratch {
  unsigned long long n_bricks;
  unsigned long long n_dual;
  unsigned long long tile;              // persistent-kernel work counter
  unsigned long long n_tri[kMaxIso];    // per iso-value triangle counters
  unsigned long long n_occupied;        // occupied brick slots (= cells unless duplicates)
  unsigned long long n_vtx;             // welded vertices of an indexed face set
  unsigned long long n_elist;           // bricks with empty slots (binned placement)
  unsigned int err;
  int lo[3];                            // bounding box: min lower corner
  int hi[3];                            // max (lower corner + width)
  int max_level;
};

// Device view of the point-location structure (Sec. 3.2).
struct Locator {
  const ulonglong2* htab;           // [hcap] {brick key (level, brick coords), brick index}:
                                    //   one 16-byte entry, so a probe is one memory transaction
  unsigned long long hmask;         // hcap - 1 (hcap a power of two)
  const int4* bricks;               // [n_bricks] origin x,y,z (finest units), level
  const unsigned long long* rec;    // [n_slots] occupant: input index (low 32 bits, all ones
                                    //   when empty) and scalar bits (high 32 bits)
  const float* scal;                // [n_slots] scalar of the slot's cell
  const unsigned* view;             // [n_slots] resolved cell slot, or kReject
  int levels;                       // max level + 1
};

// Marching Cubes table in the form the kernels read (generated on the host).
struct McConst {
  unsigned long long packed[256];   // 4-bit edge ids, 3 per triangle
  unsigned char count[256];         // triangles per case
  unsigned long long edge_a;        // 4-bit lower corner of edge k at bits 4k
  unsigned long long edge_b;        // 4-bit upper corner of edge k
};

// ---- launches (all asynchronous on `st`) --------------------------------
// Each returns the launch's cudaError_t (cudaGetLastError after launch).

// brick_limit: once this many bricks exist the table counts as full
// (ERR_HASH_FULL is raised and the remaining inserts stop early); bricks[]
// must hold brick_limit entries. htab must be all ones before the launch.
// codes (may be NULL; needs hcap << 3 log2_brick <= 2^31): per cell its slot,
// or (bit 31 set) the table entry of its brick << 3 log2_brick | its Morton
// index in the brick, for launch_bin_coarse.
cudaError_t launch_insert_bricks(int logb, const int* xyz, const unsigned char* lvl, const float* s,
                                 long long n, ulonglong2* htab,
                                 unsigned long long hmask, int4* bricks,
                                 unsigned long long brick_limit, Scratch* sc, int grid, int block,
                                 unsigned* codes, cudaStream_t st);

// rec must be all ones (kEmptyRec) before the launch.
cudaError_t launch_scatter_cells(int logb, const int* xyz, const unsigned char* lvl, const float* s,
                                 long long n, Locator loc, unsigned long long* rec, Scratch* sc,
                                 int grid, int block, cudaStream_t st);

// Binned cell placement (three passes; see kernels.cu), same result as
// launch_scatter_cells plus every slot's view (the slot itself where a cell
// occupies it, else kReject until launch_resolve_empty) and scalar. All
// three take the same staging buffer of bin_layout(n_slots).bytes bytes;
// launch_bin_coarse clears its counters first.
struct BinLayout {
  long long n_coarse = 0, n_win = 0, stage_a = 0, stage_b = 0;
  size_t bytes = 0;
};
BinLayout bin_layout(long long n_slots);
// codes: from launch_insert_bricks (required).
cudaError_t launch_bin_coarse(int logb, const float* s, long long n, Locator loc, long long n_slots, void* staging,
                              Scratch* sc, int sm_count, const unsigned* codes, cudaStream_t st);
cudaError_t launch_bin_fine(long long n_slots, void* staging, Scratch* sc, cudaStream_t st);
// Writes rec[], view[] and scal[] of every slot; elist[n_bricks] receives
// the bricks with empty slots (counted by sc->n_elist, 0 before).
cudaError_t launch_place_windows(int logb, long long n_slots, void* staging, unsigned long long* rec, unsigned* view,
                                 float* scal, unsigned* elist, Scratch* sc, cudaStream_t st);
// Resolves the empty slots of the listed bricks (view only).
cudaError_t launch_resolve_empty(int logb, Locator loc, const unsigned* elist, const Scratch* sc, unsigned* view,
                                 int grid, cudaStream_t st);

// Writes view[] and scal[] of every slot from rec[].
cudaError_t launch_resolve_views(int logb, Locator loc, unsigned* view, float* scal, long long n_slots,
                                 int check_overlap, Scratch* sc, int grid, int block,
                                 cudaStream_t st);

// nbr[n_bricks][27]: neighbour brick | level << 27, or -1 (see kernels.cu)
cudaError_t launch_brick_neighbors(int logb, Locator loc, long long n_bricks, int* nbr, int grid,
                                   cudaStream_t st);

// order: NULL (bricks in index order) or a permutation of the bricks, the
// order in which the CTAs visit them (see order.h). Only cells whose lower
// corner's x lies in [own_x0, own_x1) emit their duals.
cudaError_t launch_dual_cells(int logb, Locator loc, const int* nbr, const int* order, long long n_bricks,
                              uint4* duals, long long cap, Scratch* sc, cudaStream_t st, int own_x0 = INT_MIN,
                              int own_x1 = INT_MAX);

// Dual cells plus Marching Cubes at `iso` on each of them in the same pass;
// triangles appended through sc->n_tri[0] (reset by the caller).
cudaError_t launch_dual_cells_iso(int logb, Locator loc, const int* nbr, const int* order, long long n_bricks,
                                  uint4* duals, long long cap, Scratch* sc, float iso, float* tris,
                                  long long tri_cap, const McConst& mc, cudaStream_t st);

// tags (may be NULL): per written triangle the index of its dual in `duals`.
cudaError_t launch_mc(int logb, Locator loc, const uint4* duals, long long nd, float iso,
                      float* tris, long long cap, unsigned long long* counter,
                      unsigned char* cases, unsigned char* ntri, const McConst& mc, int grid,
                      cudaStream_t st, long long* tags = nullptr);

// Indexed face set (three passes): the kept triangles' edge keys (u64 slot
// pairs, smaller first) into tkeys[cap][3] through `counter`; the keys into
// the weld table wtab (all ones before the first pass; sc->n_vtx counts the
// vertices, whose positions go to vtx[vcap][3] and cells' input indices to
// vkeys[vcap][2] if not NULL); then tri[n_tri][3] vertex indices.
cudaError_t launch_mc_keys(int logb, Locator loc, const uint4* duals, long long nd, float iso,
                           unsigned long long* tkeys, long long cap, unsigned long long* counter, const McConst& mc,
                           int grid, cudaStream_t st);
cudaError_t launch_weld_insert(int logb, Locator loc, const unsigned long long* tkeys, long long n_keys,
                               ulonglong2* wtab, unsigned long long wmask, float iso, float* vtx, int* vkeys,
                               long long vcap, Scratch* sc, int grid, cudaStream_t st);
cudaError_t launch_weld_index(const unsigned long long* tkeys, long long n_tri, const ulonglong2* wtab,
                              unsigned long long wmask, int* tri, int grid, cudaStream_t st);

// Batched iso-values over one or several resident dual lists (see
// kernels.cu): a job is one data set's dual list with its run of n_iso
// iso-values; job j's iso-values are entries q0 .. q0 + n_iso - 1 of the
// batch's iso array, and (job, value) q owns output segment q.
constexpr int kBTile = 4096;   // most duals per tile
// Tile of a job's dual list in the batched passes: the largest power of two
// up to kBTile (at least 256) that still cuts the list into about 16384
// tiles, so that a small data set's tiles still occupy every warp.
int batch_tile(long long nd);
constexpr int kMaxJobs = 32;   // data sets in one batch

struct BatchJob {
  const uint4* duals;
  const float* scal;
  const int4* bricks;
  long long nd;
  long long tile0;   // first tile of this job in the batch's tile numbering
  long long tiles;   // tiles of this job
  long long cbase;   // first counter of this job: counters [n_iso][tiles]
  long long tile;    // duals per tile (batch_tile(nd))
  int logb;
  int q0;            // first segment (index into the batch's iso-values)
  int n_iso;
};

struct BatchTable {
  int n_jobs = 0;
  int n_q = 0;            // segments = iso-values of the batch (<= kMaxIso)
  long long n_tiles = 0;
  long long n_counters = 0;
  BatchJob job[kMaxJobs];
};

// Appends a job (the caller checks n_jobs < kMaxJobs and n_q + n_iso <= kMaxIso).
void batch_add_job(BatchTable& T, const uint4* duals, const float* scal, const int4* bricks, long long nd, int logb,
                   int n_iso);
// Device workspace of a batch with n_counters = T.n_counters.
size_t batch_workspace_bytes(long long n_counters);
// Per tile and iso-value the kept triangles (isos: the batch's device array).
cudaError_t launch_batch_count(const BatchTable& T, const float* isos, void* ws, const McConst& mc, int grid,
                               cudaStream_t st);
// off[0..n_q]: each segment's first row and, last, the total (device).
cudaError_t launch_batch_scan(const BatchTable& T, void* ws, long long* off, cudaStream_t st);
// Segment q gets rows off[q] .. off[q+1]-1, clipped to cap.
cudaError_t launch_batch_emit(const BatchTable& T, const float* isos, const void* ws, const long long* off,
                              float* tris, long long cap, const McConst& mc, int grid, cudaStream_t st);

cudaError_t launch_get_duals(const uint4* duals, long long nd, const unsigned long long* rec, int* out,
                             int grid, cudaStream_t st);

}  // namespace amriso
