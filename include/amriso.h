/*
 * amriso.h - C ABI of the B300 (sm_103a) library for dual meshes and
 * crack-free iso-surfaces of AMR data, after Wald, "A Simple, General, and
 * GPU Friendly Method for Computing Dual Mesh and Iso-Surfaces of AMR Data".
 *
 * Conventions shared by every entry point:
 *   - Return value: AMR_OK (0) or a negative AMR_ERR_* code. No C++ exception
 *     crosses this boundary. Out-parameters are written only on AMR_OK,
 *     except where an entry point says otherwise.
 *   - A cell is its lower corner (i, j, k) in finest-level units (int32) and
 *     its level l (uint8; level 0 is finest, width 2^l); the corner must be a
 *     multiple of 2^l (Sec. 3.1). Cell ID = the cell's index in the arrays
 *     given to amr_upload.
 *   - All device work runs on the context's CUDA stream, in call order.
 *     Entry points that return a count synchronise that stream once.
 *   - Pointers are device pointers unless the call's `flags` contains
 *     AMR_HOST_PTRS, in which case the library copies between host and
 *     device itself (inside the call).
 *   - One context holds one data set and everything derived from it. A
 *     context may be used from one host thread at a time.
 */
#ifndef AMRISO_H
#define AMRISO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define AMR_OK                0
#define AMR_ERR_INVALID_ARG  (-1)  /* null pointer, negative size, bad option */
#define AMR_ERR_UNALIGNED    (-2)  /* a lower corner is not a multiple of 2^l */
#define AMR_ERR_RANGE        (-3)  /* level > 14, extent >= 2^21 units per axis,
                                      a coordinate beyond +-2^30, or more than
                                      2^31-1 cells / brick slots */
#define AMR_ERR_NONFINITE    (-4)  /* a scalar is NaN or infinite */
#define AMR_ERR_DUPLICATE    (-5)  /* two cells with the same (i,j,k;l) */
#define AMR_ERR_OVERLAP      (-6)  /* a cell lies inside a coarser cell */
#define AMR_ERR_STATE        (-7)  /* call out of order (e.g. amr_iso before
                                      amr_dual_cells) */
#define AMR_ERR_OOM          (-8)  /* device allocation failed */
#define AMR_ERR_CAPACITY     (-9)  /* output buffer too small; the exact
                                      required count is still reported */
#define AMR_ERR_TIMEOUT      (-10) /* reserved for a bounded device wait that
                                      runs out; no kernel of this version
                                      waits on another thread, so no entry
                                      point returns it */
#define AMR_ERR_CUDA         (-11) /* any other CUDA runtime error */

/* ---- flags --------------------------------------------------------------- */
#define AMR_DEVICE_PTRS 0  /* arrays are device memory */
#define AMR_HOST_PTRS   1  /* arrays are host memory (pageable or pinned) */
#define AMR_COPY        2  /* amr_upload only: copy device arrays instead of
                              borrowing them */

typedef struct amr_ctx amr_ctx;

/* Options of the point-location structure (Sec. 3.2). A zeroed struct or a
 * NULL pointer selects the defaults given in brackets. */
typedef struct amr_locator_opts {
  int   log2_brick;     /* brick edge 2^log2_brick cells: 2 or 3          [3] */
  float load_factor;    /* target fill of the brick hash table, 0.05-0.9 [0.5] */
  int   block_size;     /* threads per block of cell-parallel kernels   [256] */
  int   check_overlap;  /* nonzero: reject cells inside coarser cells     [0] */
  int   partitioned;    /* cell placement: > 0 always binned (a two-level
                           split by slot, then each window of slots built in
                           shared memory and written whole), < 0 always a
                           direct scatter, 0 binned from 2^20 cells on; the
                           binned form needs a brick table of at most
                           2^(31 - 3 log2_brick) entries and otherwise falls
                           back to the direct scatter                   [0] */
} amr_locator_opts;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on CUDA device `device`, working on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream). */
int amr_create(amr_ctx** out, int device, void* cuda_stream);

/* Releases the context and every device buffer it owns. NULL is ignored. */
void amr_destroy(amr_ctx* ctx);

/* Replaces the context's stream (subsequent calls run on it). */
int amr_set_stream(amr_ctx* ctx, void* cuda_stream);

/* ---- the hot path (Sec. 3-5) -------------------------------------------- */

/* Input of the method: the unordered list of actual cells and one fp32
 * scalar per cell (Sec. 3.1; the thrust driver of Sec. 5.2 uploads the same
 * list).
 *   xyz    [n][3] int32 lower corners, finest-level units
 *   level  [n]    uint8 levels
 *   scalar [n]    fp32 cell-centred values
 * With AMR_HOST_PTRS the arrays are copied to the device inside the call.
 * With device pointers the arrays are borrowed: they must stay valid and
 * unchanged until amr_build_locator returns, and xyz and scalar as long as
 * amr_interpolate is called on the context (AMR_COPY copies them instead).
 * Validation (alignment, level range, finiteness) happens in
 * amr_build_locator. Invalidates any locator / dual cells of the context. */
int amr_upload(amr_ctx* ctx, const int32_t* xyz, const uint8_t* level,
               const float* scalar, int64_t n, int flags);

/* Builds the cell-location structure behind snap() (Sec. 3.2): per-level
 * bricks of 2^log2_brick cells per axis in one open-addressing hash table,
 * with every brick slot resolved to the actual cell that contains it (the
 * slot's own cell, a coarser cell, or none). Validates the input and fails
 * with AMR_ERR_UNALIGNED / RANGE / NONFINITE / DUPLICATE (and OVERLAP when
 * requested). Synchronises the stream. */
int amr_build_locator(amr_ctx* ctx, const amr_locator_opts* opts);

/* Emits every dual cell exactly once (Sec. 4.2-4.4): for every actual cell
 * its 8 logical duals, snapped, and kept unless a vertex is missing (rule 1),
 * finer (rule 2) or a same-level vertex is lower than the cell (rule 3). The
 * dual list stays resident in the context for later amr_iso calls.
 * *n_dual receives the number of dual cells. Synchronises the stream. */
int amr_dual_cells(amr_ctx* ctx, int64_t* n_dual);

/* amr_dual_cells restricted to one owner slab, for a data set sharded into
 * x slabs (one GPU per slab, or one after another): only the cells whose
 * lower corner's x lies in [x_begin, x_end) emit their dual cells (the
 * emitting cell of a dual is its owner, Sec. 4.4: the unique cell that rule
 * 3 lets emit it); every uploaded cell still takes part in the rules. A
 * shard that holds every cell overlapping [x_begin - w_max, x_end + w_max),
 * w_max the widest cell of the whole data set, emits exactly the whole data
 * set's dual cells owned in its slab (every vertex of such a dual contains a
 * point within one owner width of the owner, Sec. 4.2-4.4), so the slabs'
 * lists together are the whole list, each dual once. Outputs and resident
 * state as amr_dual_cells. No counterpart in the paper's GPU code (it runs
 * one GPU). */
int amr_dual_cells_owned(amr_ctx* ctx, int32_t x_begin, int32_t x_end, int64_t* n_dual);

/* amr_dual_cells and amr_iso(iso) in one pass over the locator: every dual
 * cell is emitted into the resident list (exactly as amr_dual_cells) and
 * Marching Cubes runs on it at once, from the cell scalars already staged for
 * the dual's neighbourhood - the paper's single extraction kernel (Sec. 5.1,
 * Sec. 5.2) with the dual list kept for later iso-values. Outputs as
 * amr_dual_cells (*n_dual) and amr_iso (tris, *n_tris, AMR_ERR_CAPACITY with
 * the exact count; the dual list is resident either way). Synchronises the
 * stream. */
int amr_dual_cells_iso(amr_ctx* ctx, float iso, float* tris, int64_t cap,
                       int64_t* n_dual, int64_t* n_tris, int flags);

/* Copies the resident dual cells as cell IDs: out[n_dual][8] int32, vertex
 * order e = ex + 2 ey + 4 ez (vertex e sits at the logical cell offset e
 * from the dual's lowest vertex). The order of the dual cells is unspecified
 * but equals the order of amr_iso_cases' outputs. cap = rows of `out`;
 * AMR_ERR_CAPACITY when cap < n_dual (nothing written). */
int amr_get_duals(amr_ctx* ctx, int32_t* out, int64_t cap, int flags);

/* Marching Cubes on every resident dual cell, degenerate or not (Sec. 5):
 * case bit e set iff s(vertex e) > iso; on each crossed edge the vertex is
 * interpolated between the two cell centres (from the endpoint with the
 * lower (z,y,x) corner, fp32, t = (iso - sa) / (sb - sa), P = ca + t (cb - ca),
 * no fused multiply-add); triangles without three different vertices (edge
 * keys) are dropped (Sec. 5); survivors are appended through a counter with
 * a capacity check (Sec. 5.2).
 *   tris [cap][3][3] fp32 "fat" triangles (3 complete vertices each),
 *        normals (right-hand rule) point toward decreasing s.
 *   *n_tris receives the exact triangle count; it is also written with
 *        AMR_ERR_CAPACITY when the count exceeds cap (then only the first
 *        cap triangles, in unspecified order, were written).
 * Synchronises the stream. */
int amr_iso(amr_ctx* ctx, float iso, float* tris, int64_t cap, int64_t* n_tris,
            int flags);

/* amr_iso with, beside every triangle written, the index of the dual cell
 * that produced it: the triangle -> dual map that lets a reader check the
 * triangles of each dual cell on its own (Sec. 5 extracts each dual's
 * triangles independently of every other dual's).
 *   tris     [cap][3][3] fp32, as amr_iso (the same triangles, same order
 *            rules);
 *   tri_dual [cap] int64: row t of tris came from dual tri_dual[t], an
 *            index into the resident list (the order of amr_get_duals and
 *            amr_iso_cases).
 * Both arrays are device memory, or host memory with AMR_HOST_PTRS. *n_tris
 * and AMR_ERR_CAPACITY as amr_iso. Synchronises the stream. */
int amr_iso_tagged(amr_ctx* ctx, float iso, float* tris, int64_t* tri_dual, int64_t cap,
                   int64_t* n_tris, int flags);

/* Indexed face set of the same surface (the indexed output the paper builds
 * after its extraction, Sec. 5.2, with vertices welded by their integer edge
 * key - the unordered pair of cells a vertex interpolates between - instead
 * of by sorting positions): the triangles of amr_iso, each as three vertex
 * indices in the same orientation; every edge key once as a vertex, at the
 * same fp32 position amr_iso computes for it.
 *   vtx   [vcap][3] fp32 vertex positions (unspecified order);
 *   tri   [tcap][3] int32 vertex indices;
 *   vkeys [vcap][2] int32 (may be NULL): each vertex's two cells as input
 *         indices, smaller first.
 *   *n_vtx, *n_tri receive the exact counts; when either exceeds its
 *   capacity the call returns AMR_ERR_CAPACITY and only the first vcap
 *   vertices / tcap triangles were written (a triangle may then refer to an
 *   unwritten vertex). flags: AMR_DEVICE_PTRS or AMR_HOST_PTRS for all three
 *   arrays. Synchronises the stream. */
int amr_iso_indexed(amr_ctx* ctx, float iso, float* vtx, int64_t vcap, int32_t* tri, int64_t tcap,
                    int32_t* vkeys, int64_t* n_vtx, int64_t* n_tri, int flags);

/* A second per-cell field interpolated at the vertices of an indexed face
 * set, along the same edges and with the same t as their positions (the
 * attribute mapping of the paper's introduction, Sec. 1): for vertex v with
 * cells (a, b) = vkeys[v] (input indices, as amr_iso_indexed returns them),
 * taken from the one with the lower (z,y,x) corner, t = (iso - s_a) /
 * (s_b - s_a) and out[v] = f_a + t (f_b - f_a), each fp32 operation rounded
 * on its own. iso must be the value the face set was extracted at.
 *   attr [n_cells] fp32 per input cell; vkeys [nv][2]; out [nv].
 * flags: AMR_DEVICE_PTRS or AMR_HOST_PTRS for all three arrays. A cell index
 * outside [0, n_cells) gives AMR_ERR_RANGE (and 0 for that vertex). Reads
 * the corners and scalars given to amr_upload (borrowed device arrays must
 * still be valid). Synchronises the stream. */
int amr_interpolate(amr_ctx* ctx, float iso, const float* attr, const int32_t* vkeys, int64_t nv, float* out,
                    int flags);

/* Shapes of the resident dual cells: snapping collapses a dual hexahedron
 * to a wedge, pyramid, tetrahedron or a flatter shape when several of its 8
 * vertices resolve to the same cell (Sec. 4.1, Sec. 5). counts[d] (may be
 * NULL) receives the number of distinct cells among dual d's vertices
 * (8 hexahedron, 6 wedge, 5 pyramid, 4 tetrahedron), in the dual list's
 * order (as amr_get_duals); hist[0..8] (may be NULL, host memory) the number
 * of duals with each count. flags (AMR_DEVICE_PTRS / AMR_HOST_PTRS) apply to
 * counts. Synchronises the stream. */
int amr_dual_shapes(amr_ctx* ctx, uint8_t* counts, int64_t* hist, int flags);

/* Per-dual MC case index and number of kept triangles at `iso`, in the order
 * of amr_get_duals: cases[n_dual] uint8, ntri[n_dual] uint8 (either may be
 * NULL). Synchronises the stream. */
int amr_iso_cases(amr_ctx* ctx, float iso, uint8_t* cases, uint8_t* ntri,
                  int flags);

/* Several iso-values over the resident dual cells in one persistent launch:
 * each dual's vertex IDs and scalars are read once for all values.
 *   isos    [n_iso] host array, 1 <= n_iso <= 64
 *   tris    [cap][3][3] device (or host, AMR_HOST_PTRS) output; iso k's
 *           triangles occupy rows offsets[k] .. offsets[k+1]-1
 *   offsets [n_iso+1] host int64, written on AMR_OK and on AMR_ERR_CAPACITY
 *           (then offsets[n_iso] is the required cap and nothing was
 *           written).
 * Synchronises the stream. */
int amr_iso_batch(amr_ctx* ctx, const float* isos, int n_iso, float* tris,
                  int64_t cap, int64_t* offsets, int flags);

/* amr_iso_batch without any host synchronisation or allocation, for use
 * inside a captured CUDA graph: the iso-values are read from device memory
 * when the work runs, and the segment offsets are computed on the device
 * (three kernels: per-tile counts, their prefix sums, emission; the
 * workspace was sized by amr_dual_cells).
 *   d_isos    [n_iso] device array, 1 <= n_iso <= 64
 *   tris      [cap][3][3] device output; iso k's triangles are rows
 *             d_offsets[k] .. d_offsets[k+1]-1 (rows past cap are dropped)
 *   d_offsets [n_iso+1] device int64 written by the device; the caller reads
 *             it after the stream completes and compares d_offsets[n_iso]
 *             with cap.
 * Requires amr_dual_cells to have completed on this context. Returns after
 * enqueuing. */
int amr_iso_batch_async(amr_ctx* ctx, const float* d_isos, int n_iso,
                        float* tris, int64_t cap, int64_t* d_offsets);

/* Several data sets' batches in one launch per pass (no counterpart in the
 * paper; the batching of many small data sets that serving needs): job j
 * runs Marching Cubes at n_iso iso-values over the resident dual cells of
 * jobs[j].ctx; all jobs' duals are cut into tiles that one grid shares, so
 * small data sets fill the GPU together.
 *   jobs      [n_jobs] host array, 1 <= n_jobs <= 32; every ctx after
 *             amr_dual_cells, all on one device; sum of n_iso <= 64
 *   d_isos    device array of the batch's iso-values: job 0's n_iso values,
 *             then job 1's, ...; value q of the batch is segment q
 *   tris      [cap][3][3] device output; segment q is rows d_offsets[q] ..
 *             d_offsets[q+1]-1 (rows past cap are dropped)
 *   d_offsets [segments + 1] device int64, written by the device
 *   workspace device memory of at least amr_iso_multi_workspace(jobs,
 *             n_jobs) bytes, owned by the caller (the call allocates nothing)
 *   cuda_stream the stream all work is enqueued on (NULL = legacy stream)
 * Neither synchronises nor allocates; returns after enqueuing. The result is
 * the same, segment by segment, as amr_iso_batch on each context alone. */
typedef struct amr_iso_job {
  amr_ctx* ctx;
  int n_iso;
} amr_iso_job;
int64_t amr_iso_multi_workspace(const amr_iso_job* jobs, int n_jobs);
int amr_iso_multi_async(const amr_iso_job* jobs, int n_jobs, const float* d_isos, float* tris,
                        int64_t cap, int64_t* d_offsets, void* workspace,
                        int64_t workspace_bytes, void* cuda_stream);

/* Waits for all work queued on the context's stream. */
int amr_sync(amr_ctx* ctx);

/* Frees the context's scratch workspace after waiting for its stream: the
 * staging of the binned cell placement (24 bytes per slot and 4 per cell)
 * and of host-pointer delivery. The locator, the dual cells and the input stay; later
 * calls re-create the workspace on demand. No counterpart in the paper: a
 * memory-budget aid for keeping many data sets resident. */
int amr_trim(amr_ctx* ctx);

/* Human-readable text for a return code (static storage). */
const char* amr_strerror(int code);

/* Layout version of this header's structs and signatures (AMR_ABI_VERSION
 * of the build); a binding compares it with the header it was written for
 * and refuses a library built from other sources. No counterpart in the
 * paper. */
#define AMR_ABI_VERSION 11
int amr_abi_version(void);

/* ---- introspection (host only, no device needed) ------------------------ */

/* The Marching Cubes triangle table the kernels use (Sec. 5.1; generated by
 * the library from its face rule, not copied from any other table):
 *   count[256]      triangles per case (0..5)
 *   edges[256][15]  edge indices, 3 per triangle, unused entries 255.
 * Edge k joins hexahedron corners (a,b), a < b, listed in increasing (a,b)
 * order; corner e sits at (e & 1, (e >> 1) & 1, e >> 2). */
int amr_mc_table(uint8_t* count, uint8_t* edges);

/* Sizes of the context's resident state. */
typedef struct amr_info {
  int64_t n_cells;
  int64_t n_bricks;
  int64_t n_slots;      /* n_bricks * 2^(3 log2_brick) */
  int64_t n_dual;       /* -1 before amr_dual_cells */
  int32_t n_levels;     /* max level + 1 */
  int32_t log2_brick;
  int64_t device_bytes; /* device memory held by the context */
  int32_t placement;    /* how the last amr_build_locator placed the cells:
                           0 direct scatter, 1 binned */
  int32_t reserved;
} amr_info;
int amr_get_info(amr_ctx* ctx, amr_info* info);

/* Per-kernel device time (CUDA events on the context's stream) accumulated
 * since the last call, for the kernels listed by amr_kernel_name(0..n-1).
 * Timing is off until amr_enable_timing(ctx, 1). ms[] receives one value per
 * kernel, launches[] the number of launches (either may be NULL). Returns the
 * number of kernels. Synchronises the stream. */
int amr_enable_timing(amr_ctx* ctx, int on);
int amr_kernel_times(amr_ctx* ctx, double* ms, int64_t* launches, int n);
const char* amr_kernel_name(int k);

/* ---- extraction without device allocation -------------------------------- */

/* No counterpart in the paper: this entry point exists for callers that may
 * not allocate device memory themselves - for example code embedded in a
 * host application whose device memory belongs to another allocator, or
 * real-time code that cannot afford an allocation's latency or failure.
 * It runs the whole extraction (cell location, dual cells, Marching Cubes)
 * for a small data set with every intermediate buffer taken from one fixed
 * array of AMR_NOALLOC_SCRATCH_BYTES that the library reserves on each GPU
 * that loads it, for the life of the process. It calls no allocator.
 *   xyz, level, scalar  device arrays as in amr_upload, n <= AMR_NOALLOC_MAX_CELLS
 *   tris [cap][3][3]    device output as in amr_iso; *n_tris the exact count
 *                       (also on AMR_ERR_CAPACITY, when only cap were written)
 *   cuda_stream         stream for all work (NULL = legacy default stream)
 * Errors as amr_build_locator / amr_iso, plus AMR_ERR_RANGE when n exceeds
 * the limit, when the cells fill their 4^3 bricks to less than 1/8 on
 * average, or when more than 2 * AMR_NOALLOC_MAX_CELLS dual cells result.
 * The call synchronises the stream (it reads the counts back), so it cannot
 * be captured in a CUDA graph. The first call on a device also looks up the
 * array's device address (once per device, with that device current). All
 * calls share the array and each call resets what it uses, so calls that
 * overlap on the GPU (other host threads or streams) race. */
#define AMR_NOALLOC_MAX_CELLS 65536
#define AMR_NOALLOC_SCRATCH_BYTES (16u << 20)
int amr_extract_noalloc(const int32_t* xyz, const uint8_t* level,
                        const float* scalar, int64_t n, float iso, float* tris,
                        int64_t cap, int64_t* n_tris, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* AMRISO_H */
