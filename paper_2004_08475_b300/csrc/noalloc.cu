// amr_extract_noalloc: the whole extraction (cell location, dual cells,
// Marching Cubes) for a small data set without allocating any device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside a host
// application whose device memory is owned by another allocator, real-time
// code that may not take an allocation's latency or failure mode, or plugin
// code that must not change the process's memory footprint while it runs.
// For them, every intermediate buffer of the extraction lives in one
// fixed-size array in this file, reserved when the library's device code is
// loaded on a GPU and held by that GPU until the process exits.
//
// The array is shared by all calls. Each call re-initialises what it relies
// on (counters, the hash table, the slot occupancy); calls whose work
// overlaps on the GPU (other threads, other streams) race on it.

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "amriso.h"
#include "kernels.h"
#include "mc_table.h"

using namespace amriso;

namespace {

constexpr int kLogB = 2;                                // 4^3-cell bricks
constexpr long long kMaxCells = AMR_NOALLOC_MAX_CELLS;  // 65536
constexpr long long kHashCap = 2 * kMaxCells;           // power of two, load <= 0.5
constexpr long long kMaxSlots = 8 * kMaxCells;          // bricks at least 1/8 full
constexpr long long kMaxDuals = 2 * kMaxCells;

// Byte offsets of the pieces inside the scratch array (256-byte aligned).
constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffScratch = 0;
constexpr size_t kOffTable = align256(kOffScratch + sizeof(Scratch));
constexpr size_t kOffBricks = align256(kOffTable + kHashCap * 16);
constexpr size_t kOffRec = align256(kOffBricks + kMaxCells * 16);   // a brick holds >= 1 cell
constexpr size_t kOffScal = align256(kOffRec + kMaxSlots * 8);
constexpr size_t kOffView = align256(kOffScal + kMaxSlots * 4);
constexpr size_t kOffDuals = align256(kOffView + kMaxSlots * 4);
constexpr size_t kOffNbr = align256(kOffDuals + kMaxDuals * 32);
constexpr long long kMaxBricks = kMaxSlots >> (3 * kLogB);
constexpr size_t kScratchBytes = align256(kOffNbr + kMaxBricks * 27 * 4);
static_assert(kScratchBytes <= (size_t)AMR_NOALLOC_SCRATCH_BYTES, "scratch larger than advertised");

// The scratch itself. In host code this name is only a stand-in for the
// device symbol; kernels get the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

// Once per device, with that device current: the device address of the
// scratch array.
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return AMR_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return AMR_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return AMR_OK;
}

// The Marching Cubes table in kernel form, generated once per process (a
// function-local static: initialised on first use, thread-safe).
const McConst& table_const() {
  static const McConst table = [] {
    McTable t;
    make_mc_table(&t);
    McConst m;
    for (int c = 0; c < 256; ++c) {
      m.packed[c] = t.packed[c];
      m.count[c] = t.count[c];
    }
    m.edge_a = m.edge_b = 0;
    for (int k = 0; k < 12; ++k) {
      m.edge_a |= (unsigned long long)t.edge_a[k] << (4 * k);
      m.edge_b |= (unsigned long long)t.edge_b[k] << (4 * k);
    }
    return m;
  }();
  return table;
}

int rc_of(cudaError_t e) {
  if (e == cudaSuccess) return AMR_OK;
  cudaGetLastError();
  return AMR_ERR_CUDA;
}

int err_bits(unsigned e) {
  if (e & ERR_NONFINITE) return AMR_ERR_NONFINITE;
  if (e & ERR_RANGE) return AMR_ERR_RANGE;
  if (e & ERR_UNALIGNED) return AMR_ERR_UNALIGNED;
  if (e & ERR_DUPLICATE) return AMR_ERR_DUPLICATE;
  if (e & ERR_HASH_FULL) return AMR_ERR_RANGE;
  return AMR_OK;
}

#define NA_TRY(x)                  \
  do {                             \
    const int rc_ = (x);           \
    if (rc_ != AMR_OK) return rc_; \
  } while (0)

// Copies the counters back into a host stack variable and waits.
int read_counters(Scratch* dev_sc, Scratch* host, cudaStream_t st) {
  NA_TRY(rc_of(cudaMemcpyAsync(host, dev_sc, sizeof(Scratch), cudaMemcpyDeviceToHost, st)));
  return rc_of(cudaStreamSynchronize(st));
}

}  // namespace

extern "C" int amr_extract_noalloc(const int32_t* xyz, const uint8_t* level, const float* scalar,
                                   int64_t n, float iso, float* tris, int64_t cap, int64_t* n_tris,
                                   void* cuda_stream) {
  if (n < 0 || cap < 0 || !n_tris || (n > 0 && (!xyz || !level || !scalar)) || (cap > 0 && !tris))
    return AMR_ERR_INVALID_ARG;
  if (n > kMaxCells) return AMR_ERR_RANGE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* base = nullptr;
  NA_TRY(scratch_for_current_device(&base));
  Scratch* sc = reinterpret_cast<Scratch*>(base + kOffScratch);
  ulonglong2* htab = reinterpret_cast<ulonglong2*>(base + kOffTable);
  int4* bricks = reinterpret_cast<int4*>(base + kOffBricks);
  unsigned long long* rec = reinterpret_cast<unsigned long long*>(base + kOffRec);
  float* scal = reinterpret_cast<float*>(base + kOffScal);
  unsigned* view = reinterpret_cast<unsigned*>(base + kOffView);
  uint4* duals = reinterpret_cast<uint4*>(base + kOffDuals);
  int* nbr = reinterpret_cast<int*>(base + kOffNbr);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  // counters and bounds start fresh; the hash table starts empty
  Scratch h;
  std::memset(&h, 0, sizeof(h));
  for (int a = 0; a < 3; ++a) {
    h.lo[a] = INT_MAX;
    h.hi[a] = INT_MIN;
  }
  NA_TRY(rc_of(cudaMemcpyAsync(sc, &h, sizeof(Scratch), cudaMemcpyHostToDevice, st)));
  NA_TRY(rc_of(cudaMemsetAsync(htab, 0xFF, kHashCap * 16, st)));
  const int block = 256;
  const int grid_cells = (int)std::max(1ll, std::min((long long)(n + block - 1) / block, (long long)sms * 8));
  if (n > 0)
    NA_TRY(rc_of(launch_insert_bricks(kLogB, xyz, level, scalar, n, htab, kHashCap - 1, bricks,
                                      kMaxCells, sc, grid_cells, block, nullptr, st)));
  NA_TRY(read_counters(sc, &h, st));
  NA_TRY(err_bits(h.err));
  const long long n_bricks = (long long)h.n_bricks;
  const long long n_slots = n_bricks << (3 * kLogB);
  if (n_slots > kMaxSlots) return AMR_ERR_RANGE;   // bricks too sparsely filled
  for (int a = 0; a < 3 && n > 0; ++a)
    if ((long long)h.hi[a] - (long long)h.lo[a] >= (1ll << 21) || h.lo[a] < -(1 << 30) ||
        h.hi[a] > (1 << 30))
      return AMR_ERR_RANGE;

  Locator L;
  L.htab = htab;
  L.hmask = kHashCap - 1;
  L.bricks = bricks;
  L.rec = rec;
  L.scal = scal;
  L.view = view;
  L.levels = n > 0 ? h.max_level + 1 : 0;
  long long nd = 0;
  if (n_slots > 0) {
    NA_TRY(rc_of(cudaMemsetAsync(rec, 0xFF, (size_t)n_slots * 8, st)));
    NA_TRY(rc_of(launch_scatter_cells(kLogB, xyz, level, scalar, n, L, rec, sc, grid_cells, block, st)));
    const int grid_slots = (int)std::max(1ll, std::min((n_slots + block - 1) / block, (long long)sms * 8));
    NA_TRY(rc_of(launch_resolve_views(kLogB, L, view, scal, n_slots, 0, sc, grid_slots, block, st)));
    const int grid_nb = (int)std::max(1ll, std::min((n_bricks * 27 + block - 1) / block, (long long)sms * 8));
    NA_TRY(rc_of(launch_brick_neighbors(kLogB, L, n_bricks, nbr, grid_nb, st)));
    NA_TRY(rc_of(launch_dual_cells(kLogB, L, nbr, nullptr, n_bricks, duals, kMaxDuals, sc, st)));
    NA_TRY(read_counters(sc, &h, st));
    NA_TRY(err_bits(h.err));
    if ((long long)h.n_occupied != n) return AMR_ERR_DUPLICATE;   // two cells shared a slot
    nd = (long long)h.n_dual;
    if (nd > kMaxDuals) return AMR_ERR_RANGE;
  }
  long long nt = 0;
  if (nd > 0) {
    const McConst& mc = table_const();
    const int grid_d = (int)std::max(1ll, std::min((nd + 255) / 256, (long long)sms * 8));
    NA_TRY(rc_of(launch_mc(kLogB, L, duals, nd, iso, tris, cap, &sc->n_tri[0], nullptr, nullptr, mc, grid_d,
                           st)));
    NA_TRY(read_counters(sc, &h, st));
    NA_TRY(err_bits(h.err));
    nt = (long long)h.n_tri[0];
  }
  *n_tris = nt;
  return nt > cap ? AMR_ERR_CAPACITY : AMR_OK;
}
