// C ABI of libamriso (declared in include/amriso.h): contexts, device memory,
// stream-ordered launch sequences and error mapping around the kernels.

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "amriso.h"
#include "attributes.h"
#include "kernels.h"
#include "shapes.h"
#include "mc_table.h"
#include "order.h"

using namespace amriso;

namespace {

// Inputs from this many cells on are placed by the binned passes (the direct
// scatter is bound by one store transaction per cell).
constexpr long long kBinnedMinCells = 1ll << 20;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

enum KernelId {
  KT_INSERT = 0, KT_SCATTER, KT_RESOLVE, KT_DUAL, KT_MC, KT_MC_CASES, KT_BATCH_COUNT, KT_BATCH_EMIT,
  KT_GET_DUALS, KT_NEIGHBORS, KT_BIN, KT_PLACE, KT_DUAL_ISO, KT_BIN_FINE, KT_MC_KEYS, KT_WELD_INSERT,
  KT_WELD_INDEX, KT_INTERPOLATE, KT_SHAPES, KT_ORDER_COUNT, KT_ORDER_SCAN, KT_ORDER_SCATTER, KT_MC_TAGGED,
  KT_RESOLVE_EMPTY, KT_BATCH_SCAN, KT_COUNT
};
const char* const kKernelNames[KT_COUNT] = {
    "k_insert_bricks", "k_scatter_cells", "k_resolve_views", "k_dual_cells", "k_mc",
    "k_mc_cases",      "k_batch_count", "k_batch_emit", "k_get_duals", "k_brick_neighbors",
    "k_bin_coarse", "k_place_windows", "k_dual_cells_iso", "k_bin_fine", "k_mc_keys", "k_weld_insert",
    "k_weld_index", "k_interpolate", "k_dual_shapes", "k_order_count", "k_order_scan", "k_order_scatter",
    "k_mc_tagged", "k_resolve_empty", "k_batch_scan"};

const McTable& host_table() {
  static McTable t = [] {
    McTable x;
    make_mc_table(&x);
    return x;
  }();
  return t;
}

McConst make_mc_const() {
  const McTable& t = host_table();
  McConst m;
  for (int c = 0; c < 256; ++c) {
    m.packed[c] = t.packed[c];
    m.count[c] = t.count[c];
  }
  m.edge_a = 0;
  m.edge_b = 0;
  for (int k = 0; k < 12; ++k) {
    m.edge_a |= (unsigned long long)t.edge_a[k] << (4 * k);
    m.edge_b |= (unsigned long long)t.edge_b[k] << (4 * k);
  }
  return m;
}

}  // namespace

struct amr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // the locator build's second stream: neighbours and brick order (they
  // need only the brick table) run beside the placement of the cells
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int sm_count = 148;
  // input (borrowed or owned)
  long long n = 0;
  const int* xyz = nullptr;
  const unsigned char* lvl = nullptr;
  const float* s = nullptr;
  DevBuf own_xyz, own_lvl, own_s;
  int stage = 0;  // 0 empty, 1 uploaded, 2 locator, 3 dual cells
  // locator
  int logb = 3;
  float alpha = 0.5f;
  int block = 256;
  int check_overlap = 0;
  DevBuf htab, bricks, rec, scal, view, nbr;
  DevBuf staging, codes, elist;   // binned placement workspace
  DevBuf border, bcount;   // bricks in spatial order (the dual pass's visiting order), bucket counters
  int placement = 0;   // 0 direct scatter, 1 binned
  unsigned long long hcap = 0;
  long long n_bricks = 0, n_slots = 0;
  int levels = 0;
  // dual cells
  DevBuf duals;
  long long dual_cap = 0, n_dual = -1;
  // scratch
  DevBuf scratch;
  Scratch* host_sc = nullptr;  // pinned mirror
  DevBuf stage_buf, iso_buf, seg_buf;
  DevBuf bwork;   // batched iso-values: per-tile counters and row offsets for up to kMaxIso values
  DevBuf tkeys, wtab, ostage;   // indexed face set: triangle edge keys, weld table, host-delivery staging
  long long tkeys_cap = 0;
  McConst mc;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[KT_COUNT];
  double ms_acc[KT_COUNT] = {0};
  long long launches[KT_COUNT] = {0};
};

namespace {

size_t held(const DevBuf& b) { return b.bytes; }

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

int ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (b.bytes >= bytes) return AMR_OK;
  release(b);
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return AMR_ERR_OOM;
  }
  b.bytes = bytes;
  return AMR_OK;
}

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return AMR_OK;
  if (e == cudaErrorMemoryAllocation) return AMR_ERR_OOM;
  return AMR_ERR_CUDA;
}

#define AMR_TRY(x)                 \
  do {                             \
    const int rc_ = (x);           \
    if (rc_ != AMR_OK) return rc_; \
  } while (0)

#define AMR_CUDA(x) AMR_TRY(cuda_rc(x))

cudaEvent_t take_event(amr_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Records an event pair around one kernel launch when timing is on.
struct KernelTimer {
  amr_ctx* c;
  int k;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  KernelTimer(amr_ctx* c_, int k_, cudaStream_t st_ = nullptr) : c(c_), k(k_), st(st_ ? st_ : c_->stream) {
    if (c->timing) {
      a = take_event(c);
      b = take_event(c);
      cudaEventRecord(a, st);
    }
  }
  ~KernelTimer() {
    if (c->timing) {
      cudaEventRecord(b, st);
      c->pending[k].push_back({a, b});
      c->launches[k]++;
    }
  }
};

Scratch* dev_sc(amr_ctx* c) { return static_cast<Scratch*>(c->scratch.p); }

// The context's second stream and its fork/join events, made on first use
// (on the context's device, current here).
int side_stream(amr_ctx* c) {
  if (!c->side) AMR_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  if (!c->ev_fork) AMR_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  if (!c->ev_join) AMR_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  return AMR_OK;
}

// Resets the device scratch counters (stream-ordered).
int reset_scratch(amr_ctx* c) {
  Scratch& h = *c->host_sc;
  std::memset(&h, 0, sizeof(Scratch));
  for (int a = 0; a < 3; ++a) {
    h.lo[a] = INT_MAX;
    h.hi[a] = INT_MIN;
  }
  AMR_CUDA(cudaMemcpyAsync(dev_sc(c), &h, sizeof(Scratch), cudaMemcpyHostToDevice, c->stream));
  return AMR_OK;
}

int read_scratch(amr_ctx* c) {
  AMR_CUDA(cudaMemcpyAsync(c->host_sc, dev_sc(c), sizeof(Scratch), cudaMemcpyDeviceToHost, c->stream));
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  return AMR_OK;
}

int err_code(unsigned e) {
  if (e & ERR_NONFINITE) return AMR_ERR_NONFINITE;
  if (e & ERR_RANGE) return AMR_ERR_RANGE;
  if (e & ERR_UNALIGNED) return AMR_ERR_UNALIGNED;
  if (e & ERR_DUPLICATE) return AMR_ERR_DUPLICATE;
  if (e & ERR_OVERLAP) return AMR_ERR_OVERLAP;
  if (e & ERR_HASH_FULL) return AMR_ERR_CAPACITY;
  return AMR_OK;
}

Locator make_locator(amr_ctx* c) {
  Locator L;
  L.htab = static_cast<const ulonglong2*>(c->htab.p);
  L.hmask = c->hcap - 1;
  L.bricks = static_cast<const int4*>(c->bricks.p);
  L.rec = static_cast<const unsigned long long*>(c->rec.p);
  L.scal = static_cast<const float*>(c->scal.p);
  L.view = static_cast<const unsigned*>(c->view.p);
  L.levels = c->levels;
  return L;
}

int grid_for(amr_ctx* c, long long items, int block, int per_sm) {
  const long long want = (items + block - 1) / block;
  const long long cap = (long long)c->sm_count * per_sm;
  return (int)std::max(1ll, std::min(want, cap));
}

unsigned long long pow2_at_least(unsigned long long v) {
  unsigned long long p = 1024;
  while (p < v) p <<= 1;
  return p;
}

// Copies a Marching Cubes launch's triangle counter back and waits.
int mc_result(amr_ctx* c, const unsigned long long* counter, long long* nt) {
  AMR_CUDA(cudaMemcpyAsync(&c->host_sc->n_tri[0], counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           c->stream));
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  *nt = (long long)c->host_sc->n_tri[0];
  return AMR_OK;
}

// Copies `bytes` from device `src` to `dst` (device or host per flags).
int deliver(amr_ctx* c, void* dst, const void* src, size_t bytes, int flags) {
  if (bytes == 0 || dst == src) return AMR_OK;
  const cudaMemcpyKind kind = (flags & AMR_HOST_PTRS) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  AMR_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, c->stream));
  return AMR_OK;
}

}  // namespace

extern "C" {

int amr_abi_version(void) { return AMR_ABI_VERSION; }

const char* amr_strerror(int code) {
  switch (code) {
    case AMR_OK: return "ok";
    case AMR_ERR_INVALID_ARG: return "invalid argument";
    case AMR_ERR_UNALIGNED: return "lower corner not a multiple of the cell width";
    case AMR_ERR_RANGE: return "level, extent or size out of range";
    case AMR_ERR_NONFINITE: return "non-finite scalar";
    case AMR_ERR_DUPLICATE: return "duplicate cell";
    case AMR_ERR_OVERLAP: return "cell inside a coarser cell";
    case AMR_ERR_STATE: return "call out of order";
    case AMR_ERR_OOM: return "device out of memory";
    case AMR_ERR_CAPACITY: return "output capacity exceeded";
    case AMR_ERR_TIMEOUT: return "bounded device wait timed out (reserved)";
    case AMR_ERR_CUDA: return "CUDA runtime error";
    default: return "unknown error";
  }
}

int amr_mc_table(uint8_t* count, uint8_t* edges) {
  if (!count && !edges) return AMR_ERR_INVALID_ARG;
  const McTable& t = host_table();
  if (count) std::memcpy(count, t.count, 256);
  if (edges) std::memcpy(edges, t.edges, 256 * 15);
  return AMR_OK;
}

int amr_create(amr_ctx** out, int device, void* cuda_stream) {
  if (!out) return AMR_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return AMR_ERR_INVALID_ARG;
  }
  AMR_CUDA(cudaSetDevice(device));
  amr_ctx* c = new (std::nothrow) amr_ctx();
  if (!c) return AMR_ERR_OOM;
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cudaMallocHost(reinterpret_cast<void**>(&c->host_sc), sizeof(Scratch)) != cudaSuccess ||
      ensure(c->scratch, sizeof(Scratch)) != AMR_OK) {
    cudaGetLastError();
    amr_destroy(c);
    return AMR_ERR_OOM;
  }
  c->mc = make_mc_const();
  *out = c;
  return AMR_OK;
}

void amr_destroy(amr_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  DevBuf* bufs[] = {&c->own_xyz, &c->own_lvl, &c->own_s, &c->htab, &c->bricks,
                    &c->rec, &c->scal, &c->view, &c->nbr, &c->staging, &c->codes,
                    &c->elist, &c->duals, &c->scratch,
                    &c->stage_buf, &c->iso_buf, &c->seg_buf, &c->bwork, &c->tkeys, &c->wtab,
                    &c->ostage, &c->border, &c->bcount};
  for (DevBuf* b : bufs) release(*b);
  if (c->host_sc) cudaFreeHost(c->host_sc);
  for (auto& v : c->pending)
    for (auto& p : v) {
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
}

int amr_set_stream(amr_ctx* c, void* cuda_stream) {
  if (!c) return AMR_ERR_INVALID_ARG;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  return AMR_OK;
}

int amr_sync(amr_ctx* c) {
  if (!c) return AMR_ERR_INVALID_ARG;
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  return AMR_OK;
}

int amr_trim(amr_ctx* c) {
  if (!c) return AMR_ERR_INVALID_ARG;
  AMR_CUDA(cudaSetDevice(c->device));
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  release(c->staging);
  release(c->codes);
  release(c->elist);
  release(c->stage_buf);
  release(c->tkeys);
  release(c->wtab);
  release(c->ostage);
  release(c->bcount);
  c->tkeys_cap = 0;
  return AMR_OK;
}

int amr_upload(amr_ctx* c, const int32_t* xyz, const uint8_t* level, const float* scalar, int64_t n,
               int flags) {
  if (!c || n < 0 || (n > 0 && (!xyz || !level || !scalar))) return AMR_ERR_INVALID_ARG;
  if (n > INT_MAX) return AMR_ERR_RANGE;
  AMR_CUDA(cudaSetDevice(c->device));
  c->stage = 0;
  c->n_dual = -1;
  c->n = n;
  if (flags & (AMR_HOST_PTRS | AMR_COPY)) {
    AMR_TRY(ensure(c->own_xyz, (size_t)n * 12));
    AMR_TRY(ensure(c->own_lvl, (size_t)n));
    AMR_TRY(ensure(c->own_s, (size_t)n * 4));
    const cudaMemcpyKind kind = (flags & AMR_HOST_PTRS) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (n) {
      AMR_CUDA(cudaMemcpyAsync(c->own_xyz.p, xyz, (size_t)n * 12, kind, c->stream));
      AMR_CUDA(cudaMemcpyAsync(c->own_lvl.p, level, (size_t)n, kind, c->stream));
      AMR_CUDA(cudaMemcpyAsync(c->own_s.p, scalar, (size_t)n * 4, kind, c->stream));
    }
    c->xyz = static_cast<const int*>(c->own_xyz.p);
    c->lvl = static_cast<const unsigned char*>(c->own_lvl.p);
    c->s = static_cast<const float*>(c->own_s.p);
  } else {
    c->xyz = xyz;
    c->lvl = level;
    c->s = scalar;
  }
  c->stage = 1;
  return AMR_OK;
}

int amr_build_locator(amr_ctx* c, const amr_locator_opts* opts) {
  if (!c) return AMR_ERR_INVALID_ARG;
  if (c->stage < 1) return AMR_ERR_STATE;
  AMR_CUDA(cudaSetDevice(c->device));
  int logb = 3, block = 256, overlap = 0, partitioned = 0;
  float alpha = 0.5f;
  if (opts) {
    if (opts->log2_brick) logb = opts->log2_brick;
    if (opts->load_factor > 0.f) alpha = opts->load_factor;
    if (opts->block_size) block = opts->block_size;
    overlap = opts->check_overlap;
    partitioned = opts->partitioned;
  }
  if ((logb != 2 && logb != 3) || alpha < 0.05f || alpha > 0.9f || block < 32 || block > 1024 ||
      (block & 31))
    return AMR_ERR_INVALID_ARG;
  c->logb = logb;
  c->alpha = alpha;
  c->block = block;
  c->check_overlap = overlap;
  c->stage = 1;
  c->n_dual = -1;
  const long long n = c->n;
  const int B3 = 1 << (3 * logb);
  // Table size: bricks expected at least 1/4 full, but start no larger than
  // 2^22 entries (64 MB) so the table stays in L2 while every cell probes
  // it. A table that fills up stops the insert early and is rebuilt larger.
  unsigned long long want = (unsigned long long)((double)(n * 4 / B3 + 64) / alpha);
  want = std::min<unsigned long long>(want, 1ull << 22);
  const bool binned = partitioned > 0 || (partitioned == 0 && n >= kBinnedMinCells);
  unsigned* codes = nullptr;   // binned placement: each cell's table entry, recorded by the insert pass
  OrderFrame frame{};          // bucket frame of the bricks' spatial order (from the bounding box)
  for (int attempt = 0;; ++attempt) {
    c->hcap = pow2_at_least(want);
    codes = nullptr;
    if (binned && n > 0 && c->hcap <= (1ull << (31 - 3 * logb))) {   // codes: slot or table entry below 2^31
      AMR_TRY(ensure(c->codes, (size_t)n * 4));
      codes = static_cast<unsigned*>(c->codes.p);
    }
    const unsigned long long limit =
        (unsigned long long)((double)c->hcap * std::min(0.85, 2.0 * (double)alpha));
    AMR_TRY(ensure(c->htab, c->hcap * 16));
    AMR_TRY(ensure(c->bricks, c->hcap * 16));
    AMR_CUDA(cudaMemsetAsync(c->htab.p, 0xFF, c->hcap * 16, c->stream));
    AMR_TRY(reset_scratch(c));
    if (n > 0) {
      KernelTimer kt(c, KT_INSERT);
      AMR_CUDA(launch_insert_bricks(logb, c->xyz, c->lvl, c->s, n,
                                    static_cast<ulonglong2*>(c->htab.p), c->hcap - 1,
                                    static_cast<int4*>(c->bricks.p), limit, dev_sc(c),
                                    grid_for(c, n, block, 2048 / block), block, codes, c->stream));
    }
    AMR_TRY(read_scratch(c));
    const Scratch& h = *c->host_sc;
    const unsigned full = h.err & ERR_HASH_FULL;
    const int rc = err_code(h.err & ~ERR_HASH_FULL);
    if (rc != AMR_OK) return rc;
    if (full) {
      if (attempt >= 4) return AMR_ERR_RANGE;
      want = (unsigned long long)(std::max<double>((double)h.n_bricks, (double)c->hcap) * 4.0 / alpha);
      continue;
    }
    c->n_bricks = (long long)h.n_bricks;
    c->levels = n > 0 ? h.max_level + 1 : 0;
    for (int a = 0; a < 3 && n > 0; ++a)
      if ((long long)h.hi[a] - (long long)h.lo[a] >= (1ll << 21) || h.lo[a] < -(1 << 30) ||
          h.hi[a] > (1 << 30))
        return AMR_ERR_RANGE;
    if (n > 0) frame = order_frame(h.lo, h.hi);
    break;
  }
  c->n_slots = c->n_bricks * B3;
  if (c->n_slots >= (long long)INT_MAX) return AMR_ERR_RANGE;
  AMR_TRY(ensure(c->rec, (size_t)c->n_slots * 8));
  AMR_TRY(ensure(c->scal, (size_t)c->n_slots * 4));
  AMR_TRY(ensure(c->view, (size_t)c->n_slots * 4));
  const bool binned_ok = binned && codes != nullptr;
  if (c->n_slots) {
    // neighbours and the brick order need only the brick table and the
    // bricks: they run on the side stream while the cells are placed
    AMR_TRY(ensure(c->nbr, (size_t)c->n_bricks * 27 * 4));
    AMR_TRY(ensure(c->border, (size_t)c->n_bricks * 4));
    AMR_TRY(ensure(c->bcount, (size_t)kOrderBuckets * 4));
    AMR_TRY(side_stream(c));
    AMR_CUDA(cudaEventRecord(c->ev_fork, c->stream));
    AMR_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    const Locator Lt = make_locator(c);
    {
      KernelTimer kt(c, KT_NEIGHBORS, c->side);
      AMR_CUDA(launch_brick_neighbors(logb, Lt, c->n_bricks, static_cast<int*>(c->nbr.p),
                                      grid_for(c, c->n_bricks * 27, 256, 8), c->side));
    }
    // the dual pass visits the bricks bucket by bucket along a Morton curve
    unsigned* cnt = static_cast<unsigned*>(c->bcount.p);
    AMR_CUDA(cudaMemsetAsync(cnt, 0, (size_t)kOrderBuckets * 4, c->side));
    {
      KernelTimer kt(c, KT_ORDER_COUNT, c->side);
      AMR_CUDA(launch_brick_order_count(Lt.bricks, c->n_bricks, frame, cnt, grid_for(c, c->n_bricks, 256, 8),
                                        c->side));
    }
    {
      KernelTimer kt(c, KT_ORDER_SCAN, c->side);
      AMR_CUDA(launch_brick_order_scan(cnt, c->side));
    }
    {
      KernelTimer kt(c, KT_ORDER_SCATTER, c->side);
      AMR_CUDA(launch_brick_order_scatter(Lt.bricks, c->n_bricks, frame, cnt, static_cast<int*>(c->border.p),
                                          grid_for(c, c->n_bricks, 256, 8), c->side));
    }
    AMR_CUDA(cudaEventRecord(c->ev_join, c->side));
    // binned placement unless asked otherwise or the input is small; it
    // needs the insert pass's cell codes, so a table too large for them
    // (after rebuilds) falls back to the direct scatter
    c->placement = binned_ok ? 1 : 0;
    if (binned_ok) {
      AMR_TRY(ensure(c->staging, bin_layout(c->n_slots).bytes));
      AMR_TRY(ensure(c->elist, (size_t)c->n_bricks * 4));
      const Locator L0 = make_locator(c);
      {
        KernelTimer kt(c, KT_BIN);
        AMR_CUDA(launch_bin_coarse(logb, c->s, n, L0, c->n_slots, c->staging.p, dev_sc(c), c->sm_count, codes,
                                   c->stream));
      }
      {
        KernelTimer kt(c, KT_BIN_FINE);
        AMR_CUDA(launch_bin_fine(c->n_slots, c->staging.p, dev_sc(c), c->stream));
      }
      KernelTimer kt(c, KT_PLACE);
      AMR_CUDA(launch_place_windows(logb, c->n_slots, c->staging.p, static_cast<unsigned long long*>(c->rec.p),
                                    static_cast<unsigned*>(c->view.p), static_cast<float*>(c->scal.p),
                                    static_cast<unsigned*>(c->elist.p), dev_sc(c), c->stream));
    } else {
      AMR_CUDA(cudaMemsetAsync(c->rec.p, 0xFF, (size_t)c->n_slots * 8, c->stream));
      KernelTimer kt(c, KT_SCATTER);
      AMR_CUDA(launch_scatter_cells(logb, c->xyz, c->lvl, c->s, n, make_locator(c),
                                    static_cast<unsigned long long*>(c->rec.p), dev_sc(c),
                                    grid_for(c, n, block, 2048 / block), block, c->stream));
    }
    const Locator L = make_locator(c);
    if (binned_ok && !overlap) {   // only the bricks with empty slots are left to resolve
      KernelTimer kt(c, KT_RESOLVE_EMPTY);
      AMR_CUDA(launch_resolve_empty(logb, L, static_cast<const unsigned*>(c->elist.p), dev_sc(c),
                                    static_cast<unsigned*>(c->view.p), c->sm_count * 8, c->stream));
    } else {   // every slot (and, on request, every occupied slot checked against coarser cells)
      if (binned_ok)   // the window pass counted the occupied slots already
        AMR_CUDA(cudaMemsetAsync(&dev_sc(c)->n_occupied, 0, sizeof(unsigned long long), c->stream));
      KernelTimer kt(c, KT_RESOLVE);
      AMR_CUDA(launch_resolve_views(logb, L, static_cast<unsigned*>(c->view.p), static_cast<float*>(c->scal.p),
                                    c->n_slots, overlap, dev_sc(c), grid_for(c, c->n_slots, block, 2048 / block),
                                    block, c->stream));
    }
    AMR_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    AMR_TRY(read_scratch(c));
    const int rc = err_code(c->host_sc->err);
    if (rc != AMR_OK) return rc;
    if ((long long)c->host_sc->n_occupied != n) return AMR_ERR_DUPLICATE;  // two cells, one slot
  }
  c->stage = 2;
  return AMR_OK;
}

namespace {
int dual_cells_owned(amr_ctx* c, int x0, int x1, int64_t* n_dual);
}

int amr_dual_cells(amr_ctx* c, int64_t* n_dual) { return dual_cells_owned(c, INT_MIN, INT_MAX, n_dual); }

int amr_dual_cells_owned(amr_ctx* c, int32_t x_begin, int32_t x_end, int64_t* n_dual) {
  if (x_end < x_begin) return AMR_ERR_INVALID_ARG;
  return dual_cells_owned(c, x_begin, x_end, n_dual);
}

namespace {
int dual_cells_owned(amr_ctx* c, int x0, int x1, int64_t* n_dual) {
  if (!c || !n_dual) return AMR_ERR_INVALID_ARG;
  if (c->stage < 2) return AMR_ERR_STATE;
  AMR_CUDA(cudaSetDevice(c->device));
  long long cap = std::max(c->dual_cap, c->n + c->n / 4 + 1024);
  AMR_TRY(ensure(c->iso_buf, sizeof(float) * kMaxIso));
  AMR_TRY(ensure(c->seg_buf, sizeof(long long) * (kMaxIso + 1)));
  for (int attempt = 0; attempt < 2; ++attempt) {
    AMR_TRY(ensure(c->duals, (size_t)cap * 32));
    c->dual_cap = (long long)(c->duals.bytes / 32);
    AMR_CUDA(cudaMemsetAsync(&dev_sc(c)->n_dual, 0, sizeof(unsigned long long), c->stream));
    {
      KernelTimer kt(c, KT_DUAL);
      AMR_CUDA(launch_dual_cells(c->logb, make_locator(c), static_cast<const int*>(c->nbr.p),
                                 static_cast<const int*>(c->border.p), c->n_bricks, static_cast<uint4*>(c->duals.p),
                                 c->dual_cap, dev_sc(c), c->stream, x0, x1));
    }
    AMR_CUDA(cudaMemcpyAsync(&c->host_sc->n_dual, &dev_sc(c)->n_dual, sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c->stream));
    AMR_CUDA(cudaStreamSynchronize(c->stream));
    const long long nd = (long long)c->host_sc->n_dual;
    if (nd <= c->dual_cap) {
      c->n_dual = nd;
      AMR_TRY(ensure(c->bwork, batch_workspace_bytes((nd + batch_tile(nd) - 1) / batch_tile(nd) * kMaxIso)));
      c->stage = 3;
      *n_dual = nd;
      return AMR_OK;
    }
    cap = nd;  // exact count known: grow and run again
  }
  return AMR_ERR_CUDA;
}
}  // namespace

int amr_dual_cells_iso(amr_ctx* c, float iso, float* tris, int64_t cap, int64_t* n_dual, int64_t* n_tris,
                       int flags) {
  if (!c || !n_dual || !n_tris || cap < 0 || (cap > 0 && !tris)) return AMR_ERR_INVALID_ARG;
  if (c->stage < 2) return AMR_ERR_STATE;
  AMR_CUDA(cudaSetDevice(c->device));
  float* dst = tris;
  if ((flags & AMR_HOST_PTRS) && cap > 0) {
    AMR_TRY(ensure(c->stage_buf, (size_t)cap * 36));
    dst = static_cast<float*>(c->stage_buf.p);
  }
  long long dcap = std::max(c->dual_cap, c->n + c->n / 4 + 1024);
  AMR_TRY(ensure(c->iso_buf, sizeof(float) * kMaxIso));
  AMR_TRY(ensure(c->seg_buf, sizeof(long long) * (kMaxIso + 1)));
  for (int attempt = 0; attempt < 2; ++attempt) {
    AMR_TRY(ensure(c->duals, (size_t)dcap * 32));
    c->dual_cap = (long long)(c->duals.bytes / 32);
    AMR_CUDA(cudaMemsetAsync(&dev_sc(c)->n_dual, 0, sizeof(unsigned long long), c->stream));
    AMR_CUDA(cudaMemsetAsync(&dev_sc(c)->n_tri[0], 0, sizeof(unsigned long long), c->stream));
    {
      KernelTimer kt(c, KT_DUAL_ISO);
      AMR_CUDA(launch_dual_cells_iso(c->logb, make_locator(c), static_cast<const int*>(c->nbr.p),
                                     static_cast<const int*>(c->border.p), c->n_bricks,
                                     static_cast<uint4*>(c->duals.p), c->dual_cap, dev_sc(c), iso, dst, cap,
                                     c->mc, c->stream));
    }
    AMR_CUDA(cudaMemcpyAsync(&c->host_sc->n_dual, &dev_sc(c)->n_dual, sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c->stream));
    AMR_CUDA(cudaMemcpyAsync(&c->host_sc->n_tri[0], &dev_sc(c)->n_tri[0], sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c->stream));
    AMR_CUDA(cudaStreamSynchronize(c->stream));
    const long long nd = (long long)c->host_sc->n_dual;
    if (nd > c->dual_cap) {
      dcap = nd;   // exact count known: grow and run again
      continue;
    }
    const long long nt = (long long)c->host_sc->n_tri[0];
    c->n_dual = nd;
    AMR_TRY(ensure(c->bwork, batch_workspace_bytes((nd + batch_tile(nd) - 1) / batch_tile(nd) * kMaxIso)));
    c->stage = 3;
    *n_dual = nd;
    *n_tris = nt;
    if (flags & AMR_HOST_PTRS) {
      AMR_TRY(deliver(c, tris, dst, (size_t)std::min<long long>(nt, cap) * 36, flags));
      AMR_CUDA(cudaStreamSynchronize(c->stream));
    }
    return nt > cap ? AMR_ERR_CAPACITY : AMR_OK;
  }
  return AMR_ERR_CUDA;
}

int amr_get_duals(amr_ctx* c, int32_t* out, int64_t cap, int flags) {
  if (!c || (!out && cap > 0) || cap < 0) return AMR_ERR_INVALID_ARG;
  if (c->stage < 3) return AMR_ERR_STATE;
  if (cap < c->n_dual) return AMR_ERR_CAPACITY;
  AMR_CUDA(cudaSetDevice(c->device));
  if (c->n_dual == 0) return AMR_OK;
  const size_t bytes = (size_t)c->n_dual * 32;
  int* dst = reinterpret_cast<int*>(out);
  if (flags & AMR_HOST_PTRS) {
    AMR_TRY(ensure(c->stage_buf, bytes));
    dst = static_cast<int*>(c->stage_buf.p);
  }
  {
    KernelTimer kt(c, KT_GET_DUALS);
    AMR_CUDA(launch_get_duals(static_cast<const uint4*>(c->duals.p), c->n_dual,
                              static_cast<const unsigned long long*>(c->rec.p), dst,
                              grid_for(c, 2 * c->n_dual, 256, 8),
                              c->stream));
  }
  AMR_TRY(deliver(c, out, dst, bytes, flags));
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  return AMR_OK;
}

int amr_iso(amr_ctx* c, float iso, float* tris, int64_t cap, int64_t* n_tris, int flags) {
  if (!c || !n_tris || cap < 0 || (cap > 0 && !tris)) return AMR_ERR_INVALID_ARG;
  if (c->stage < 3) return AMR_ERR_STATE;
  AMR_CUDA(cudaSetDevice(c->device));
  float* dst = tris;
  if ((flags & AMR_HOST_PTRS) && cap > 0) {
    AMR_TRY(ensure(c->stage_buf, (size_t)cap * 36));
    dst = static_cast<float*>(c->stage_buf.p);
  }
  unsigned long long* counter = &dev_sc(c)->n_tri[0];
  AMR_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), c->stream));
  {
    KernelTimer kt(c, KT_MC);
    AMR_CUDA(launch_mc(c->logb, make_locator(c), static_cast<const uint4*>(c->duals.p), c->n_dual, iso, dst,
                       cap, counter, nullptr, nullptr, c->mc, grid_for(c, c->n_dual, 256, 8),
                       c->stream));
  }
  long long nt = 0;
  AMR_TRY(mc_result(c, counter, &nt));
  *n_tris = nt;
  if (flags & AMR_HOST_PTRS) {
    AMR_TRY(deliver(c, tris, dst, (size_t)std::min<long long>(nt, cap) * 36, flags));
    AMR_CUDA(cudaStreamSynchronize(c->stream));
  }
  return nt > cap ? AMR_ERR_CAPACITY : AMR_OK;
}

int amr_iso_tagged(amr_ctx* c, float iso, float* tris, int64_t* tri_dual, int64_t cap, int64_t* n_tris,
                   int flags) {
  if (!c || !n_tris || cap < 0 || (cap > 0 && (!tris || !tri_dual))) return AMR_ERR_INVALID_ARG;
  if (c->stage < 3) return AMR_ERR_STATE;
  AMR_CUDA(cudaSetDevice(c->device));
  float* dst = tris;
  long long* dtag = reinterpret_cast<long long*>(tri_dual);
  const bool host = (flags & AMR_HOST_PTRS) != 0;
  if (host && cap > 0) {
    AMR_TRY(ensure(c->stage_buf, (size_t)cap * 44));
    dst = static_cast<float*>(c->stage_buf.p);
    dtag = reinterpret_cast<long long*>(static_cast<unsigned char*>(c->stage_buf.p) + (size_t)cap * 36);
  }
  unsigned long long* counter = &dev_sc(c)->n_tri[0];
  AMR_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), c->stream));
  if (cap > 0) {   // without an output there is nothing to tag: count only
    KernelTimer kt(c, KT_MC_TAGGED);
    AMR_CUDA(launch_mc(c->logb, make_locator(c), static_cast<const uint4*>(c->duals.p), c->n_dual, iso, dst, cap,
                       counter, nullptr, nullptr, c->mc, grid_for(c, c->n_dual, 256, 8), c->stream,
                       dtag));
  } else {
    KernelTimer kt(c, KT_MC);
    AMR_CUDA(launch_mc(c->logb, make_locator(c), static_cast<const uint4*>(c->duals.p), c->n_dual, iso, nullptr,
                       0, counter, nullptr, nullptr, c->mc, grid_for(c, c->n_dual, 256, 8),
                       c->stream));
  }
  long long nt = 0;
  AMR_TRY(mc_result(c, counter, &nt));
  *n_tris = nt;
  if (host && cap > 0) {
    const size_t w = (size_t)std::min<long long>(nt, cap);
    AMR_TRY(deliver(c, tris, dst, w * 36, flags));
    AMR_TRY(deliver(c, tri_dual, dtag, w * 8, flags));
    AMR_CUDA(cudaStreamSynchronize(c->stream));
  }
  return nt > cap ? AMR_ERR_CAPACITY : AMR_OK;
}

int amr_iso_indexed(amr_ctx* c, float iso, float* vtx, int64_t vcap, int32_t* tri, int64_t tcap, int32_t* vkeys,
                    int64_t* n_vtx, int64_t* n_tri, int flags) {
  if (!c || !n_vtx || !n_tri || vcap < 0 || tcap < 0 || (vcap > 0 && !vtx) || (tcap > 0 && !tri))
    return AMR_ERR_INVALID_ARG;
  if (c->stage < 3) return AMR_ERR_STATE;
  AMR_CUDA(cudaSetDevice(c->device));
  const Locator L = make_locator(c);
  const uint4* du = static_cast<const uint4*>(c->duals.p);
  unsigned long long* counter = &dev_sc(c)->n_tri[0];
  // 1. the kept triangles' edge keys (rerun once with the exact count if short)
  long long kcap = std::max(c->tkeys_cap, c->n_dual / 4 + 1024);
  long long nt = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    AMR_TRY(ensure(c->tkeys, (size_t)kcap * 24));
    c->tkeys_cap = (long long)(c->tkeys.bytes / 24);
    AMR_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), c->stream));
    {
      KernelTimer kt(c, KT_MC_KEYS);
      AMR_CUDA(launch_mc_keys(c->logb, L, du, c->n_dual, iso, static_cast<unsigned long long*>(c->tkeys.p),
                              c->tkeys_cap, counter, c->mc, grid_for(c, c->n_dual, 256, 8),
                              c->stream));
    }
    AMR_TRY(mc_result(c, counter, &nt));
    if (nt <= c->tkeys_cap) break;
    kcap = nt;
  }
  if (nt > c->tkeys_cap) return AMR_ERR_CUDA;
  // outputs: the caller's device buffers, or staging for host delivery
  const bool host = (flags & AMR_HOST_PTRS) != 0;
  const size_t vbytes = (size_t)vcap * 12, kbytes = vkeys ? (size_t)vcap * 8 : 0, tbytes = (size_t)tcap * 12;
  float* dv = vtx;
  int* dk = vkeys;
  int* dt = tri;
  if (host) {
    AMR_TRY(ensure(c->ostage, vbytes + kbytes + tbytes + 16));
    unsigned char* b = static_cast<unsigned char*>(c->ostage.p);
    dv = reinterpret_cast<float*>(b);
    dk = vkeys ? reinterpret_cast<int*>(b + vbytes) : nullptr;
    dt = reinterpret_cast<int*>(b + vbytes + kbytes);
  }
  // 2. weld: table sized for up to nt distinct vertices at half load (a closed
  //    surface has about nt / 2), rebuilt four times larger if it fills up
  unsigned long long want = pow2_at_least((unsigned long long)std::max(2 * nt, 1024ll));
  long long nv = 0;
  for (int attempt = 0;; ++attempt) {
    AMR_TRY(ensure(c->wtab, (size_t)want * 16));
    AMR_CUDA(cudaMemsetAsync(c->wtab.p, 0xFF, (size_t)want * 16, c->stream));
    AMR_TRY(reset_scratch(c));
    {
      KernelTimer kt(c, KT_WELD_INSERT);
      AMR_CUDA(launch_weld_insert(c->logb, L, static_cast<const unsigned long long*>(c->tkeys.p), 3 * nt,
                                  static_cast<ulonglong2*>(c->wtab.p), want - 1, iso, dv, dk, vcap, dev_sc(c),
                                  grid_for(c, 3 * nt, 256, 8), c->stream));
    }
    AMR_TRY(read_scratch(c));
    if (c->host_sc->err & ERR_HASH_FULL) {
      if (attempt >= 3) return AMR_ERR_RANGE;
      want *= 4;
      continue;
    }
    nv = (long long)c->host_sc->n_vtx;
    break;
  }
  // 3. the triangles' vertex indices
  {
    KernelTimer kt(c, KT_WELD_INDEX);
    AMR_CUDA(launch_weld_index(static_cast<const unsigned long long*>(c->tkeys.p), std::min<long long>(nt, tcap),
                               static_cast<const ulonglong2*>(c->wtab.p), want - 1, dt,
                               grid_for(c, 3 * std::min<long long>(nt, tcap), 256, 8), c->stream));
  }
  *n_vtx = nv;
  *n_tri = nt;
  if (host) {
    const long long wv = std::min(nv, (long long)vcap), wt = std::min(nt, (long long)tcap);
    if (wv > 0) AMR_TRY(deliver(c, vtx, dv, (size_t)wv * 12, flags));
    if (wv > 0 && vkeys) AMR_TRY(deliver(c, vkeys, dk, (size_t)wv * 8, flags));
    if (wt > 0) AMR_TRY(deliver(c, tri, dt, (size_t)wt * 12, flags));
  }
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  return (nv > vcap || nt > tcap) ? AMR_ERR_CAPACITY : AMR_OK;
}

int amr_interpolate(amr_ctx* c, float iso, const float* attr, const int32_t* vkeys, int64_t nv, float* out,
                    int flags) {
  if (!c || nv < 0 || (nv > 0 && (!attr || !vkeys || !out))) return AMR_ERR_INVALID_ARG;
  if (c->stage < 1) return AMR_ERR_STATE;
  AMR_CUDA(cudaSetDevice(c->device));
  if (nv == 0) return AMR_OK;
  const float* da = attr;
  const int* dk = vkeys;
  float* dout = out;
  const bool host = (flags & AMR_HOST_PTRS) != 0;
  if (host) {   // staging: attribute per cell, keys and results per vertex
    const size_t abytes = (size_t)c->n * 4, kbytes = (size_t)nv * 8;
    AMR_TRY(ensure(c->ostage, abytes + kbytes + (size_t)nv * 4 + 16));
    unsigned char* b = static_cast<unsigned char*>(c->ostage.p);
    AMR_CUDA(cudaMemcpyAsync(b, attr, abytes, cudaMemcpyHostToDevice, c->stream));
    AMR_CUDA(cudaMemcpyAsync(b + abytes, vkeys, kbytes, cudaMemcpyHostToDevice, c->stream));
    da = reinterpret_cast<const float*>(b);
    dk = reinterpret_cast<const int*>(b + abytes);
    dout = reinterpret_cast<float*>(b + abytes + kbytes);
  }
  AMR_TRY(reset_scratch(c));
  {
    KernelTimer kt(c, KT_INTERPOLATE);
    AMR_CUDA(launch_interpolate(c->xyz, c->s, da, c->n, dk, nv, iso, dout, dev_sc(c), grid_for(c, nv, 256, 8),
                                c->stream));
  }
  if (host) AMR_TRY(deliver(c, out, dout, (size_t)nv * 4, flags));
  AMR_TRY(read_scratch(c));
  return err_code(c->host_sc->err);
}

int amr_dual_shapes(amr_ctx* c, uint8_t* counts, int64_t* hist, int flags) {
  if (!c || (!counts && !hist)) return AMR_ERR_INVALID_ARG;
  if (c->stage < 3) return AMR_ERR_STATE;
  AMR_CUDA(cudaSetDevice(c->device));
  const long long nd = c->n_dual;
  unsigned char* dc = counts ? reinterpret_cast<unsigned char*>(counts) : nullptr;
  const bool host = (flags & AMR_HOST_PTRS) != 0;
  AMR_TRY(ensure(c->ostage, (size_t)(host && counts ? nd : 0) + 16 * 9));
  unsigned long long* dh = static_cast<unsigned long long*>(c->ostage.p);
  if (host && counts) dc = static_cast<unsigned char*>(c->ostage.p) + 16 * 9;
  AMR_CUDA(cudaMemsetAsync(dh, 0, 9 * sizeof(unsigned long long), c->stream));
  {
    KernelTimer kt(c, KT_SHAPES);
    AMR_CUDA(launch_dual_shapes(static_cast<const uint4*>(c->duals.p), nd, dc, dh, grid_for(c, nd, 256, 8),
                                c->stream));
  }
  if (host && counts && nd > 0) AMR_TRY(deliver(c, counts, dc, (size_t)nd, flags));
  unsigned long long hh[9];
  AMR_CUDA(cudaMemcpyAsync(hh, dh, sizeof(hh), cudaMemcpyDeviceToHost, c->stream));
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  if (hist)
    for (int k = 0; k < 9; ++k) hist[k] = (int64_t)hh[k];
  return AMR_OK;
}

int amr_iso_cases(amr_ctx* c, float iso, uint8_t* cases, uint8_t* ntri, int flags) {
  if (!c || (!cases && !ntri)) return AMR_ERR_INVALID_ARG;
  if (c->stage < 3) return AMR_ERR_STATE;
  AMR_CUDA(cudaSetDevice(c->device));
  const long long nd = c->n_dual;
  unsigned char* dc = cases;
  unsigned char* dn = ntri;
  if (flags & AMR_HOST_PTRS) {
    AMR_TRY(ensure(c->stage_buf, (size_t)nd * 2 + 256));
    dc = cases ? static_cast<unsigned char*>(c->stage_buf.p) : nullptr;
    dn = ntri ? static_cast<unsigned char*>(c->stage_buf.p) + nd : nullptr;
  }
  {
    KernelTimer kt(c, KT_MC_CASES);
    AMR_CUDA(launch_mc(c->logb, make_locator(c), static_cast<const uint4*>(c->duals.p), nd, iso, nullptr, 0,
                       &dev_sc(c)->n_tri[0], dc, dn, c->mc, grid_for(c, nd, 256, 8), c->stream));
  }
  long long unused = 0;
  AMR_TRY(mc_result(c, &dev_sc(c)->n_tri[0], &unused));
  if (cases) AMR_TRY(deliver(c, cases, dc, (size_t)nd, flags));
  if (ntri) AMR_TRY(deliver(c, ntri, dn, (size_t)nd, flags));
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  return AMR_OK;
}

namespace {
BatchTable single_job(amr_ctx* c, int n_iso) {
  BatchTable T;
  batch_add_job(T, static_cast<const uint4*>(c->duals.p), static_cast<const float*>(c->scal.p),
                static_cast<const int4*>(c->bricks.p), c->n_dual, c->logb, n_iso);
  return T;
}
}  // namespace

int amr_iso_batch(amr_ctx* c, const float* isos, int n_iso, float* tris, int64_t cap, int64_t* offsets,
                  int flags) {
  if (!c || !isos || !offsets || n_iso < 1 || n_iso > kMaxIso || cap < 0 || (cap > 0 && !tris))
    return AMR_ERR_INVALID_ARG;
  if (c->stage < 3) return AMR_ERR_STATE;
  AMR_CUDA(cudaSetDevice(c->device));
  AMR_TRY(ensure(c->iso_buf, sizeof(float) * kMaxIso));
  AMR_TRY(ensure(c->seg_buf, sizeof(long long) * (kMaxIso + 1)));
  float* d_iso = static_cast<float*>(c->iso_buf.p);
  long long* d_off = static_cast<long long*>(c->seg_buf.p);
  AMR_CUDA(cudaMemcpyAsync(d_iso, isos, sizeof(float) * n_iso, cudaMemcpyHostToDevice, c->stream));
  const BatchTable T = single_job(c, n_iso);
  const int grid = c->sm_count * 8;
  {
    KernelTimer kt(c, KT_BATCH_COUNT);
    AMR_CUDA(launch_batch_count(T, d_iso, c->bwork.p, c->mc, grid, c->stream));
  }
  {
    KernelTimer kt(c, KT_BATCH_SCAN);
    AMR_CUDA(launch_batch_scan(T, c->bwork.p, d_off, c->stream));
  }
  AMR_CUDA(cudaMemcpyAsync(c->host_sc->n_tri, d_off, sizeof(long long) * (n_iso + 1), cudaMemcpyDeviceToHost,
                           c->stream));
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  for (int k = 0; k <= n_iso; ++k) offsets[k] = (int64_t)c->host_sc->n_tri[k];
  const long long run = offsets[n_iso];
  if (run > cap) return AMR_ERR_CAPACITY;
  float* dst = tris;
  if (flags & AMR_HOST_PTRS) {
    AMR_TRY(ensure(c->stage_buf, (size_t)std::max<long long>(run, 1) * 36));
    dst = static_cast<float*>(c->stage_buf.p);
  }
  {
    KernelTimer kt(c, KT_BATCH_EMIT);
    AMR_CUDA(launch_batch_emit(T, d_iso, c->bwork.p, d_off, dst, run, c->mc, grid, c->stream));
  }
  if (flags & AMR_HOST_PTRS) AMR_TRY(deliver(c, tris, dst, (size_t)run * 36, flags));
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  return AMR_OK;
}

int amr_iso_batch_async(amr_ctx* c, const float* d_isos, int n_iso, float* tris, int64_t cap,
                        int64_t* d_offsets) {
  if (!c || !d_isos || !d_offsets || n_iso < 1 || n_iso > kMaxIso || cap < 0 || (cap > 0 && !tris))
    return AMR_ERR_INVALID_ARG;
  if (c->stage < 3) return AMR_ERR_STATE;
  const BatchTable T = single_job(c, n_iso);
  long long* off = reinterpret_cast<long long*>(d_offsets);
  const int grid = c->sm_count * 8;
  {
    KernelTimer kt(c, KT_BATCH_COUNT);
    AMR_CUDA(launch_batch_count(T, d_isos, c->bwork.p, c->mc, grid, c->stream));
  }
  {
    KernelTimer kt(c, KT_BATCH_SCAN);
    AMR_CUDA(launch_batch_scan(T, c->bwork.p, off, c->stream));
  }
  {
    KernelTimer kt(c, KT_BATCH_EMIT);
    AMR_CUDA(launch_batch_emit(T, d_isos, c->bwork.p, off, tris, cap, c->mc, grid, c->stream));
  }
  return AMR_OK;
}

namespace {
// The batch table of a multi-data-set batch; AMR_OK or the reason it is refused.
int multi_table(const amr_iso_job* jobs, int n_jobs, BatchTable* T) {
  if (!jobs || n_jobs < 1 || n_jobs > kMaxJobs) return AMR_ERR_INVALID_ARG;
  int dev = -1;
  for (int j = 0; j < n_jobs; ++j) {
    amr_ctx* c = jobs[j].ctx;
    if (!c || jobs[j].n_iso < 1) return AMR_ERR_INVALID_ARG;
    if (T->n_q + jobs[j].n_iso > kMaxIso) return AMR_ERR_INVALID_ARG;
    if (c->stage < 3) return AMR_ERR_STATE;
    if (dev >= 0 && c->device != dev) return AMR_ERR_INVALID_ARG;
    dev = c->device;
    batch_add_job(*T, static_cast<const uint4*>(c->duals.p), static_cast<const float*>(c->scal.p),
                  static_cast<const int4*>(c->bricks.p), c->n_dual, c->logb, jobs[j].n_iso);
  }
  return AMR_OK;
}
}  // namespace

int64_t amr_iso_multi_workspace(const amr_iso_job* jobs, int n_jobs) {
  BatchTable T;
  const int rc = multi_table(jobs, n_jobs, &T);
  if (rc != AMR_OK) return rc;
  return (int64_t)batch_workspace_bytes(T.n_counters);
}

int amr_iso_multi_async(const amr_iso_job* jobs, int n_jobs, const float* d_isos, float* tris, int64_t cap,
                        int64_t* d_offsets, void* workspace, int64_t workspace_bytes, void* cuda_stream) {
  BatchTable T;
  AMR_TRY(multi_table(jobs, n_jobs, &T));
  if (!d_isos || !d_offsets || !workspace || cap < 0 || (cap > 0 && !tris) ||
      workspace_bytes < (int64_t)batch_workspace_bytes(T.n_counters))
    return AMR_ERR_INVALID_ARG;
  amr_ctx* c0 = jobs[0].ctx;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  long long* off = reinterpret_cast<long long*>(d_offsets);
  const int grid = c0->sm_count * 8;
  AMR_CUDA(launch_batch_count(T, d_isos, workspace, c0->mc, grid, st));
  AMR_CUDA(launch_batch_scan(T, workspace, off, st));
  AMR_CUDA(launch_batch_emit(T, d_isos, workspace, off, tris, cap, c0->mc, grid, st));
  return AMR_OK;
}

int amr_get_info(amr_ctx* c, amr_info* info) {
  if (!c || !info) return AMR_ERR_INVALID_ARG;
  info->n_cells = c->n;
  info->n_bricks = c->stage >= 2 ? c->n_bricks : 0;
  info->n_slots = c->stage >= 2 ? c->n_slots : 0;
  info->n_dual = c->stage >= 3 ? c->n_dual : -1;
  info->n_levels = c->stage >= 2 ? c->levels : 0;
  info->log2_brick = c->logb;
  info->placement = c->placement;
  info->reserved = 0;
  const DevBuf* bufs[] = {&c->own_xyz, &c->own_lvl, &c->own_s, &c->htab, &c->bricks,
                          &c->rec, &c->scal, &c->view, &c->nbr, &c->staging, &c->codes,
                          &c->elist, &c->duals,
                          &c->scratch, &c->stage_buf, &c->iso_buf, &c->seg_buf, &c->bwork, &c->tkeys, &c->wtab,
                          &c->ostage, &c->border, &c->bcount};
  long long total = 0;
  for (const DevBuf* b : bufs) total += (long long)held(*b);
  info->device_bytes = total;
  return AMR_OK;
}

int amr_enable_timing(amr_ctx* c, int on) {
  if (!c) return AMR_ERR_INVALID_ARG;
  c->timing = on != 0;
  return AMR_OK;
}

int amr_kernel_times(amr_ctx* c, double* ms, int64_t* launches, int n) {
  if (!c) return AMR_ERR_INVALID_ARG;
  AMR_CUDA(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < KT_COUNT; ++k) {
    for (auto& p : c->pending[k]) {
      float t = 0.f;
      cudaEventElapsedTime(&t, p.first, p.second);
      c->ms_acc[k] += t;
      c->ev_pool.push_back(p.first);
      c->ev_pool.push_back(p.second);
    }
    c->pending[k].clear();
    if (k < n) {
      if (ms) ms[k] = c->ms_acc[k];
      if (launches) launches[k] = c->launches[k];
    }
    c->ms_acc[k] = 0;
    c->launches[k] = 0;
  }
  return KT_COUNT;
}

const char* amr_kernel_name(int k) { return (k >= 0 && k < KT_COUNT) ? kKernelNames[k] : nullptr; }

}  // extern "C"
