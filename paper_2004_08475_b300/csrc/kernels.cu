// CUDA kernels (sm_103a) for AMR dual cells and iso-surfaces (Wald, Sec. 3-5).
//
// Data layout in HBM (one data set):
//   input        xyz[n][3] int32, level[n] u8, scalar[n] f32 (caller order)
//   brick hash   htab[hcap] 16-byte entries {u64 key = (level, brick coords), brick index}
//   bricks       bricks[n_bricks] int4 = lower corner of the brick (finest
//                units) and its level; a level-l brick covers B^3 logical
//                level-l cells, B = 2^LOGB
//   slots        one per logical cell of every brick, Morton order inside a
//                brick: rec[] (8 bytes: input index and scalar bits of the
//                occupant, all ones when empty), scal[] (its scalar), view[]
//                (the slot of the actual cell containing the logical cell:
//                itself, a coarser cell, or kReject)
//   dual cells   duals[D] = 2 x uint4: the 8 vertex slots, order ex+2ey+4ez;
//                bit 31 of the first is set when all 8 vertices are cells of
//                one level at 8 different positions (hence 8 different cells)
//   triangles    tris[T][3][3] f32
//
// snap() of Sec. 3.2 becomes: find the brick of the query at the query's
// level (one hash probe), read the slot's view. A missing brick at level l
// means no level-l cell near the query; the first existing brick at a
// coarser level then holds the answer, because an aligned level-l brick lies
// inside one aligned brick of every coarser level.

#include <algorithm>
#include <climits>
#include <cstdint>

#include "kernels.h"

namespace amriso {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Home entry of a key: Fibonacci (multiplicative) hashing (Knuth, The Art
// of Computer Programming vol. 3, Sec. 6.4), the top log2(hcap) bits of
// key * 2^64/phi, rounded down to an even entry so that the first probe
// reads one 32-byte sector of two entries. Probing is linear from there.
// hcap >= 2.
__device__ __forceinline__ unsigned long long home_of(unsigned long long key, unsigned long long hmask) {
  return ((key * 0x9E3779B97F4A7C15ull) >> (64 - __popcll(hmask))) & ~1ull;
}

// Key of the level-l brick containing finest-level point (x,y,z). Brick
// coordinates are kept modulo 2^20, which is exact because extents are
// below 2^21 finest units.
template <int LOGB>
__device__ __forceinline__ unsigned long long brick_key(int x, int y, int z, int l) {
  const int sh = l + LOGB;
  const unsigned long long bx = (unsigned)(x >> sh) & 0xFFFFFu;
  const unsigned long long by = (unsigned)(y >> sh) & 0xFFFFFu;
  const unsigned long long bz = (unsigned)(z >> sh) & 0xFFFFFu;
  return ((unsigned long long)l << 60) | (bz << 40) | (by << 20) | bx;
}

// Bits b of v (v < 2^LOGB) moved to bit 3b.
template <int LOGB>
__device__ __forceinline__ unsigned spread(unsigned v) {
  static_assert(LOGB == 2 || LOGB == 3, "bricks of 4^3 or 8^3 cells");
  if constexpr (LOGB == 3) return (v | (v << 2) | (v << 4)) & 0x49u;
  else return (v | (v << 2)) & 0x9u;
}

template <int LOGB>
__device__ __forceinline__ int compact(unsigned m) {
  unsigned r = 0;
#pragma unroll
  for (int b = 0; b < LOGB; ++b) r |= ((m >> (3 * b)) & 1u) << b;
  return (int)r;
}

// Morton index, inside its level-l brick, of the logical level-l cell
// containing (x,y,z).
template <int LOGB>
__device__ __forceinline__ unsigned local_index(int x, int y, int z, int l) {
  constexpr unsigned M = (1u << LOGB) - 1u;
  return spread<LOGB>((unsigned)(x >> l) & M) | (spread<LOGB>((unsigned)(y >> l) & M) << 1) |
         (spread<LOGB>((unsigned)(z >> l) & M) << 2);
}

__device__ __forceinline__ int find_brick(const Locator& L, unsigned long long key) {
  unsigned long long h = home_of(key, L.hmask);
  for (unsigned long long p = 0; p <= L.hmask; p += 2) {   // one sector (two entries) per step
    const ulonglong2 e0 = __ldg(L.htab + h), e1 = __ldg(L.htab + h + 1);
    if (e0.x == key) return (int)e0.y;
    if (e0.x == kEmptyKey) return -1;
    if (e1.x == key) return (int)e1.y;
    if (e1.x == kEmptyKey) return -1;
    h = (h + 2) & L.hmask;
  }
  return -1;
}

// First probe, for callers that issue several at once: the key's home
// sector; returns the brick index, or -2 when the key lies further on.
__device__ __forceinline__ int probe_home(const Locator& L, unsigned long long key) {
  const unsigned long long h = home_of(key, L.hmask);
  const ulonglong2 e0 = __ldg(L.htab + h), e1 = __ldg(L.htab + h + 1);
  if (e0.x == key) return (int)e0.y;
  if (e0.x == kEmptyKey) return -1;
  if (e1.x == key) return (int)e1.y;
  if (e1.x == kEmptyKey) return -1;
  return -2;
}

// Lower corner and level of the cell stored in `slot`.
template <int LOGB>
__device__ __forceinline__ int4 slot_cell(const int4* __restrict__ bricks, unsigned slot) {
  const int4 b = __ldg(bricks + (slot >> (3 * LOGB)));
  const unsigned loc = slot & ((1u << (3 * LOGB)) - 1u);
  return make_int4(b.x + (compact<LOGB>(loc) << b.w), b.y + (compact<LOGB>(loc >> 1) << b.w),
                   b.z + (compact<LOGB>(loc >> 2) << b.w), b.w);
}

__device__ __forceinline__ unsigned warp_or(unsigned v) { return __reduce_or_sync(kFull, v); }

// Morton index inside a brick -> cell offsets x | y << 4 | z << 8, as a
// shared-memory table (filled by fill_cell_table before a barrier): one
// load instead of the bit compaction per axis in the vertex loops.
template <int LOGB>
__device__ __forceinline__ void fill_cell_table(unsigned short* tab) {
  for (int m = threadIdx.x; m < (1 << (3 * LOGB)); m += blockDim.x)
    tab[m] = (unsigned short)(compact<LOGB>(m) | (compact<LOGB>(m >> 1) << 4) | (compact<LOGB>(m >> 2) << 8));
}

// slot_cell through the table.
template <int LOGB>
__device__ __forceinline__ int4 slot_cell_tab(const int4* __restrict__ bricks, const unsigned short* tab,
                                              unsigned slot) {
  const int4 b = __ldg(bricks + (slot >> (3 * LOGB)));
  const unsigned t = tab[slot & ((1u << (3 * LOGB)) - 1u)];
  return make_int4(b.x + ((int)(t & 15u) << b.w), b.y + ((int)((t >> 4) & 15u) << b.w),
                   b.z + ((int)(t >> 8) << b.w), b.w);
}

// ---------------------------------------------------------------------------
// Locator build (Sec. 3.2)
// ---------------------------------------------------------------------------

constexpr int kUnroll = 4;   // cells per lane per trip of the cell-parallel loops

// The home sector of a probe, entries h and h + 1 (h even, the table 32-byte
// aligned), in one 32-byte load.
__device__ __forceinline__ void load_home_sector(const ulonglong2* p, ulonglong2& a, ulonglong2& b) {
  asm("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
      : "=l"(a.x), "=l"(a.y), "=l"(b.x), "=l"(b.y)
      : "l"(p));
}

// Pass 1 over the cells: validate corners and levels, take the bounding box
// and the deepest level, and insert every cell's brick key into the hash
// table (scalars are checked in pass 2). The CAS winner of a key numbers the
// brick and records its corner and level. Each lane takes kUnroll = 4
// consecutive cells per trip (their corners as three 16-byte loads and
// their levels as one 4-byte load when the arrays are aligned for it), loads
// and first probes hoisted, so that their memory latencies overlap; the
// first probe reads the home sector's two entries whole (keys and brick
// indices) in one load. Lanes holding the same key simply both find it (or
// race on one CAS, which one of them wins).
// codes (binned placement): per cell its slot (brick index << 3 LOGB | its
// Morton index in the brick) when the brick's index was already readable,
// else kCodeEntry | its brick's table entry << 3 LOGB | Morton index (the
// winner of that brick had not stored the index yet; k_bin_coarse reads it).
constexpr unsigned kCodeEntry = 0x80000000u;

template <int LOGB>
__global__ void __launch_bounds__(1024) k_insert_bricks(
    const int* __restrict__ xyz, const unsigned char* __restrict__ lvl,
    const float* __restrict__ s, long long n, ulonglong2* htab,
    unsigned long long hmask, int4* bricks, unsigned long long brick_limit, Scratch* sc,
    unsigned* __restrict__ codes) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int hshift = 64 - __popcll(hmask);
  int lo0 = INT_MAX, lo1 = INT_MAX, lo2 = INT_MAX;
  int hi0 = INT_MIN, hi1 = INT_MIN, hi2 = INT_MIN;
  int ml = 0;
  unsigned err = 0;
  // a table this crowded is rebuilt larger by the host: fail fast
  const unsigned long long limit = hmask < 4095ull ? hmask + 1 : 4096ull;
  static_assert(kUnroll == 4, "a lane's cells are read as one 4-byte load of levels");
  const bool vec = ((reinterpret_cast<uintptr_t>(xyz) & 15u) | (reinterpret_cast<uintptr_t>(lvl) & 3u) |
                    (reinterpret_cast<uintptr_t>(codes) & 15u)) == 0;
  int trip = 0;
  for (long long base = wid * 32 * kUnroll; base < n; base += nwarps * 32 * kUnroll) {
    if ((trip++ & 31) == 0 && __any_sync(kFull, (__ldcg(&sc->err) & ERR_HASH_FULL) != 0u)) break;
    int x[kUnroll], y[kUnroll], z[kUnroll], l[kUnroll];
    const long long c0 = base + kUnroll * lane;   // the lane's first cell
    const bool whole = vec && c0 + kUnroll <= n;
    if (whole) {   // streamed once: evict first, keep the hash table in L2
      const int4* p = reinterpret_cast<const int4*>(xyz + 3 * c0);
      const int4 a = __ldcs(p), b = __ldcs(p + 1), c = __ldcs(p + 2);
      const unsigned lv = __ldcs(reinterpret_cast<const unsigned*>(lvl + c0));
      x[0] = a.x; y[0] = a.y; z[0] = a.z;
      x[1] = a.w; y[1] = b.x; z[1] = b.y;
      x[2] = b.z; y[2] = b.w; z[2] = c.x;
      x[3] = c.y; y[3] = c.z; z[3] = c.w;
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) l[u] = (int)((lv >> (8 * u)) & 255u);
    } else {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const long long i = c0 + u;
        x[u] = y[u] = z[u] = 0;
        l[u] = -1;
        if (i < n) {
          x[u] = __ldcs(xyz + 3 * i);
          y[u] = __ldcs(xyz + 3 * i + 1);
          z[u] = __ldcs(xyz + 3 * i + 2);
          l[u] = __ldcs(lvl + i);
        }
      }
    }
    unsigned long long key[kUnroll];
    ulonglong2 e0[kUnroll];
    unsigned long long cur1[kUnroll];
    unsigned h[kUnroll], loc[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      key[u] = kEmptyKey;
      loc[u] = 0;
      h[u] = 0;
      if (l[u] >= 0) {
        if (l[u] > kMaxLevel) {
          err |= ERR_RANGE;
        } else if ((x[u] | y[u] | z[u]) & ((1 << l[u]) - 1)) {
          err |= ERR_UNALIGNED;
        } else if (max(max(x[u], y[u]), z[u]) > (1 << 30) || min(min(x[u], y[u]), z[u]) < -(1 << 30)) {
          err |= ERR_RANGE;   // corners beyond +-2^30 (so that x + w stays below 2^31)
        } else {
          const int w = 1 << l[u];
          lo0 = min(lo0, x[u]);
          lo1 = min(lo1, y[u]);
          lo2 = min(lo2, z[u]);
          hi0 = max(hi0, x[u] + w);
          hi1 = max(hi1, y[u] + w);
          hi2 = max(hi2, z[u] + w);
          ml = max(ml, l[u]);
          key[u] = brick_key<LOGB>(x[u], y[u], z[u], l[u]);
          loc[u] = local_index<LOGB>(x[u], y[u], z[u], l[u]);
          h[u] = (unsigned)((key[u] * 0x9E3779B97F4A7C15ull) >> hshift) & ~1u;   // home_of
        }
      }
      // independent first probes: the home sector (entry h whole, entry h + 1's key)
      e0[u] = make_ulonglong2(0ull, 0ull);
      cur1[u] = 0ull;
      if (key[u] != kEmptyKey) {
        ulonglong2 e1;
        load_home_sector(htab + h[u], e0[u], e1);
        cur1[u] = e1.x;
      }
    }
    unsigned code4[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      code4[u] = kReject;
      if (key[u] == kEmptyKey) continue;
      const long long i = c0 + u;
      unsigned code;
      if (e0[u].x == key[u]) {   // at home, the common case: the brick index came with the key
        code = e0[u].y != kEmptyKey ? ((unsigned)e0[u].y << (3 * LOGB)) | loc[u]
                                    : kCodeEntry | (h[u] << (3 * LOGB)) | loc[u];
      } else if (cur1[u] == key[u]) {
        code = kCodeEntry | ((h[u] + 1) << (3 * LOGB)) | loc[u];
      } else {
        unsigned long long hh = h[u];
        bool done = false;
        code = kReject;
        for (unsigned long long p = 0; p < limit; ++p) {
          const unsigned long long c = p == 0 ? e0[u].x : (p == 1 ? cur1[u] : __ldcg(&htab[hh].x));
          if (c == key[u]) { done = true; break; }
          if (c == kEmptyKey) {
            const unsigned long long prev = atomicCAS(&htab[hh].x, kEmptyKey, key[u]);
            if (prev == kEmptyKey) {
              const unsigned long long bi = atomicAdd(&sc->n_bricks, 1ull);
              htab[hh].y = bi;
              if (bi < brick_limit) {   // bricks[] holds brick_limit entries; the cell is read again
                const int lv = lvl[i];
                const int m = ~((1 << (lv + LOGB)) - 1);
                bricks[bi] = make_int4(xyz[3 * i] & m, xyz[3 * i + 1] & m, xyz[3 * i + 2] & m, lv);
                code = ((unsigned)bi << (3 * LOGB)) | loc[u];
              } else {
                atomicOr(&sc->err, (unsigned)ERR_HASH_FULL);
              }
              done = true;
              break;
            }
            if (prev == key[u]) { done = true; break; }
          }
          hh = (hh + 1) & hmask;
        }
        if (!done) err |= ERR_HASH_FULL;
        else if (code == kReject) code = kCodeEntry | ((unsigned)hh << (3 * LOGB)) | loc[u];
      }
      code4[u] = code;
      if (codes && !whole) __stcs(codes + i, code);
    }
    // (an invalid cell's code is never read: the host stops on its error)
    if (codes && whole)
      __stcs(reinterpret_cast<uint4*>(codes + c0), make_uint4(code4[0], code4[1], code4[2], code4[3]));
  }
  // block reduction, then one set of atomics per block
  __shared__ int red[8][32];
  const int w = threadIdx.x >> 5;
  lo0 = __reduce_min_sync(kFull, lo0);
  lo1 = __reduce_min_sync(kFull, lo1);
  lo2 = __reduce_min_sync(kFull, lo2);
  hi0 = __reduce_max_sync(kFull, hi0);
  hi1 = __reduce_max_sync(kFull, hi1);
  hi2 = __reduce_max_sync(kFull, hi2);
  ml = __reduce_max_sync(kFull, ml);
  err = warp_or(err);
  if (lane == 0) {
    red[0][w] = lo0; red[1][w] = lo1; red[2][w] = lo2;
    red[3][w] = hi0; red[4][w] = hi1; red[5][w] = hi2;
    red[6][w] = ml;  red[7][w] = (int)err;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    const bool ok = lane < nw;
    int a0 = ok ? red[0][lane] : INT_MAX, a1 = ok ? red[1][lane] : INT_MAX,
        a2 = ok ? red[2][lane] : INT_MAX;
    int b0 = ok ? red[3][lane] : INT_MIN, b1 = ok ? red[4][lane] : INT_MIN,
        b2 = ok ? red[5][lane] : INT_MIN;
    int m = ok ? red[6][lane] : 0;
    unsigned e = ok ? (unsigned)red[7][lane] : 0u;
    a0 = __reduce_min_sync(kFull, a0);
    a1 = __reduce_min_sync(kFull, a1);
    a2 = __reduce_min_sync(kFull, a2);
    b0 = __reduce_max_sync(kFull, b0);
    b1 = __reduce_max_sync(kFull, b1);
    b2 = __reduce_max_sync(kFull, b2);
    m = __reduce_max_sync(kFull, m);
    e = warp_or(e);
    if (lane == 0) {
      if (a0 != INT_MAX) {
        atomicMin(&sc->lo[0], a0); atomicMin(&sc->lo[1], a1); atomicMin(&sc->lo[2], a2);
        atomicMax(&sc->hi[0], b0); atomicMax(&sc->hi[1], b1); atomicMax(&sc->hi[2], b2);
        atomicMax(&sc->max_level, m);
      }
      if (e) atomicOr(&sc->err, e);
    }
  }
}

// Pass 2 over the cells: store every cell (index and scalar bits, one
// 8-byte record) into its brick slot with a plain store - no atomic, so the
// random writes do not wait on each other. A duplicate label (i,j,k;l) makes
// two cells share a slot; the slot pass below then counts fewer occupied
// slots than cells. Finite scalars never form the all-ones empty pattern.
template <int LOGB>
__global__ void __launch_bounds__(1024) k_scatter_cells(
    const int* __restrict__ xyz, const unsigned char* __restrict__ lvl,
    const float* __restrict__ s, long long n, Locator L, unsigned long long* rec, Scratch* sc) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  unsigned err = 0;
  for (long long base = wid * 32 * kUnroll; base < n; base += nwarps * 32 * kUnroll) {
    int x[kUnroll], y[kUnroll], z[kUnroll], l[kUnroll];
    float v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long i = base + u * 32 + lane;
      x[u] = y[u] = z[u] = 0;
      l[u] = -1;
      v[u] = 0.f;
      if (i < n) {
        x[u] = __ldcs(xyz + 3 * i);
        y[u] = __ldcs(xyz + 3 * i + 1);
        z[u] = __ldcs(xyz + 3 * i + 2);
        l[u] = __ldcs(lvl + i);
        v[u] = __ldcs(s + i);
        if (!isfinite(v[u])) err |= ERR_NONFINITE;
      }
    }
    unsigned long long key[kUnroll];
    int b0[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {   // first probe of every key, issued together
      key[u] = (l[u] >= 0 && l[u] <= kMaxLevel) ? brick_key<LOGB>(x[u], y[u], z[u], l[u]) : kEmptyKey;
      b0[u] = key[u] != kEmptyKey ? probe_home(L, key[u]) : -1;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (key[u] == kEmptyKey) continue;
      const int bi = b0[u] != -2 ? b0[u] : find_brick(L, key[u]);
      if (bi < 0) {
        err |= ERR_HASH_FULL;
        continue;
      }
      const long long i = base + u * 32 + lane;
      const long long slot = ((long long)bi << (3 * LOGB)) | local_index<LOGB>(x[u], y[u], z[u], l[u]);
      rec[slot] = ((unsigned long long)__float_as_uint(v[u]) << 32) | (unsigned)i;
    }
  }
  err = warp_or(err);
  if (lane == 0 && err) atomicOr(&sc->err, err);
}

// Binned form of pass 2. Random 8-byte stores run at one memory transaction
// each however small the address range they fall in, so k_scatter_cells is
// bound by its store transactions, not by DRAM. The binned form writes only
// whole runs: a two-level radix split of the cells by slot, then one CTA per
// window of 2^kWinShift slots builds the window's records in shared memory
// and writes them out in full lines (empty slots included, so `rec` needs
// no clearing).
//   k_bin_coarse: per tile of cells, find the slot, sort the tile by coarse
//     bin (2^kCoarseShift slots) in shared memory, append each bin's run to
//     the bin's region of stage A (one global atomic per bin and tile);
//   k_bin_fine: per tile of one coarse bin, the same split by window into
//     stage B;
//   k_place_windows: per window, scatter its entries into shared memory.
// Stages are three 32-bit arrays each (slot, cell index, scalar bits); a
// coarse bin holds at most 2^kCoarseShift entries and a window 2^kWinShift,
// more means two cells in one slot (ERR_DUPLICATE).
constexpr int kCoarseShift = 21;
constexpr int kMaxCoarse = 1 << (31 - kCoarseShift);   // slot indices stay below 2^31
constexpr int kWinShift = 13;
constexpr int kWinSlots = 1 << kWinShift;
constexpr int kFinePerCoarse = 1 << (kCoarseShift - kWinShift);
constexpr int kCoarseThreads = 512;
constexpr int kCoarsePer = 8;
constexpr int kCoarseTile = kCoarseThreads * kCoarsePer;
constexpr int kFineThreads = 256;   // five CTAs per SM: their barriers overlap
constexpr int kFinePer = 8;
constexpr int kFineTile = kFineThreads * kFinePer;
constexpr int kPlaceThreads = 512;

struct Stage {
  unsigned* slot;
  unsigned* idx;
  unsigned* val;
};

// Exclusive scan of cnt[0..m) in place (m <= PER * blockDim.x) and, for
// every non-empty entry, a run reserved in the global counter gcount[goff +
// b]; returns the total. All threads of the CTA must call it.
template <int PER>
__device__ __forceinline__ unsigned scan_and_reserve(unsigned* cnt, unsigned* gbase, int m,
                                                     unsigned* gcount, long long goff, unsigned* wsum) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  unsigned c[PER];
  unsigned v = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int b = PER * t + k;
    c[k] = b < m ? cnt[b] : 0u;
    if (c[k]) gbase[b] = atomicAdd(gcount + goff + b, c[k]);
    v += c[k];
  }
  unsigned incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    const unsigned x = lane < nw ? wsum[lane] : 0u;
    unsigned cc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, cc, o);
      if (lane >= o) cc += y;
    }
    if (lane < nw) wsum[lane] = cc - x;
    if (lane == 31) wsum[32] = cc;
  }
  __syncthreads();
  unsigned ex = wsum[w] + incl - v;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int b = PER * t + k;
    if (b < m) cnt[b] = ex;
    ex += c[k];
  }
  const unsigned total = wsum[32];
  __syncthreads();
  return total;
}

// A cell's slot is its code (from k_insert_bricks), or one table read away
// when the code holds the table entry of its brick instead.
template <int LOGB>
__global__ void __launch_bounds__(kCoarseThreads, 3) k_bin_coarse(const float* __restrict__ s, long long n, Locator L,
                                                               int n_coarse, Stage A,
                                                               unsigned* __restrict__ coarse_count, Scratch* sc,
                                                               const unsigned* __restrict__ codes) {
  extern __shared__ unsigned smem[];
  unsigned* start = smem;                     // [n_coarse] counts, then run starts in the tile
  unsigned* gbase = start + n_coarse;         // [n_coarse] run starts in the bins
  unsigned* t_slot = gbase + n_coarse;        // [kCoarseTile] the tile sorted by bin
  unsigned* t_idx = t_slot + kCoarseTile;
  unsigned* t_val = t_idx + kCoarseTile;
  __shared__ unsigned wsum[33];
  const int t = threadIdx.x, lane = t & 31;
  unsigned err = 0;
  for (long long tile0 = (long long)blockIdx.x * kCoarseTile; tile0 < n;
       tile0 += (long long)gridDim.x * kCoarseTile) {
    for (int b = t; b < n_coarse; b += kCoarseThreads) start[b] = 0;
    __syncthreads();
    unsigned slot[kCoarsePer], rank[kCoarsePer], val[kCoarsePer];
#pragma unroll
    for (int j = 0; j < kCoarsePer; ++j) {
      const long long i = tile0 + (long long)j * kCoarseThreads + t;
      slot[j] = kReject;
      rank[j] = 0;
      val[j] = 0u;
      if (i < n) {
        const unsigned c = __ldcs(codes + i);
        const float v = __ldcs(s + i);
        if (!isfinite(v)) err |= ERR_NONFINITE;
        val[j] = __float_as_uint(v);
        slot[j] = c;
        if (c & kCodeEntry) {   // the brick's index was not stored yet when the cell was inserted
          const unsigned bi = (unsigned)__ldg(&L.htab[(c & ~kCodeEntry) >> (3 * LOGB)].y);
          slot[j] = (bi << (3 * LOGB)) | (c & ((1u << (3 * LOGB)) - 1u));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kCoarsePer; ++j)
      if (slot[j] != kReject) rank[j] = atomicAdd(&start[slot[j] >> kCoarseShift], 1u);
    __syncthreads();
    const unsigned total = scan_and_reserve<kMaxCoarse / kCoarseThreads>(start, gbase, n_coarse, coarse_count, 0,
                                                                         wsum);
#pragma unroll
    for (int j = 0; j < kCoarsePer; ++j) {
      if (slot[j] == kReject) continue;
      const unsigned pos = start[slot[j] >> kCoarseShift] + rank[j];
      t_slot[pos] = slot[j];
      t_idx[pos] = (unsigned)(tile0 + (long long)j * kCoarseThreads + t);
      t_val[pos] = val[j];
    }
    __syncthreads();
    for (unsigned p = t; p < total; p += kCoarseThreads) {   // runs of one bin are contiguous: coalesced
      const unsigned sl = t_slot[p];
      const unsigned b = sl >> kCoarseShift;
      const unsigned r = gbase[b] + (p - start[b]);
      if (r >= (1u << kCoarseShift)) {
        err |= ERR_DUPLICATE;
        continue;
      }
      const long long dst = ((long long)b << kCoarseShift) + r;
      A.slot[dst] = sl;
      A.idx[dst] = t_idx[p];
      A.val[dst] = t_val[p];
    }
    __syncthreads();
  }
  err = warp_or(err);
  if (lane == 0 && err) atomicOr(&sc->err, err);
}

// Grid (tiles of one coarse bin, coarse bins).
__global__ void __launch_bounds__(kFineThreads) k_bin_fine(Stage A, const unsigned* __restrict__ coarse_count,
                                                          Stage B, unsigned* __restrict__ win_count, Scratch* sc) {
  extern __shared__ unsigned smem[];
  unsigned* start = smem;                      // [kFinePerCoarse]
  unsigned* gbase = start + kFinePerCoarse;    // [kFinePerCoarse]
  unsigned* t_slot = gbase + kFinePerCoarse;   // [kFineTile]
  unsigned* t_idx = t_slot + kFineTile;
  unsigned* t_val = t_idx + kFineTile;
  __shared__ unsigned wsum[33];
  const int t = threadIdx.x;
  const long long cb = blockIdx.y;
  const unsigned cnt = min(__ldg(coarse_count + cb), 1u << kCoarseShift);
  const unsigned tile0 = blockIdx.x * (unsigned)kFineTile;
  if (tile0 >= cnt) return;   // uniform over the CTA
  for (int b = t; b < kFinePerCoarse; b += kFineThreads) start[b] = 0;
  __syncthreads();
  unsigned slot[kFinePer], rank[kFinePer], idx[kFinePer], val[kFinePer];
  const long long src0 = (cb << kCoarseShift) + tile0;
#pragma unroll
  for (int j = 0; j < kFinePer; ++j) {
    const unsigned e = tile0 + j * kFineThreads + t;
    slot[j] = kReject;
    rank[j] = 0;
    if (e < cnt) {
      const long long src = src0 + j * kFineThreads + t;
      slot[j] = __ldcs(A.slot + src);
      idx[j] = __ldcs(A.idx + src);
      val[j] = __ldcs(A.val + src);
      rank[j] = atomicAdd(&start[(slot[j] >> kWinShift) & (kFinePerCoarse - 1)], 1u);
    }
  }
  __syncthreads();
  const unsigned total = scan_and_reserve<kFinePerCoarse / kFineThreads>(start, gbase, kFinePerCoarse, win_count,
                                                                         cb << (kCoarseShift - kWinShift), wsum);
#pragma unroll
  for (int j = 0; j < kFinePer; ++j) {
    if (slot[j] == kReject) continue;
    const unsigned pos = start[(slot[j] >> kWinShift) & (kFinePerCoarse - 1)] + rank[j];
    t_slot[pos] = slot[j];
    t_idx[pos] = idx[j];
    t_val[pos] = val[j];
  }
  __syncthreads();
  unsigned err = 0;
  for (unsigned p = t; p < total; p += kFineThreads) {
    const unsigned sl = t_slot[p];
    const unsigned f = (sl >> kWinShift) & (kFinePerCoarse - 1);
    const unsigned r = gbase[f] + (p - start[f]);
    if (r >= (unsigned)kWinSlots) {
      err |= ERR_DUPLICATE;
      continue;
    }
    const long long dst = ((long long)(sl >> kWinShift) << kWinShift) + r;
    B.slot[dst] = sl;
    B.idx[dst] = t_idx[p];
    B.val[dst] = t_val[p];
  }
  err = warp_or(err);
  if ((t & 31) == 0 && err) atomicOr(&sc->err, err);
}

// One CTA per window of kWinSlots slots: the records built in shared memory
// and written whole (empty slots as kEmptyRec), and with them each slot's
// view (the slot itself where a cell occupies it, else kReject for now) and
// scalar (0 when empty); counts the occupied slots and lists the bricks that
// have empty slots (elist, counted by sc->n_elist) for k_resolve_empty.
template <int LOGB>
__global__ void __launch_bounds__(kPlaceThreads) k_place_windows(Stage B, const unsigned* __restrict__ win_count,
                                                                 long long n_slots, unsigned long long* rec,
                                                                 unsigned* view, float* scal,
                                                                 unsigned* __restrict__ elist, Scratch* sc) {
  constexpr int kBricksPerWin = kWinSlots >> (3 * LOGB);
  extern __shared__ __align__(16) unsigned long long win[];   // [kWinSlots]
  __shared__ unsigned char holes[kBricksPerWin];
  __shared__ unsigned occ_w[kPlaceThreads / 32];
  const int t = threadIdx.x;
  const long long w0 = (long long)blockIdx.x << kWinShift;
  for (int k = t; k < kWinSlots; k += kPlaceThreads) win[k] = kEmptyRec;
  for (int k = t; k < kBricksPerWin; k += kPlaceThreads) holes[k] = 0;
  __syncthreads();
  const unsigned cnt = min(__ldg(win_count + blockIdx.x), (unsigned)kWinSlots);
  for (unsigned e = t; e < cnt; e += kPlaceThreads) {
    const unsigned sl = __ldcs(B.slot + w0 + e);
    win[sl & (kWinSlots - 1)] = ((unsigned long long)__ldcs(B.val + w0 + e) << 32) | __ldcs(B.idx + w0 + e);
  }
  __syncthreads();
  // n_slots is a multiple of the brick size (>= 64), so windows end on pairs
  const long long m = min((long long)kWinSlots, n_slots - w0);
  ulonglong2* dst = reinterpret_cast<ulonglong2*>(rec + w0);
  uint2* vdst = reinterpret_cast<uint2*>(view + w0);
  float2* sdst = reinterpret_cast<float2*>(scal + w0);
  const ulonglong2* srcw = reinterpret_cast<const ulonglong2*>(win);
  unsigned occ = 0;
  for (long long k = t; k < m / 2; k += kPlaceThreads) {
    const ulonglong2 r = srcw[k];
    dst[k] = r;
    const bool o0 = r.x != kEmptyRec, o1 = r.y != kEmptyRec;
    const unsigned s0 = (unsigned)(w0 + 2 * k);
    vdst[k] = make_uint2(o0 ? s0 : kReject, o1 ? s0 + 1 : kReject);
    sdst[k] = make_float2(o0 ? __uint_as_float((unsigned)(r.x >> 32)) : 0.f,
                          o1 ? __uint_as_float((unsigned)(r.y >> 32)) : 0.f);
    occ += (o0 ? 1u : 0u) + (o1 ? 1u : 0u);
    if (!(o0 && o1)) holes[(2 * k) >> (3 * LOGB)] = 1;
  }
  occ = __reduce_add_sync(kFull, occ);
  if ((t & 31) == 0) occ_w[t >> 5] = occ;
  __syncthreads();
  if (t < 32) {
    unsigned a = t < kPlaceThreads / 32 ? occ_w[t] : 0u;
    a = __reduce_add_sync(kFull, a);
    if (t == 0 && a) atomicAdd(&sc->n_occupied, (unsigned long long)a);
    // bricks of this window with empty slots, one reservation per window
    const int nb = (int)(m >> (3 * LOGB));
    for (int b0 = 0; b0 < nb; b0 += 32) {
      const bool h = b0 + t < nb && holes[b0 + t];
      const unsigned bal = __ballot_sync(kFull, h);
      if (!bal) continue;
      unsigned long long base = 0;
      if (t == 0) base = atomicAdd(&sc->n_elist, (unsigned long long)__popc(bal));
      base = __shfl_sync(kFull, base, 0);
      if (h) elist[base + __popc(bal & ((1u << t) - 1u))] = (unsigned)((w0 >> (3 * LOGB)) + b0 + t);
    }
  }
}

// Pass over the bricks listed by k_place_windows: each of their empty slots
// resolved to the actual cell containing its logical cell - the first
// occupied slot at a coarser level (a slot is occupied iff its view is
// itself), else kReject (finer cells or a hole). The list's length is read
// on the device (sc->n_elist).
template <int LOGB>
__global__ void __launch_bounds__(256) k_resolve_empty(Locator L, const unsigned* __restrict__ elist,
                                                       const Scratch* sc, unsigned* view) {
  constexpr int kB3 = 1 << (3 * LOGB);
  const long long total = (long long)__ldcg(&sc->n_elist) * kB3;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const unsigned slot = (__ldg(elist + (i >> (3 * LOGB))) << (3 * LOGB)) | (unsigned)(i & (kB3 - 1));
    if (view[slot] != kReject) continue;   // occupied: view is the slot itself
    const int4 c = slot_cell<LOGB>(L.bricks, slot);
    for (int lv = c.w + 1; lv < L.levels; ++lv) {
      const int bj = find_brick(L, brick_key<LOGB>(c.x, c.y, c.z, lv));
      if (bj < 0) continue;
      const unsigned s2 = ((unsigned)bj << (3 * LOGB)) | local_index<LOGB>(c.x, c.y, c.z, lv);
      if (view[s2] == s2) {   // an empty slot's view is never itself, whether resolved yet or not
        view[slot] = s2;
        break;
      }
    }
  }
}

// Pass over the slots: resolve every logical cell of every brick to the
// actual cell containing it - its own occupant, else the first occupied slot
// at a coarser level, else kReject (finer cells or a hole). With
// check_overlap, an occupied slot that is also covered by a coarser cell
// flags ERR_OVERLAP.
template <int LOGB>
__global__ void __launch_bounds__(1024) k_resolve_views(Locator L, unsigned* view, float* scal,
                                                       long long n_slots, int check_overlap, Scratch* sc) {
  unsigned err = 0;
  unsigned occ = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x; slot < n_slots;
       slot += stride) {
    const int4 c = slot_cell<LOGB>(L.bricks, (unsigned)slot);
    const unsigned long long r = L.rec[slot];
    const bool occupied = r != kEmptyRec;
    unsigned v = occupied ? (unsigned)slot : kReject;
    if (!occupied || check_overlap) {
      for (int lv = c.w + 1; lv < L.levels; ++lv) {
        const int bj = find_brick(L, brick_key<LOGB>(c.x, c.y, c.z, lv));
        if (bj < 0) continue;
        const unsigned s2 = ((unsigned)bj << (3 * LOGB)) | local_index<LOGB>(c.x, c.y, c.z, lv);
        if (__ldg(L.rec + s2) != kEmptyRec) {
          if (occupied) err |= ERR_OVERLAP;
          else v = s2;
          break;
        }
      }
    }
    view[slot] = v;
    scal[slot] = occupied ? __uint_as_float((unsigned)(r >> 32)) : 0.f;
    occ += occupied ? 1u : 0u;
  }
  if (err) atomicOr(&sc->err, err);
  // occupied-slot count (duplicate labels show as fewer slots than cells)
  __shared__ unsigned occ_w[32];
  occ = __reduce_add_sync(kFull, occ);
  if ((threadIdx.x & 31) == 0) occ_w[threadIdx.x >> 5] = occ;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned t = threadIdx.x < (blockDim.x >> 5) ? occ_w[threadIdx.x] : 0u;
    t = __reduce_add_sync(kFull, t);
    if (threadIdx.x == 0 && t) atomicAdd(&sc->n_occupied, (unsigned long long)t);
  }
}

// Pass over (brick, neighbour) pairs: for every brick its 26 neighbouring
// brick regions (and itself) resolved once - the same-level brick there, or
// the first coarser brick covering that region, or none. An aligned level-l
// brick region lies inside exactly one brick region of each coarser level,
// so one brick answers for the whole neighbour region. Value: brick index |
// level << 27, or -1.
template <int LOGB>
__global__ void __launch_bounds__(256) k_brick_neighbors(Locator L, long long n_bricks,
                                                         int* __restrict__ nbr) {
  constexpr int B = 1 << LOGB;
  const long long total = n_bricks * 27;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const long long bi = i / 27;
    const int t = (int)(i - bi * 27);
    const int4 b = __ldg(L.bricks + bi);
    const int l = b.w;
    int out = -1;
    if (t == 13) {
      out = (int)bi | (l << 27);
    } else {
      const int ext = B << l;
      const int qx = b.x + (t % 3 - 1) * ext, qy = b.y + ((t / 3) % 3 - 1) * ext,
                qz = b.z + (t / 9 - 1) * ext;
      for (int lv = l; lv < L.levels; ++lv) {
        const int bj = find_brick(L, brick_key<LOGB>(qx, qy, qz, lv));
        if (bj >= 0) { out = bj | (lv << 27); break; }
      }
    }
    nbr[i] = out;
  }
}

// ---------------------------------------------------------------------------
// Dual cells (Sec. 4.2 - 4.4)
// ---------------------------------------------------------------------------

// 27-bit masks over the 3x3x3 neighbourhood (offset o = ox + 3 oy + 9 oz,
// o in {0,1,2}^3 relative to the cell minus one) of the 8 vertices of dual
// delta (vertices at offsets delta + e) and of the vertices with e below the
// cell's own position e_S = 1 - delta.
struct DualMasks {
  unsigned all[8];
  unsigned lower[8];
};

__host__ __device__ constexpr DualMasks make_dual_masks() {
  DualMasks m{};
  for (int d = 0; d < 8; ++d) {
    const int dx = d & 1, dy = (d >> 1) & 1, dz = d >> 2;
    const int es = 7 - d;
    unsigned all = 0, lower = 0;
    for (int e = 0; e < 8; ++e) {
      const int o = (dx + (e & 1)) + 3 * (dy + ((e >> 1) & 1)) + 9 * (dz + (e >> 2));
      all |= 1u << o;
      if (e < es) lower |= 1u << o;
    }
    m.all[d] = all;
    m.lower[d] = lower;
  }
  return m;
}

__constant__ DualMasks c_masks = make_dual_masks();

// The one-cell halo of a brick's (B+2)^3 region as a list, so that the
// threads load it without walking (and skipping) the interior: per entry
// the region coordinates rx, ry, rz (4 bits each), the neighbour region
// nbi = 0..26 (5 bits) and the Morton index of the cell inside a same-level
// neighbour brick (from bit 17).
template <int LOGB>
struct HaloList {
  static constexpr int B = 1 << LOGB, R = B + 2;
  static constexpr int kCount = R * R * R - B * B * B;
  unsigned e[kCount];
};

template <int LOGB>
__host__ __device__ constexpr HaloList<LOGB> make_halo_list() {
  HaloList<LOGB> h{};
  constexpr int B = HaloList<LOGB>::B, R = HaloList<LOGB>::R;
  int k = 0;
  for (int rz = 0; rz < R; ++rz)
    for (int ry = 0; ry < R; ++ry)
      for (int rx = 0; rx < R; ++rx) {
        if (rx >= 1 && rx <= B && ry >= 1 && ry <= B && rz >= 1 && rz <= B) continue;
        const int nbi = (rx == 0 ? 0 : (rx == R - 1 ? 2 : 1)) + 3 * (ry == 0 ? 0 : (ry == R - 1 ? 2 : 1)) +
                        9 * (rz == 0 ? 0 : (rz == R - 1 ? 2 : 1));
        const int lx = (rx - 1 + B) % B, ly = (ry - 1 + B) % B, lz = (rz - 1 + B) % B;
        unsigned m = 0;
        for (int b = 0; b < LOGB; ++b)
          m |= (unsigned)(((lx >> b) & 1) << (3 * b)) | (unsigned)(((ly >> b) & 1) << (3 * b + 1)) |
               (unsigned)(((lz >> b) & 1) << (3 * b + 2));
        h.e[k++] = (unsigned)rx | ((unsigned)ry << 4) | ((unsigned)rz << 8) | ((unsigned)nbi << 12) | (m << 17);
      }
  return h;
}

__device__ const HaloList<2> g_halo2 = make_halo_list<2>();
__device__ const HaloList<3> g_halo3 = make_halo_list<3>();

template <int LOGB>
__device__ __forceinline__ const unsigned* halo_list() {
  if constexpr (LOGB == 2) return g_halo2.e;
  else return g_halo3.e;
}

// ---------------------------------------------------------------------------
// Marching Cubes on dual cells (Sec. 5, 5.1, 5.2)
// ---------------------------------------------------------------------------

struct McShared {
  unsigned long long packed[256];
  unsigned char count[256];
};

__device__ __forceinline__ void load_mc(McShared& sh, const McConst& mc) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    sh.packed[i] = mc.packed[i];
    sh.count[i] = mc.count[i];
  }
}

constexpr unsigned kDistinct = 0x80000000u;   // dual flag: 8 different cells (slots stay below 2^31)

// Reads dual d; returns its kDistinct flag (cleared from v[0]).
__device__ __forceinline__ bool load_dual(const uint4* __restrict__ duals, long long d, unsigned v[8]) {
  const uint4 a = __ldcs(duals + 2 * d);   // streamed: keep the scalars in L2 instead
  const uint4 c = __ldcs(duals + 2 * d + 1);
  v[0] = a.x & ~kDistinct; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = c.x; v[5] = c.y; v[6] = c.z; v[7] = c.w;
  return (a.x & kDistinct) != 0;
}

// v[i] for a run-time i without moving v to local memory.
__device__ __forceinline__ unsigned sel8(const unsigned v[8], int i) {
  unsigned r = v[0];
#pragma unroll
  for (int e = 1; e < 8; ++e) r = (i == e) ? v[e] : r;
  return r;
}

// Edge key (unordered pair of cells) of hexahedron edge k.
__device__ __forceinline__ unsigned long long edge_key(const unsigned v[8], int k,
                                                       unsigned long long ea, unsigned long long eb) {
  const unsigned a = sel8(v, (int)((ea >> (4 * k)) & 15)), b = sel8(v, (int)((eb >> (4 * k)) & 15));
  return a < b ? ((unsigned long long)a << 32) | b : ((unsigned long long)b << 32) | a;
}

// Bit t set when triangle t of the case has three different edge keys.
__device__ __forceinline__ unsigned kept_triangles(unsigned long long packed, int cnt, const unsigned v[8],
                                                   unsigned long long ea, unsigned long long eb) {
  unsigned keep = 0;
  for (int t = 0; t < cnt; ++t) {
    const unsigned long long k0 = edge_key(v, (int)((packed >> (12 * t)) & 15), ea, eb);
    const unsigned long long k1 = edge_key(v, (int)((packed >> (12 * t + 4)) & 15), ea, eb);
    const unsigned long long k2 = edge_key(v, (int)((packed >> (12 * t + 8)) & 15), ea, eb);
    if (k0 != k1 && k1 != k2 && k0 != k2) keep |= 1u << t;
  }
  return keep;
}

// kept_triangles, short-cut for a dual of 8 different cells: no two of its
// edges share an edge key, so every triangle of the case is kept.
__device__ __forceinline__ unsigned kept_of(bool distinct, unsigned long long packed, int cnt, const unsigned v[8],
                                            unsigned long long ea, unsigned long long eb) {
  return distinct ? (1u << cnt) - 1u : kept_triangles(packed, cnt, v, ea, eb);
}

// Interpolated vertex on the edge between cells a and b: from the cell with
// the lower (z,y,x) corner, t = (iso - sa) / (sb - sa), P = ca + t (cb - ca),
// every operation rounded on its own (no contraction).
__device__ __forceinline__ float3 edge_vertex(int4 pa, float sa, int4 pb, float sb, float iso) {
  const bool swap = (pb.z < pa.z) || (pb.z == pa.z && (pb.y < pa.y || (pb.y == pa.y && pb.x < pa.x)));
  if (swap) {
    const int4 tp = pa; pa = pb; pb = tp;
    const float ts = sa; sa = sb; sb = ts;
  }
  const float ha = __fmul_rn(__int2float_rn(1 << pa.w), 0.5f);
  const float hb = __fmul_rn(__int2float_rn(1 << pb.w), 0.5f);
  const float d = __fsub_rn(sb, sa);
  const float t = __fdiv_rn(__fsub_rn(iso, sa), d);
  float3 p;
  {
    const float ca = __fadd_rn(__int2float_rn(pa.x), ha), cb = __fadd_rn(__int2float_rn(pb.x), hb);
    p.x = __fadd_rn(ca, __fmul_rn(t, __fsub_rn(cb, ca)));
  }
  {
    const float ca = __fadd_rn(__int2float_rn(pa.y), ha), cb = __fadd_rn(__int2float_rn(pb.y), hb);
    p.y = __fadd_rn(ca, __fmul_rn(t, __fsub_rn(cb, ca)));
  }
  {
    const float ca = __fadd_rn(__int2float_rn(pa.z), ha), cb = __fadd_rn(__int2float_rn(pb.z), hb);
    p.z = __fadd_rn(ca, __fmul_rn(t, __fsub_rn(cb, ca)));
  }
  return p;
}

// Warp-level append: exclusive prefix of k over the warp plus one atomic per
// warp; returns this lane's first output index.
__device__ __forceinline__ long long warp_append(unsigned k, unsigned long long* counter) {
  const int lane = threadIdx.x & 31;
  unsigned incl = k;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  const unsigned total = __shfl_sync(kFull, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total) base = atomicAdd(counter, (unsigned long long)total);
  base = __shfl_sync(kFull, base, 31);
  return (long long)base + incl - k;
}

// Writes the kept triangles of one dual. The dual's 8 vertex slots and
// scalars sit in this thread's shared-memory row (indexed by table-driven
// corner numbers, which registers cannot be).
template <int LOGB>
__device__ __forceinline__ void write_triangles(const int4* __restrict__ bricks, const unsigned* vr,
                                                const float* sr, float iso, unsigned long long packed,
                                                unsigned keep, long long idx, long long cap,
                                                float* __restrict__ tris, unsigned long long ea,
                                                unsigned long long eb) {
  for (int t = 0; t < 5; ++t) {
    if (!((keep >> t) & 1u)) continue;
    if (idx < cap) {
      float* out = tris + 9 * idx;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int k = (int)((packed >> (12 * t + 4 * c)) & 15);
        const int a = (int)((ea >> (4 * k)) & 15), b = (int)((eb >> (4 * k)) & 15);
        const float3 q = edge_vertex(slot_cell<LOGB>(bricks, vr[a]), sr[a], slot_cell<LOGB>(bricks, vr[b]),
                                     sr[b], iso);
        out[3 * c + 0] = q.x;
        out[3 * c + 1] = q.y;
        out[3 * c + 2] = q.z;
      }
    }
    ++idx;
  }
}

constexpr int kRow = 9;   // shared-memory row stride (words): conflict-free across a warp
constexpr int kTriStage = 80;   // triangles a warp stages in shared memory per step

__device__ __forceinline__ void stage_row(unsigned* vr, float* sr, const unsigned v[8], const float sv[8]) {
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    vr[e] = v[e];
    sr[e] = sv[e];
  }
}

__device__ __forceinline__ int case_of(const unsigned v[8], float sv[8], const float* __restrict__ scal,
                                       float iso) {
  int cas = 0;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    sv[e] = __ldg(scal + v[e]);
    cas |= (sv[e] > iso ? 1 : 0) << e;
  }
  return cas;
}

// Threads of the dual-cell CTA: one per brick slot up to 256, so that eight
// CTAs fit an SM at B = 8 (each thread then owns two cells).
template <int LOGB>
struct DualShape {
  static constexpr int kCells = 1 << (3 * LOGB);
  static constexpr int kThreads = kCells < 256 ? kCells : 256;
  static constexpr int kPerThread = kCells / kThreads;
};

// One CTA per brick. The CTA loads the brick's resolved views plus a
// one-cell halo ((B+2)^3 entries, from the 26 neighbouring bricks of the same
// level or the first coarser brick that covers them) into shared memory,
// marking same-level cells in bit 31, and condenses every row of the region
// into a mask (bit x: a cell exists, bit 16+x: it is of this brick's level).
// Each cell then reads 9 row masks and decides its 8 duals: a dual is emitted
// iff every vertex exists (rule 1), none is finer (rule 2: finer regions
// resolve to kReject) and every same-level vertex comes after the cell in
// (z,y,x) order (rule 3). Survivors are compacted with one atomic per CTA.
//
// With ISO, the same pass also runs Marching Cubes at `iso` on every dual it
// emits (the first iso-value of a data set, fused as in the paper's single
// extraction kernel): the region's scalars are staged in shared memory too,
// and the kept triangles are appended with one atomic per warp - the same
// triangles, bit for bit, as k_mc over the resident dual list.
//
// Only cells whose lower corner's x lies in [own_x0, own_x1) emit (the
// owner slab of a sharded data set; the whole range otherwise): every other
// cell still takes part in its neighbours' rules.
template <int LOGB, bool ISO>
__global__ void __launch_bounds__(DualShape<LOGB>::kThreads) k_dual_cells(
    Locator L, const int* __restrict__ nbr, const int* __restrict__ order, long long n_bricks,
    uint4* __restrict__ duals, long long cap, Scratch* sc, float iso, float* __restrict__ tris, long long tri_cap,
    int own_x0, int own_x1, const __grid_constant__ McConst mc) {
  constexpr int B = 1 << LOGB;
  constexpr int R = B + 2;
  constexpr int NT = DualShape<LOGB>::kThreads;
  constexpr int CPT = DualShape<LOGB>::kPerThread;
  constexpr int NR = R * R * R;
  // padded region layout: row stride RS, plane stride PS, chosen so that the
  // 32 cells of a warp (a 4x4x2 Morton block) hit 32 different banks
  constexpr int RS = R + 2;
  constexpr int PS = ((RS * R + 15) / 32) * 32 + (RS % 8 == 0 ? 4 : 16) +
                     (((RS * R + 15) / 32) * 32 + (RS % 8 == 0 ? 4 : 16) < RS * R ? 32 : 0);
  constexpr int NP = PS * R;
  constexpr int NW = (NT + 31) / 32;
  constexpr unsigned kSame = 0x80000000u;   // slot indices stay below 2^31
  __shared__ unsigned rv[NP];
  __shared__ unsigned rmask[R * R];
  __shared__ unsigned wsum[NW + 1];
  __shared__ unsigned long long cta_base;
  __shared__ float rsc[ISO ? NP : 1];                 // scalars of the region's cells
  __shared__ McShared msh;
  // ISO: per warp the step's triangle list and staged vertices (the stage
  // doubles as the warp's per-thread rows when the list overflows)
  __shared__ unsigned tlist[ISO ? NW : 1][ISO ? kTriStage : 1];
  __shared__ __align__(16) float tstage[ISO ? NW : 1][ISO ? kTriStage * 9 : 1];
  static_assert(!ISO || 32 * 2 * kRow <= kTriStage * 9, "fallback rows fit the stage");
  const int t = threadIdx.x;
  const int lane = t & 31, wp = t >> 5;
  if (ISO) {
    load_mc(msh, mc);   // made visible by the first barrier below
  }
  int c0[CPT], px[CPT], py[CPT], pz[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const int m = t + j * NT;   // Morton index of the cell inside the brick
    px[j] = compact<LOGB>(m);
    py[j] = compact<LOGB>(m >> 1);
    pz[j] = compact<LOGB>(m >> 2);
    c0[j] = px[j] + RS * py[j] + PS * pz[j];   // neighbourhood origin (cell - 1)
  }
  for (int row = t; row < R * R; row += NT) rmask[row] = 0;   // cleared again after each use
  __syncthreads();
  for (int it = blockIdx.x; it < n_bricks; it += gridDim.x) {   // n_bricks * B^3 < 2^31
    // bricks in the given spatial order (neighbours' halos then stay in L2)
    const int bi = order ? __ldg(order + it) : it;
    const int4 b = __ldg(L.bricks + bi);
    const int l = b.w;
    bool mine[CPT];
    bool level_only = true;   // every region entry this thread loads is a cell of level l
#pragma unroll
    for (int j = 0; j < CPT; ++j) {   // the brick itself: coalesced reads
      const unsigned s2 = ((unsigned)bi << (3 * LOGB)) | (unsigned)(t + j * NT);
      const unsigned v = __ldg(L.view + s2);
      mine[j] = v == s2;
      level_only = level_only && mine[j];
      const int r = c0[j] + 1 + RS + PS;
      rv[r] = mine[j] ? (v | kSame) : v;
    }
    const unsigned* halo = halo_list<LOGB>();
    for (int k = t; k < HaloList<LOGB>::kCount; k += NT) {   // the one-cell halo
      const unsigned h = __ldg(halo + k);
      const int rx = (int)(h & 15u), ry = (int)((h >> 4) & 15u), rz = (int)((h >> 8) & 15u);
      const int e = __ldg(nbr + bi * 27 + ((h >> 12) & 31u));
      unsigned v = kReject;
      bool same = false;
      if (e >= 0) {
        const int fb = e & ((1 << 27) - 1), lv = e >> 27;
        unsigned s2;
        if (lv == l) {
          s2 = ((unsigned)fb << (3 * LOGB)) | (h >> 17);
        } else {
          const int x = b.x + ((rx - 1) << l), y = b.y + ((ry - 1) << l), z = b.z + ((rz - 1) << l);
          s2 = ((unsigned)fb << (3 * LOGB)) | local_index<LOGB>(x, y, z, lv);
        }
        v = __ldg(L.view + s2);
        same = lv == l && v == s2;
      }
      rv[rx + RS * ry + PS * rz] = same ? (v | kSame) : v;
      level_only = level_only && same;
    }
    // A region made only of level-l cells leaves each cell exactly one dual:
    // the one it is the lowest vertex of (d = 7); rules 1-3 need not run,
    // and the row masks are built only for the other bricks.
    const bool uniform = __syncthreads_and(level_only) != 0;
    if (!uniform) {
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const unsigned v = rv[c0[j] + 1 + RS + PS];
        if (v != kReject)
          atomicOr(&rmask[(py[j] + 1) + R * (pz[j] + 1)],
                   (1u << (px[j] + 1)) | ((v & kSame) ? 1u << (16 + px[j] + 1) : 0u));
      }
      for (int k = t; k < HaloList<LOGB>::kCount; k += NT) {
        const unsigned h = __ldg(halo + k);
        const int rx = (int)(h & 15u), ry = (int)((h >> 4) & 15u), rz = (int)((h >> 8) & 15u);
        const unsigned v = rv[rx + RS * ry + PS * rz];
        if (v != kReject) atomicOr(&rmask[ry + R * rz], (1u << rx) | ((v & kSame) ? 1u << (16 + rx) : 0u));
      }
      __syncthreads();
    }
    if (ISO) {
      for (int q = t; q < NR; q += NT) {
        const int r = q % R + RS * ((q / R) % R) + PS * (q / (R * R));
        const unsigned v = rv[r];
        rsc[r] = v != kReject ? __ldg(L.scal + (v & ~kSame)) : 0.f;
      }
      __syncthreads();
    }
    unsigned emit[CPT];
    unsigned cnt = 0;   // per-thread dual count of cell j in bits 16j..16j+15
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      emit[j] = 0;
      if (!mine[j]) continue;   // the slot holds no level-l cell
      const int cx = b.x + (px[j] << l);
      if (cx < own_x0 || cx >= own_x1) continue;   // owned by another slab
      if (uniform) {
        emit[j] = 0x80u;
        cnt += 1u << (16 * j);
        continue;
      }
      unsigned exist = 0, samem = 0;
#pragma unroll
      for (int oz = 0; oz < 3; ++oz)
#pragma unroll
        for (int oy = 0; oy < 3; ++oy) {
          const unsigned m = rmask[(py[j] + oy) + R * (pz[j] + oz)];
          const int sh = 3 * oy + 9 * oz;
          exist |= ((m >> px[j]) & 7u) << sh;
          samem |= ((m >> (16 + px[j])) & 7u) << sh;
        }
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        const bool ok = ((exist & c_masks.all[d]) == c_masks.all[d]) && !(samem & c_masks.lower[d]);
        emit[j] |= (ok ? 1u : 0u) << d;
      }
      cnt += (unsigned)__popc(emit[j]) << (16 * j);
    }
    // CTA-wide exclusive scan of the packed counts: the duals of all cells
    // t (first half) come before those of all cells t + NT, keeping the
    // output in the brick's Morton order (totals stay below 2^16)
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wp] = incl;
    __syncthreads();
    for (int row = t; row < R * R; row += NT) rmask[row] = 0;   // every cell has read its masks
    if (t == 0) {
      unsigned run = 0;
      for (int w = 0; w < NW; ++w) {
        const unsigned x = wsum[w];
        wsum[w] = run;
        run += x;
      }
      wsum[NW] = run;   // packed per-half totals
      unsigned tot = 0;
#pragma unroll
      for (int j = 0; j < CPT; ++j) tot += (run >> (16 * j)) & 0xFFFFu;
      cta_base = tot ? atomicAdd(&sc->n_dual, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    const unsigned excl = wsum[wp] + incl - cnt;
    long long half_base = (long long)cta_base;
    unsigned ntri = 0;   // ISO: kept triangles of this thread's duals
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      long long idx = half_base + ((excl >> (16 * j)) & 0xFFFFu);
      half_base += (wsum[NW] >> (16 * j)) & 0xFFFFu;
      for (unsigned todo = emit[j]; todo; todo &= todo - 1u) {   // the emitted duals only
        const int d = __ffs(todo) - 1;
        const int rd = c0[j] + (d & 1) + RS * ((d >> 1) & 1) + PS * (d >> 2);
        unsigned v[8];
        unsigned all_same = kSame;
        int cas = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int r = rd + (e & 1) + RS * ((e >> 1) & 1) + PS * (e >> 2);
          all_same &= rv[r];
          v[e] = rv[r] & ~kSame;
          if (ISO) cas |= (rsc[r] > iso ? 1 : 0) << e;
        }
        // 8 same-level cells at 8 positions are 8 different cells (kSame and
        // kDistinct are the same bit)
        if (idx < cap) {   // written once, read much later: evict first
          __stcs(duals + 2 * idx, make_uint4(v[0] | all_same, v[1], v[2], v[3]));
          __stcs(duals + 2 * idx + 1, make_uint4(v[4], v[5], v[6], v[7]));
        }
        ++idx;
        if (ISO && msh.count[cas])
          ntri += __popc(kept_of(all_same != 0, msh.packed[cas], msh.count[cas], v, mc.edge_a, mc.edge_b));
      }
    }
    if (ISO) {   // append this warp's triangles, then compute their vertices lane-parallel
      long long tidx = warp_append(ntri, &sc->n_tri[0]);
      const unsigned total = __reduce_add_sync(kFull, ntri);
      const long long first = __shfl_sync(kFull, tidx, 0);
      float* wst = tstage[wp];
      unsigned* lst = tlist[wp];
      if (total <= (unsigned)kTriStage) {
        unsigned pos = (unsigned)(tidx - first);
#pragma unroll 1
        for (int j = 0; j < CPT; ++j) {
          if (!ntri) break;
#pragma unroll 1
          for (int d = 0; d < 8; ++d) {
            if (!((emit[j] >> d) & 1u)) continue;
            const int dx = d & 1, dy = (d >> 1) & 1, dz = d >> 2;
            unsigned v[8];
            unsigned all_same = kSame;
            int cas = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int r = c0[j] + (dx + (e & 1)) + RS * (dy + ((e >> 1) & 1)) + PS * (dz + (e >> 2));
              all_same &= rv[r];
              v[e] = rv[r] & ~kSame;
              cas |= (rsc[r] > iso ? 1 : 0) << e;
            }
            if (!msh.count[cas]) continue;
            const unsigned long long pk = msh.packed[cas];
            const unsigned keep = kept_of(all_same != 0, pk, msh.count[cas], v, mc.edge_a, mc.edge_b);
            for (int tt = 0; tt < 5; ++tt)   // entry: source lane, cell j, dual d, the triangle's 3 edges
              if ((keep >> tt) & 1u)
                lst[pos++] = (unsigned)lane | ((unsigned)j << 5) | ((unsigned)d << 6) |
                             (((unsigned)(pk >> (12 * tt)) & 0xFFFu) << 9);
          }
        }
        __syncwarp();
        for (unsigned q = lane; q < 3u * total; q += 32) {   // one vertex per lane
          const unsigned e = q / 3u, c = q - 3u * e;
          const unsigned ent = lst[e];
          const int m = wp * 32 + (int)(ent & 31u) + (int)((ent >> 5) & 1u) * NT;   // the source cell
          const int d = (int)((ent >> 6) & 7u);
          const int cb = compact<LOGB>(m) + (d & 1) + RS * (compact<LOGB>(m >> 1) + ((d >> 1) & 1)) +
                         PS * (compact<LOGB>(m >> 2) + (d >> 2));
          const int k = (int)((ent >> (9 + 4 * c)) & 15u);
          const int a = (int)((mc.edge_a >> (4 * k)) & 15), b = (int)((mc.edge_b >> (4 * k)) & 15);
          const int ra = cb + (a & 1) + RS * ((a >> 1) & 1) + PS * (a >> 2);
          const int rb = cb + (b & 1) + RS * ((b >> 1) & 1) + PS * (b >> 2);
          const float3 p = edge_vertex(slot_cell<LOGB>(L.bricks, rv[ra] & ~kSame), rsc[ra],
                                       slot_cell<LOGB>(L.bricks, rv[rb] & ~kSame), rsc[rb], iso);
          wst[3 * q] = p.x;
          wst[3 * q + 1] = p.y;
          wst[3 * q + 2] = p.z;
        }
        __syncwarp();
        const long long lim = min((long long)total, tri_cap - first) * 9;   // capacity: exact prefix only
        for (long long k = lane; k < lim; k += 32) tris[9 * first + k] = wst[k];
      } else {   // more triangles than the stage holds: each thread writes its own
        unsigned* vr = reinterpret_cast<unsigned*>(wst) + lane * 2 * kRow;
        float* sr = wst + lane * 2 * kRow + kRow;
#pragma unroll 1
        for (int j = 0; j < CPT; ++j) {
          if (!ntri) break;
#pragma unroll 1
          for (int d = 0; d < 8; ++d) {
            if (!((emit[j] >> d) & 1u)) continue;
            const int dx = d & 1, dy = (d >> 1) & 1, dz = d >> 2;
            unsigned v[8];
            float sv[8];
            unsigned all_same = kSame;
            int cas = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int r = c0[j] + (dx + (e & 1)) + RS * (dy + ((e >> 1) & 1)) + PS * (dz + (e >> 2));
              all_same &= rv[r];
              v[e] = rv[r] & ~kSame;
              sv[e] = rsc[r];
              cas |= (sv[e] > iso ? 1 : 0) << e;
            }
            if (!msh.count[cas]) continue;
            const unsigned keep = kept_of(all_same != 0, msh.packed[cas], msh.count[cas], v, mc.edge_a, mc.edge_b);
            if (!keep) continue;
            stage_row(vr, sr, v, sv);
            write_triangles<LOGB>(L.bricks, vr, sr, iso, msh.packed[cas], keep, tidx, tri_cap, tris, mc.edge_a,
                                  mc.edge_b);
            tidx += __popc(keep);
          }
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
}

// Dynamic shared memory of k_mc<·, EMIT> per CTA of 256 threads: per warp
// 64 rows (two duals per lane) of 8 vertex slots, a list of the step's kept
// triangles and their staged vertices (46 KB with the static table: four
// CTAs per SM).
constexpr int kMcRowsWords = 8 * 64 * kRow;
constexpr int kMcSmemBytes = 4 * (kMcRowsWords + 8 * kTriStage + 8 * kTriStage * 9);

// One lane per dual, two duals per lane per step: gather the 8 vertex
// scalars, build the case index (bit e set iff s_e > iso), keep the case's
// triangles that have three different edge keys and append them with one
// atomic per warp. The vertices are then computed lane-parallel: each lane
// with triangles stages its duals' slots and scalars and lists its kept
// triangles; the warp's 32 lanes take the step's 3T vertices in turn, stage
// them, and write the step's triangles as one coalesced run. Optionally
// writes per-dual case and triangle count instead.
// A dual's tuple (32 bytes) on its way to L2 ahead of its load.
__device__ __forceinline__ void prefetch_dual(const uint4* duals, long long d) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(duals + 2 * d));
}

// Edge key of a triangle vertex: the unordered pair of slots it interpolates
// between (slots stay below 2^31), smaller first.
__device__ __forceinline__ unsigned long long slot_pair(unsigned a, unsigned b) {
  return a < b ? ((unsigned long long)a << 32) | b : ((unsigned long long)b << 32) | a;
}

// KEYS: instead of vertex positions, each triangle's 3 edge keys (u64) go to
// tris reinterpreted as [cap][3] u64 (for the indexed face set).
// TAG: besides each triangle, tags[row] = the index of its dual cell in the
// list (what lets a reader check the triangles dual by dual).
template <int LOGB, bool EMIT, bool CASES, bool KEYS = false, bool TAG = false>
__global__ void __launch_bounds__(256, 4) k_mc(Locator L, const uint4* __restrict__ duals, long long nd,
                                            float iso, float* __restrict__ tris, long long cap,
                                            unsigned long long* counter, unsigned char* cases,
                                            unsigned char* ntri, long long* __restrict__ tags,
                                            const __grid_constant__ McConst mc) {
  __shared__ McShared sh;
  extern __shared__ __align__(16) unsigned mc_smem[];
  __shared__ unsigned short cell_tab[1 << (3 * LOGB)];
  load_mc(sh, mc);
  fill_cell_table<LOGB>(cell_tab);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + w;
  unsigned* rows_v = mc_smem + w * 64 * kRow;                               // [64][kRow]
  unsigned* list = mc_smem + kMcRowsWords + w * kTriStage;                 // [kTriStage]
  float* wst = reinterpret_cast<float*>(mc_smem + kMcRowsWords + 8 * kTriStage) + w * kTriStage * 9;
  for (long long base = wid * 64; base < nd; base += nwarps * 64) {
    const long long d0 = base + lane, d1 = base + 32 + lane;
    const bool a0 = d0 < nd, a1 = d1 < nd;
    if (!KEYS) {   // the warp's next step, fetched while this one runs (measured: the keys
                   // variant ran 60 % slower with it, the others 4 % faster)
      const long long n0 = d0 + nwarps * 64, n1 = d1 + nwarps * 64;
      if (n0 < nd) prefetch_dual(duals, n0);
      if (n1 < nd) prefetch_dual(duals, n1);
    }
    unsigned v0[8], v1[8];
    float s0[8], s1[8];
    bool x0 = false, x1 = false;
    if (a0) x0 = load_dual(duals, d0, v0);
    if (a1) x1 = load_dual(duals, d1, v1);
    int c0 = 0, c1 = 0;
    if (a0) c0 = case_of(v0, s0, L.scal, iso);
    if (a1) c1 = case_of(v1, s1, L.scal, iso);
    unsigned k0 = 0, k1 = 0;
    if (a0 && sh.count[c0]) k0 = kept_of(x0, sh.packed[c0], sh.count[c0], v0, mc.edge_a, mc.edge_b);
    if (a1 && sh.count[c1]) k1 = kept_of(x1, sh.packed[c1], sh.count[c1], v1, mc.edge_a, mc.edge_b);
    if (CASES) {
      if (a0) {
        if (cases) cases[d0] = (unsigned char)c0;
        if (ntri) ntri[d0] = (unsigned char)__popc(k0);
      }
      if (a1) {
        if (cases) cases[d1] = (unsigned char)c1;
        if (ntri) ntri[d1] = (unsigned char)__popc(k1);
      }
    }
    if (EMIT) {
      if (__ballot_sync(kFull, (k0 | k1) != 0) == 0) continue;
      const unsigned mine = __popc(k0) + __popc(k1);
      // the warp's run of output rows: one atomic per warp, whose result is
      // read only where the rows are written, so that its round trip
      // overlaps the vertex work
      unsigned incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned total = __shfl_sync(kFull, incl, 31), excl = incl - mine;
      unsigned long long wbase = 0;
      if (lane == 31) wbase = atomicAdd(counter, (unsigned long long)total);
      unsigned* r0 = rows_v + lane * kRow;   // rows lane and 32 + lane: conflict-free
      if (k0) {
#pragma unroll
        for (int e = 0; e < 8; ++e) r0[e] = v0[e];
      }
      if (k1) {
#pragma unroll
        for (int e = 0; e < 8; ++e) r0[32 * kRow + e] = v1[e];
      }
      if (total <= (unsigned)kTriStage) {
        unsigned pos = excl;
        const unsigned long long p0 = sh.packed[c0], p1 = sh.packed[c1];
        for (int t = 0; t < 5; ++t)
          if ((k0 >> t) & 1u) list[pos++] = (unsigned)lane | ((unsigned)(p0 >> (12 * t)) & 0xFFFu) << 8;
        for (int t = 0; t < 5; ++t)
          if ((k1 >> t) & 1u) list[pos++] = (32u + lane) | ((unsigned)(p1 >> (12 * t)) & 0xFFFu) << 8;
        __syncwarp();
        for (unsigned q = lane; q < 3u * total; q += 32) {   // one vertex per lane
          const unsigned e = q / 3u, c = q - 3u * e;
          const unsigned ent = list[e];
          const unsigned* rv = rows_v + (ent & 0xFFu) * kRow;
          const int k = (int)((ent >> (8 + 4 * c)) & 15u);
          const int a = (int)((mc.edge_a >> (4 * k)) & 15), b = (int)((mc.edge_b >> (4 * k)) & 15);
          const unsigned va = rv[a], vb = rv[b];   // scalars gathered again: just read, so cached
          if (KEYS) {
            reinterpret_cast<unsigned long long*>(wst)[q] = slot_pair(va, vb);
          } else {
            const float3 p = edge_vertex(slot_cell_tab<LOGB>(L.bricks, cell_tab, va), __ldg(L.scal + va),
                                         slot_cell_tab<LOGB>(L.bricks, cell_tab, vb), __ldg(L.scal + vb), iso);
            wst[3 * q] = p.x;
            wst[3 * q + 1] = p.y;
            wst[3 * q + 2] = p.z;
          }
        }
        __syncwarp();
        const long long first = (long long)__shfl_sync(kFull, wbase, 31);
        if (KEYS) {
          const long long lim = min((long long)total, cap - first) * 3;
          unsigned long long* out = reinterpret_cast<unsigned long long*>(tris) + 3 * first;
          for (long long k = lane; k < lim; k += 32) out[k] = reinterpret_cast<const unsigned long long*>(wst)[k];
        } else {
          const long long lim = min((long long)total, cap - first) * 9;   // capacity: exact prefix only
          for (long long k = lane; k < lim; k += 32) tris[9 * first + k] = wst[k];
          if (TAG)
            for (long long k = lane; k < lim / 9; k += 32) tags[first + k] = base + (long long)(list[k] & 0xFFu);
        }
        __syncwarp();
      } else if (KEYS) {   // more triangles than the stage holds: each lane writes its own keys
        long long idx = (long long)__shfl_sync(kFull, wbase, 31) + excl;
        unsigned long long* out = reinterpret_cast<unsigned long long*>(tris);
        const unsigned long long kp[2] = {sh.packed[c0], sh.packed[c1]};
        const unsigned km[2] = {k0, k1};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const unsigned* rv = r0 + 32 * kRow * j;
          for (int t = 0; t < 5; ++t) {
            if (!((km[j] >> t) & 1u)) continue;
            if (idx < cap) {
#pragma unroll
              for (int cc = 0; cc < 3; ++cc) {
                const int kk = (int)((kp[j] >> (12 * t + 4 * cc)) & 15);
                out[3 * idx + cc] = slot_pair(rv[(mc.edge_a >> (4 * kk)) & 15], rv[(mc.edge_b >> (4 * kk)) & 15]);
              }
            }
            ++idx;
          }
        }
        __syncwarp();
      } else {   // more triangles than the stage holds: each lane writes its own (scalars in the stage)
        long long idx = (long long)__shfl_sync(kFull, wbase, 31) + excl;
        float* q0 = wst + lane * 2 * kRow;
        if (k0) {
#pragma unroll
          for (int e = 0; e < 8; ++e) q0[e] = s0[e];
          write_triangles<LOGB>(L.bricks, r0, q0, iso, sh.packed[c0], k0, idx, cap, tris, mc.edge_a, mc.edge_b);
          if (TAG)
            for (int t = 0; t < __popc(k0); ++t)
              if (idx + t < cap) tags[idx + t] = d0;
          idx += __popc(k0);
        }
        if (k1) {
#pragma unroll
          for (int e = 0; e < 8; ++e) q0[kRow + e] = s1[e];
          write_triangles<LOGB>(L.bricks, r0 + 32 * kRow, q0 + kRow, iso, sh.packed[c1], k1, idx, cap, tris,
                                mc.edge_a, mc.edge_b);
          if (TAG)
            for (int t = 0; t < __popc(k1); ++t)
              if (idx + t < cap) tags[idx + t] = d1;
        }
        __syncwarp();
      }
    }
  }
}

// Indexed face set, welding pass: every triangle vertex's edge key goes into
// a hash table (16-byte entries {key, vertex index}, Fibonacci home, linear
// probing); the thread whose CAS places a key numbers the vertex (one atomic
// per warp), computes its position once and records its cells' input
// indices. Neighbouring triangles share edges, so a warp's 32 keys repeat:
// only the first lane holding each distinct key probes. A probe run longer
// than `limit` sets ERR_HASH_FULL (the host rebuilds the table larger).
template <int LOGB>
__global__ void __launch_bounds__(256) k_weld_insert(Locator L, const unsigned long long* __restrict__ tkeys,
                                                     long long n_keys, ulonglong2* wtab, unsigned long long wmask,
                                                     float iso, float* __restrict__ vtx, int* __restrict__ vkeys,
                                                     long long vcap, Scratch* sc) {
  const unsigned long long limit = wmask < 4095ull ? wmask + 1 : 4096ull;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long nk = (n_keys + 31) & ~31ll;   // whole warps, for the warp-wide append
  unsigned err = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += stride) {
    const bool live = i < n_keys;
    const unsigned long long key = live ? __ldcs(tkeys + i) : kEmptyKey;
    const unsigned peers = __match_any_sync(kFull, key);   // lanes holding the same key
    bool won = false;
    unsigned long long h = 0;
    if (live && (threadIdx.x & 31) == __ffs(peers) - 1) {
      h = home_of(key, wmask);
      bool done = false;
      for (unsigned long long p = 0; p < limit; ++p) {
        const unsigned long long c = __ldcg(&wtab[h].x);
        if (c == key) { done = true; break; }
        if (c == kEmptyKey) {
          const unsigned long long prev = atomicCAS(&wtab[h].x, kEmptyKey, key);
          if (prev == kEmptyKey) { won = true; done = true; break; }
          if (prev == key) { done = true; break; }
        }
        h = (h + 1) & wmask;
      }
      if (!done) err |= ERR_HASH_FULL;
    }
    const long long vid = warp_append(won ? 1u : 0u, &sc->n_vtx);
    if (won) {
      wtab[h].y = (unsigned long long)vid;
      if (vid < vcap) {
        const unsigned va = (unsigned)(key >> 32), vb = (unsigned)key;
        const float3 p = edge_vertex(slot_cell<LOGB>(L.bricks, va), __ldg(L.scal + va),
                                     slot_cell<LOGB>(L.bricks, vb), __ldg(L.scal + vb), iso);
        vtx[3 * vid] = p.x;
        vtx[3 * vid + 1] = p.y;
        vtx[3 * vid + 2] = p.z;
        if (vkeys) {   // the edge's two cells as input indices, smaller first
          const int ia = (int)(unsigned)__ldg(L.rec + va), ib = (int)(unsigned)__ldg(L.rec + vb);
          vkeys[2 * vid] = min(ia, ib);
          vkeys[2 * vid + 1] = max(ia, ib);
        }
      }
    }
  }
  err = warp_or(err);
  if ((threadIdx.x & 31) == 0 && err) atomicOr(&sc->err, err);
}

// Indexed face set, index pass: each triangle's three keys looked up in the
// completed table, once per distinct key of a warp.
__global__ void __launch_bounds__(256) k_weld_index(const unsigned long long* __restrict__ tkeys, long long n_tri,
                                                    const ulonglong2* __restrict__ wtab, unsigned long long wmask,
                                                    int* __restrict__ tri) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long nk = (3 * n_tri + 31) & ~31ll;   // whole warps: the lanes share lookups
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += stride) {
    const bool live = i < 3 * n_tri;
    const unsigned long long key = live ? __ldcs(tkeys + i) : kEmptyKey;
    const unsigned peers = __match_any_sync(kFull, key);   // lanes holding the same key
    const int leader = __ffs(peers) - 1;
    int vid = -1;
    if (live && (threadIdx.x & 31) == leader) {
      unsigned long long h = home_of(key, wmask);
      for (unsigned long long p = 0; p <= wmask; ++p) {   // every key is in the table
        const ulonglong2 e = __ldg(wtab + h);
        if (e.x == key) { vid = (int)e.y; break; }
        if (e.x == kEmptyKey) break;
        h = (h + 1) & wmask;
      }
    }
    vid = __shfl_sync(kFull, vid, leader);
    if (live) tri[i] = vid;
  }
}

// Batched iso-values over one or several resident dual lists (one launch per
// pass for all of them). Each dual list is cut into tiles (batch_tile duals);
// a job is one data set's dual list with its run of iso-values, and every
// (job, iso-value) pair owns one output segment. Three passes:
//   k_batch_count: per tile, the kept triangles of every iso-value of its
//     job (each dual's vertex slots and scalars read once for all values,
//     work only for the (dual, iso-value) pairs that cross);
//   k_batch_scan: per segment, the exclusive prefix over the job's tiles
//     (each tile's first row inside the segment) and the segment's total;
//     k_batch_bases: the segments' first rows (the caller's offsets);
//   k_batch_emit: per tile, the same crossing pairs again; each pair
//     reserves its triangles inside the tile's run of its segment with a
//     shared-memory atomic, and the warp computes the listed triangles'
//     vertices together and writes them to their rows.
// No global atomics and no waiting: every tile knows where its triangles go.
__device__ __forceinline__ int job_of_tile(const BatchTable& T, long long g) {
  int j = 0;
  while (j + 1 < T.n_jobs && g >= T.job[j + 1].tile0) ++j;
  return j;
}

// The job's iso-values in increasing order, sorted once per tile. A dual
// crosses iso (its case is neither 0 nor 255) exactly when
// min(scalars) <= iso < max(scalars), so the values crossing it are one run
// [below(min), below(max)) of the sorted list: the passes below visit only
// (dual, iso-value) pairs that cross, spread evenly over the warp's lanes.
struct BatchIsos {
  float v[kMaxIso];             // sorted values (NaN last, ties by index)
  unsigned char idx[kMaxIso];   // each one's index in the job's run
};

__device__ __forceinline__ bool iso_before(float b, int j, float a, int k) {
  if (b != b) return a != a && j < k;
  return a != a || b < a || (b == a && j < k);
}

// S from the job's values iso[0..n) (a rank per value), by the lanes of one
// warp.
__device__ __forceinline__ void batch_sort_isos(const float* __restrict__ iso, int n, BatchIsos& S) {
  for (int k = threadIdx.x & 31; k < n; k += 32) {
    const float a = __ldg(iso + k);
    int r = 0;
    for (int j = 0; j < n; ++j) r += iso_before(__ldg(iso + j), j, a, k) ? 1 : 0;
    S.v[r] = a;
    S.idx[r] = (unsigned char)k;
  }
}

// How many of the n sorted values lie below x (a NaN never does).
__device__ __forceinline__ int batch_below(const BatchIsos& S, int n, float x) {
  int lo = 0;
#pragma unroll
  for (int s = kMaxIso; s > 0; s >>= 1)
    if (lo + s <= n && S.v[lo + s - 1] < x) lo += s;
  return lo;
}

__device__ __forceinline__ unsigned warp_incl_scan(unsigned x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// The warp's pairs are numbered lane by lane (lane j owns [excl_j, excl_j +
// n_j)); the owner of pair p is the last lane whose first pair is <= p.
// Every lane of the warp takes part (the shuffles read other lanes' excl).
__device__ __forceinline__ int pair_owner(unsigned excl, unsigned p) {
  int src = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const unsigned e = __shfl_sync(kFull, excl, src + s);
    if (e <= p) src += s;
  }
  return src;
}

// Case index of a dual at iso from its 8 scalars s[e * stride].
__device__ __forceinline__ int batch_case(const float* s, int stride, float iso) {
  int cas = 0;
#pragma unroll
  for (int e = 0; e < 8; ++e) cas |= (s[e * stride] > iso ? 1 : 0) << e;
  return cas;
}

// Kept-triangle mask of a crossing dual: every triangle of its case when its
// 8 vertices are 8 different cells, else the non-degenerate ones (slots
// v[e * stride]).
__device__ __forceinline__ unsigned batch_kept(bool distinct, int cas, const unsigned* v, int stride,
                                               const McShared& sh, unsigned long long ea, unsigned long long eb) {
  if (distinct) return (1u << sh.count[cas]) - 1u;
  unsigned vv[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) vv[e] = v[e * stride];
  return kept_triangles(sh.packed[cas], sh.count[cas], vv, ea, eb);
}

// Duals per warp step of k_batch_count (two per lane).
constexpr int kCountStep = 64;

// A tile's iso-values and counters in k_batch_count: tiles are handed to
// warps, so that a warp never waits for the other warps of its CTA.
struct CountTile {
  BatchIsos S;
  unsigned cnt[kMaxIso];   // by position in S
};

__global__ void __launch_bounds__(256, 5) k_batch_count(const __grid_constant__ BatchTable T,
                                                     const float* __restrict__ isos, unsigned* __restrict__ counts,
                                                     const __grid_constant__ McConst mc) {
  __shared__ McShared sh;
  __shared__ CountTile tiles[8];
  __shared__ unsigned wv[8][8][kCountStep];   // per warp: vertex slot e of dual i at [e][i]
  __shared__ float wsc[8][8][kCountStep];     // and its scalar
  load_mc(sh, mc);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  CountTile& C = tiles[w];
  const BatchIsos& S = C.S;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long g = (long long)blockIdx.x * (blockDim.x >> 5) + w; g < T.n_tiles; g += nwarps) {
    const BatchJob& J = T.job[job_of_tile(T, g)];
    const long long t = g - J.tile0;
    const int n_iso = J.n_iso;
    for (int k = lane; k < n_iso; k += 32) C.cnt[k] = 0;
    batch_sort_isos(isos + J.q0, n_iso, C.S);
    __syncwarp();
    const long long d_hi = min(J.nd, (t + 1) * J.tile);
    for (long long base = t * J.tile; base < d_hi; base += kCountStep) {
      if (base + kCountStep + lane < d_hi) prefetch_dual(J.duals, base + kCountStep + lane);
      if (base + kCountStep + 32 + lane < d_hi) prefetch_dual(J.duals, base + kCountStep + 32 + lane);
      // duals lane and lane + 32 of the step: slots and scalars to shared
      // memory, the run of sorted iso-values crossing each
      int klo0 = 0, n0 = 0, klo1 = 0, n1 = 0;
      unsigned dm0 = 0, dm1 = 0;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const long long d = base + lane + 32 * j;
        const int i = lane + 32 * j;
        bool distinct = false;
        int klo = 0, n = 0;
        if (d < d_hi) {
          unsigned v[8];
          float sv[8];
          distinct = load_dual(J.duals, d, v);
          float mn = 3.4e38f, mx = -3.4e38f;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            sv[e] = __ldg(J.scal + v[e]);
            mn = fminf(mn, sv[e]);
            mx = fmaxf(mx, sv[e]);
          }
          klo = batch_below(S, n_iso, mn);
          n = max(0, batch_below(S, n_iso, mx) - klo);
          if (n > 0) {   // (the slots matter only for a dual of fewer than 8 cells)
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              if (!distinct) wv[w][e][i] = v[e];
              wsc[w][e][i] = sv[e];
            }
          }
        }
        const unsigned dm = __ballot_sync(kFull, distinct);
        if (j == 0) { klo0 = klo; n0 = n; dm0 = dm; } else { klo1 = klo; n1 = n; dm1 = dm; }
      }
      const unsigned mine = (unsigned)(n0 + n1);
      const unsigned incl = warp_incl_scan(mine, lane), excl = incl - mine;
      const unsigned n_pairs = __shfl_sync(kFull, incl, 31);
      __syncwarp();
      for (unsigned p0 = 0; p0 < n_pairs; p0 += 32) {
        const unsigned p = p0 + lane;
        const int src = pair_owner(excl, p);
        const int r = (int)(p - __shfl_sync(kFull, excl, src));
        const int sn0 = __shfl_sync(kFull, n0, src);
        const int slo0 = __shfl_sync(kFull, klo0, src), slo1 = __shfl_sync(kFull, klo1, src);
        if (p >= n_pairs) continue;   // no shuffles below
        const bool second = r >= sn0;
        const int i = src + (second ? 32 : 0);
        const int ks = second ? slo1 + r - sn0 : slo0 + r;
        const int cas = batch_case(&wsc[w][0][i], kCountStep, S.v[ks]);
        const unsigned keep = batch_kept((((second ? dm1 : dm0) >> src) & 1u) != 0, cas, &wv[w][0][i], kCountStep,
                                         sh, mc.edge_a, mc.edge_b);
        if (keep) atomicAdd(&C.cnt[ks], (unsigned)__popc(keep));
      }
      __syncwarp();
    }
    for (int k = lane; k < n_iso; k += 32) counts[J.cbase + (long long)S.idx[k] * J.tiles + t] = C.cnt[k];
    __syncwarp();
  }
}

// One CTA per segment: rel[...] = exclusive prefix of the segment's tile
// counts, totals[q] = their sum.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
__global__ void __launch_bounds__(kScanThreads) k_batch_scan(const __grid_constant__ BatchTable T,
                                                            const unsigned* __restrict__ counts,
                                                            long long* __restrict__ rel, long long* totals) {
  __shared__ long long ws[kScanThreads / 32 + 1];
  const int q = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  int j = 0;
  while (j + 1 < T.n_jobs && q >= T.job[j + 1].q0) ++j;
  const BatchJob& J = T.job[j];
  const long long n = J.tiles;
  const unsigned* c = counts + J.cbase + (long long)(q - J.q0) * n;
  long long* r = rel + J.cbase + (long long)(q - J.q0) * n;
  long long running = 0;
  for (long long c0 = 0; c0 < n; c0 += (long long)kScanThreads * kScanPer) {
    unsigned v[kScanPer];
    long long sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      const long long i = c0 + (long long)t * kScanPer + k;
      v[k] = i < n ? c[i] : 0u;
      sum += v[k];
    }
    long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    if (w == 0) {
      const long long x = ws[lane];
      long long cc = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, cc, o);
        if (lane >= o) cc += y;
      }
      ws[lane] = cc - x;
      if (lane == 31) ws[32] = cc;
    }
    __syncthreads();
    long long ex = running + ws[w] + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      const long long i = c0 + (long long)t * kScanPer + k;
      if (i < n) r[i] = ex;
      ex += v[k];
    }
    running += ws[32];
    __syncthreads();
  }
  if (t == 0) totals[q] = running;
}

// off[q] = first row of segment q (exclusive prefix of the totals),
// off[n_q] = all rows. One thread.
__global__ void k_batch_bases(int n_q, const long long* totals, long long* off) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long run = 0;
  for (int q = 0; q < n_q; ++q) {
    off[q] = run;
    run += totals[q];
  }
  off[n_q] = run;
}

// Per warp of k_batch_emit, the 32 duals of a warp step, by (vertex, dual):
// vertex e of dual i at [e][i], so that lanes reading one vertex of
// different duals meet in different banks (the float4 rows carry one entry
// of padding: lanes reading vertex e of dual i and vertex e' of dual i'
// share a bank group only when e + i == e' + i' mod 8).
struct BatchWarp {
  float4 c[8][33];              // centre x, y, z and scalar (the fp32 operations of edge_vertex)
  float s[8][32];               // the scalars again, for the case loop
  unsigned char ab[12][32];     // per edge its two vertices, the lower one in (z, y, x) order first
};
// A tile's iso-values and rows in k_batch_emit: tiles are handed to warps,
// so that a warp never waits for the other warps of its CTA.
struct EmitTile {           // per iso-value, by position in S:
  BatchIsos S;
  unsigned tcnt[kMaxIso];      // rows of the tile taken so far
  long long row0[kMaxIso];     // the tile's first row
  long long rowend[kMaxIso];   // end of the segment's rows that fit the buffer
};
// Triangles a warp lists before computing their vertices (one round of 32
// pairs adds at most 32 x 5).
constexpr int kBatchList = 224;

// Vertex on edge k of dual i at iso: from the cell with the lower corner,
// t = (iso - sa) / (sb - sa), P = ca + t (cb - ca), every operation rounded
// on its own (edge_vertex's order).
__device__ __forceinline__ float3 batch_vertex(const BatchWarp& W, int i, int k, float iso) {
  const unsigned ab = W.ab[k][i];
  const float4 pa = W.c[ab & 15u][i], pb = W.c[ab >> 4][i];
  const float t = __fdiv_rn(__fsub_rn(iso, pa.w), __fsub_rn(pb.w, pa.w));
  return make_float3(__fadd_rn(pa.x, __fmul_rn(t, __fsub_rn(pb.x, pa.x))),
                     __fadd_rn(pa.y, __fmul_rn(t, __fsub_rn(pb.y, pa.y))),
                     __fadd_rn(pa.z, __fmul_rn(t, __fsub_rn(pb.z, pa.z))));
}

// List entry of k_batch_emit: the triangle's row inside its tile's run of
// its segment (bits 0-31), the dual's lane (32-36), the iso-value's position
// among the job's sorted values (37-42) and the triangle's three edge ids
// (43-54).
__device__ __forceinline__ unsigned long long batch_entry(unsigned row, unsigned lane, unsigned k, unsigned edges) {
  return (unsigned long long)row | ((unsigned long long)lane << 32) | ((unsigned long long)k << 37) |
         ((unsigned long long)edges << 43);
}

// The warp's listed triangles, one vertex per lane in turn: interpolated
// from the dual's vertex data and written straight to its row (a run of
// consecutive rows per segment, so consecutive lanes write consecutive
// 12-byte vertices). fits: every row of the job lies below the capacity.
__device__ __forceinline__ void batch_flush(const unsigned long long* lst, unsigned len, const BatchWarp& W,
                                            const EmitTile& E, float* __restrict__ tris, bool fits) {
  for (unsigned q = threadIdx.x & 31; q < 3u * len; q += 32) {
    const unsigned e = q / 3u, c = q - 3u * e;
    const unsigned long long ent = lst[e];
    const unsigned hi = (unsigned)(ent >> 32);   // lane, iso-value, edges
    const unsigned k = (hi >> 5) & 63u;
    const long long row = E.row0[k] + (long long)(unsigned)ent;
    if (!fits && row >= E.rowend[k]) continue;   // capacity: exact prefix only
    const float3 p = batch_vertex(W, (int)(hi & 31u), (int)((hi >> (11 + 4 * c)) & 15u), E.S.v[k]);
    float* out = tris + 9 * row + 3 * c;
    out[0] = p.x;
    out[1] = p.y;
    out[2] = p.z;
  }
}

__global__ void __launch_bounds__(256, 3) k_batch_emit(const __grid_constant__ BatchTable T,
                                                    const float* __restrict__ isos,
                                                    const long long* __restrict__ rel,
                                                    const long long* __restrict__ off, float* __restrict__ tris,
                                                    long long total_cap, const __grid_constant__ McConst mc) {
  __shared__ McShared sh;
  __shared__ unsigned short cell_tab3[1 << 9], cell_tab2[1 << 6];
  __shared__ EmitTile tiles[8];
  __shared__ BatchWarp wdata[8];
  __shared__ unsigned long long tlist[8][kBatchList];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long* lst = tlist[w];
  BatchWarp& W = wdata[w];
  EmitTile& E = tiles[w];
  load_mc(sh, mc);
  fill_cell_table<3>(cell_tab3);
  fill_cell_table<2>(cell_tab2);
  __syncthreads();
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long g = (long long)blockIdx.x * (blockDim.x >> 5) + w; g < T.n_tiles; g += nwarps) {
    const BatchJob& J = T.job[job_of_tile(T, g)];
    const long long t = g - J.tile0;
    const int n_iso = J.n_iso;
    batch_sort_isos(isos + J.q0, n_iso, E.S);
    __syncwarp();
    const BatchIsos& S = E.S;
    for (int ks = lane; ks < n_iso; ks += 32) {
      const int k = S.idx[ks];
      E.tcnt[ks] = 0;
      E.row0[ks] = __ldg(off + J.q0 + k) + __ldg(rel + J.cbase + (long long)k * J.tiles + t);
      E.rowend[ks] = min(__ldg(off + J.q0 + k + 1), total_cap);
    }
    __syncwarp();
    const bool fits = __ldg(off + J.q0 + n_iso) <= total_cap;   // every row of the job fits
    const long long d_hi = min(J.nd, (t + 1) * J.tile);
    for (long long base = t * J.tile; base < d_hi; base += 32) {
      const long long d = base + lane;
      if (d + 32 < d_hi) prefetch_dual(J.duals, d + 32);
      bool distinct = false;
      int klo = 0, n = 0;
      unsigned v[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};   // (slot 0 stands in past the tile's end)
      float sv[8];
      if (d < d_hi) {
        distinct = load_dual(J.duals, d, v);
        float mn = 3.4e38f, mx = -3.4e38f;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          sv[e] = __ldg(J.scal + v[e]);
          mn = fminf(mn, sv[e]);
          mx = fmaxf(mx, sv[e]);
        }
        klo = batch_below(S, n_iso, mn);
        n = max(0, batch_below(S, n_iso, mx) - klo);
      }
      if (__any_sync(kFull, n > 0)) {   // vertex data of the warp's crossing duals, once for all values
        // the hexahedron's 12 edges (a, b), a < b, in increasing order: the
        // numbering the case table's edge ids use
        constexpr int kEa[12] = {0, 0, 0, 1, 1, 2, 2, 3, 4, 4, 5, 6};
        constexpr int kEb[12] = {1, 2, 4, 3, 5, 3, 6, 7, 5, 6, 7, 7};
        unsigned sw = 0;   // bit k: edge k's vertex b's cell lies lower in (z, y, x) order
        if (__all_sync(kFull, distinct || n == 0)) {
          // every crossing dual of the step is 8 cells of one level: they sit
          // one width apart along each axis from vertex 0's, and no edge
          // is reversed
          const int4 c0 = J.logb == 3 ? slot_cell_tab<3>(J.bricks, cell_tab3, v[0])
                                      : slot_cell_tab<2>(J.bricks, cell_tab2, v[0]);
          const float h = __fmul_rn(__int2float_rn(1 << c0.w), 0.5f);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int x = c0.x + ((e & 1) << c0.w), y = c0.y + (((e >> 1) & 1) << c0.w),
                      z = c0.z + ((e >> 2) << c0.w);
            W.c[e][lane] = make_float4(__fadd_rn(__int2float_rn(x), h), __fadd_rn(__int2float_rn(y), h),
                                       __fadd_rn(__int2float_rn(z), h), sv[e]);
            W.s[e][lane] = sv[e];
          }
        } else {
          int lmin = 64, lmax = -1;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int4 cr = J.logb == 3 ? slot_cell_tab<3>(J.bricks, cell_tab3, v[e])
                                        : slot_cell_tab<2>(J.bricks, cell_tab2, v[e]);
            lmin = min(lmin, cr.w);
            lmax = max(lmax, cr.w);
            const float h = __fmul_rn(__int2float_rn(1 << cr.w), 0.5f);
            W.c[e][lane] = make_float4(__fadd_rn(__int2float_rn(cr.x), h), __fadd_rn(__int2float_rn(cr.y), h),
                                       __fadd_rn(__int2float_rn(cr.z), h), sv[e]);
            W.s[e][lane] = sv[e];
            if (e == 3) __syncwarp();   // at most four cells' loads in flight per lane: fewer live registers
          }
          // edge k's bit: its vertex b's cell lies lower in (z, y, x) order.
          // With all 8 cells on one level the cells sit one width apart along
          // each edge's axis, so no bit is set; otherwise compare the corners,
          // as one 64-bit key each relative to vertex 0's corner (they differ
          // by less than 2^16 per axis: every vertex cell holds a point within
          // one cell width of the dual's owner), an edge's bit taken as soon
          // as its upper vertex's key is known
          if (__any_sync(kFull, lmin != lmax)) {
            unsigned long long key[8];
            int c0x = 0, c0y = 0, c0z = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int4 cr = J.logb == 3 ? slot_cell_tab<3>(J.bricks, cell_tab3, v[e])
                                          : slot_cell_tab<2>(J.bricks, cell_tab2, v[e]);
              if (e == 0) { c0x = cr.x; c0y = cr.y; c0z = cr.z; }
              key[e] = ((unsigned long long)(unsigned)(cr.z - c0z + 65536) << 34) |
                       ((unsigned long long)(unsigned)(cr.y - c0y + 65536) << 17) | (unsigned)(cr.x - c0x + 65536);
#pragma unroll
              for (int k = 0; k < 12; ++k)
                if (kEb[k] == e) sw |= (key[e] < key[kEa[k]] ? 1u : 0u) << k;
              if (e == 3) __syncwarp();
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k)
          W.ab[k][lane] = (unsigned char)(((sw >> k) & 1u) ? (kEb[k] | (kEa[k] << 4)) : (kEa[k] | (kEb[k] << 4)));
      }
      const unsigned dmask = __ballot_sync(kFull, distinct);
      const unsigned incl = warp_incl_scan((unsigned)n, lane), excl = incl - (unsigned)n;
      const unsigned n_pairs = __shfl_sync(kFull, incl, 31);
      __syncwarp();
      unsigned len = 0;   // entries in the warp's list
      for (unsigned p0 = 0; p0 < n_pairs; p0 += 32) {
        const unsigned p = p0 + lane;
        const int src = pair_owner(excl, p);
        const int ks = __shfl_sync(kFull, klo, src) + (int)(p - __shfl_sync(kFull, excl, src));
        const bool live = p < n_pairs;
        unsigned keep = 0;
        int cas = 0;
        if (live) {
          cas = batch_case(&W.s[0][src], 32, S.v[ks]);
          if ((dmask >> src) & 1u) {
            keep = (1u << sh.count[cas]) - 1u;
          } else {   // a dual of fewer than 8 cells: its slots again (about 2 % of duals)
            unsigned vv[8];
            load_dual(J.duals, base + src, vv);
            keep = kept_triangles(sh.packed[cas], sh.count[cas], vv, mc.edge_a, mc.edge_b);
          }
        }
        const unsigned c = __popc(keep);
        const unsigned ci = warp_incl_scan(c, lane);
        const unsigned total = __shfl_sync(kFull, ci, 31);
        if (total == 0) continue;
        if (len + total > (unsigned)kBatchList) {   // list full: its vertices first
          __syncwarp();
          batch_flush(lst, len, W, E, tris, fits);
          __syncwarp();
          len = 0;
        }
        if (c) {
          unsigned row = atomicAdd(&E.tcnt[ks], c);   // rows inside the tile's run of the segment
          unsigned pos = len + ci - c;
          const unsigned long long pk = sh.packed[cas];
          for (int tt = 0; tt < 5; ++tt)
            if ((keep >> tt) & 1u)
              lst[pos++] = batch_entry(row++, (unsigned)src, (unsigned)ks, (unsigned)(pk >> (12 * tt)) & 0xFFFu);
        }
        len += total;
      }
      __syncwarp();
      batch_flush(lst, len, W, E, tris, fits);
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(256) k_get_duals(const uint4* __restrict__ duals, long long nd,
                                                   const unsigned long long* __restrict__ rec,
                                                   int* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * nd; i += stride) {
    const uint4 a = __ldg(duals + i);   // first word of a dual: kDistinct cleared
    reinterpret_cast<int4*>(out)[i] = make_int4((int)__ldg(rec + ((i & 1) ? a.x : (a.x & ~kDistinct))),
                                                (int)__ldg(rec + a.y),
                                                (int)__ldg(rec + a.z), (int)__ldg(rec + a.w));
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------

#define AMR_DISPATCH(logb, ...)            \
  do {                                     \
    if ((logb) == 2) {                     \
      constexpr int LB = 2;                \
      __VA_ARGS__;                         \
    } else {                               \
      constexpr int LB = 3;                \
      __VA_ARGS__;                         \
    }                                      \
  } while (0)

cudaError_t launch_insert_bricks(int logb, const int* xyz, const unsigned char* lvl, const float* s,
                                 long long n, ulonglong2* htab,
                                 unsigned long long hmask, int4* bricks,
                                 unsigned long long brick_limit, Scratch* sc, int grid, int block,
                                 unsigned* codes, cudaStream_t st) {
  AMR_DISPATCH(logb, (k_insert_bricks<LB><<<grid, block, 0, st>>>(xyz, lvl, s, n, htab, hmask,
                                                                   bricks, brick_limit, sc, codes)));
  return cudaGetLastError();
}

cudaError_t launch_scatter_cells(int logb, const int* xyz, const unsigned char* lvl, const float* s,
                                 long long n, Locator loc, unsigned long long* rec, Scratch* sc,
                                 int grid, int block, cudaStream_t st) {
  AMR_DISPATCH(logb, (k_scatter_cells<LB><<<grid, block, 0, st>>>(xyz, lvl, s, n, loc, rec, sc)));
  return cudaGetLastError();
}

BinLayout bin_layout(long long n_slots) {
  BinLayout b;
  b.n_coarse = (n_slots + (1ll << kCoarseShift) - 1) >> kCoarseShift;
  b.n_win = (n_slots + kWinSlots - 1) >> kWinShift;
  b.stage_a = b.n_coarse << kCoarseShift;
  b.stage_b = b.n_win << kWinShift;
  b.bytes = (size_t)(12 * (b.stage_a + b.stage_b) + 4 * (b.n_coarse + b.n_win));
  return b;
}

namespace {
constexpr int kSmemCoarse = (2 * kMaxCoarse + 3 * kCoarseTile) * 4;
constexpr int kSmemFine = (2 * kFinePerCoarse + 3 * kFineTile) * 4;
constexpr int kSmemPlace = kWinSlots * 8;

struct Stages {
  Stage a, b;
  unsigned* coarse_count;
  unsigned* win_count;
};

Stages stages_of(const BinLayout& lay, void* staging) {
  unsigned* base = static_cast<unsigned*>(staging);
  unsigned* bb = base + 3 * lay.stage_a;
  Stages S;
  S.a = Stage{base, base + lay.stage_a, base + 2 * lay.stage_a};
  S.b = Stage{bb, bb + lay.stage_b, bb + 2 * lay.stage_b};
  S.coarse_count = bb + 3 * lay.stage_b;
  S.win_count = S.coarse_count + lay.n_coarse;
  return S;
}
}  // namespace

cudaError_t launch_bin_coarse(int logb, const float* s, long long n, Locator loc, long long n_slots, void* staging,
                              Scratch* sc, int sm_count, const unsigned* codes, cudaStream_t st) {
  const BinLayout lay = bin_layout(n_slots);
  if (n_slots <= 0) return cudaSuccess;
  if (lay.n_coarse > kMaxCoarse || n > 0xFFFFFFFFll || !codes) return cudaErrorInvalidValue;
  const Stages S = stages_of(lay, staging);
  cudaError_t e = cudaMemsetAsync(S.coarse_count, 0, 4 * (size_t)(lay.n_coarse + lay.n_win), st);
  if (e != cudaSuccess) return e;
  // dynamic shared memory above the 48 KB default (an attribute of the
  // current device's context, so set on every build)
  if ((e = cudaFuncSetAttribute(k_bin_coarse<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCoarse)) ||
      (e = cudaFuncSetAttribute(k_bin_coarse<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCoarse)) ||
      (e = cudaFuncSetAttribute(k_bin_fine, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFine)) ||
      (e = cudaFuncSetAttribute(k_place_windows<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemPlace)) ||
      (e = cudaFuncSetAttribute(k_place_windows<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemPlace)))
    return e;
  if (n <= 0) return cudaSuccess;
  const long long tiles = (n + kCoarseTile - 1) / kCoarseTile;
  const int smem_coarse = (2 * (int)lay.n_coarse + 3 * kCoarseTile) * 4;   // kSmemCoarse at most
  AMR_DISPATCH(logb, ({
    int per_sm = 0;   // one resident wave: the tile loop is grid-strided
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_coarse<LB>, kCoarseThreads,
                                                           smem_coarse)) != cudaSuccess)
      return e;
    const int grid = (int)std::min<long long>(tiles, (long long)sm_count * std::max(per_sm, 1));
    k_bin_coarse<LB><<<grid, kCoarseThreads, smem_coarse, st>>>(s, n, loc, (int)lay.n_coarse, S.a, S.coarse_count,
                                                                sc, codes);
  }));
  return cudaGetLastError();
}

cudaError_t launch_bin_fine(long long n_slots, void* staging, Scratch* sc, cudaStream_t st) {
  const BinLayout lay = bin_layout(n_slots);
  if (n_slots <= 0) return cudaSuccess;
  const Stages S = stages_of(lay, staging);
  k_bin_fine<<<dim3((1u << kCoarseShift) / kFineTile, (unsigned)lay.n_coarse), kFineThreads, kSmemFine, st>>>(
      S.a, S.coarse_count, S.b, S.win_count, sc);
  return cudaGetLastError();
}

cudaError_t launch_place_windows(int logb, long long n_slots, void* staging, unsigned long long* rec, unsigned* view,
                                 float* scal, unsigned* elist, Scratch* sc, cudaStream_t st) {
  const BinLayout lay = bin_layout(n_slots);
  if (n_slots <= 0) return cudaSuccess;
  const Stages S = stages_of(lay, staging);
  AMR_DISPATCH(logb, (k_place_windows<LB><<<(unsigned)lay.n_win, kPlaceThreads, kSmemPlace, st>>>(
                         S.b, S.win_count, n_slots, rec, view, scal, elist, sc)));
  return cudaGetLastError();
}

cudaError_t launch_resolve_empty(int logb, Locator loc, const unsigned* elist, const Scratch* sc, unsigned* view,
                                 int grid, cudaStream_t st) {
  AMR_DISPATCH(logb, (k_resolve_empty<LB><<<grid, 256, 0, st>>>(loc, elist, sc, view)));
  return cudaGetLastError();
}

cudaError_t launch_resolve_views(int logb, Locator loc, unsigned* view, float* scal, long long n_slots,
                                 int check_overlap, Scratch* sc, int grid, int block,
                                 cudaStream_t st) {
  AMR_DISPATCH(logb, (k_resolve_views<LB><<<grid, block, 0, st>>>(loc, view, scal, n_slots, check_overlap,
                                                                   sc)));
  return cudaGetLastError();
}

cudaError_t launch_brick_neighbors(int logb, Locator loc, long long n_bricks, int* nbr, int grid,
                                   cudaStream_t st) {
  if (n_bricks <= 0) return cudaSuccess;
  AMR_DISPATCH(logb, (k_brick_neighbors<LB><<<grid, 256, 0, st>>>(loc, n_bricks, nbr)));
  return cudaGetLastError();
}

cudaError_t launch_dual_cells(int logb, Locator loc, const int* nbr, const int* order, long long n_bricks,
                              uint4* duals, long long cap, Scratch* sc, cudaStream_t st, int own_x0, int own_x1) {
  if (n_bricks <= 0) return cudaSuccess;
  const int grid = (int)(n_bricks < (1ll << 30) ? n_bricks : (1ll << 30));
  McConst none{};
  AMR_DISPATCH(logb, (k_dual_cells<LB, false><<<grid, DualShape<LB>::kThreads, 0, st>>>(
                         loc, nbr, order, n_bricks, duals, cap, sc, 0.f, nullptr, 0, own_x0, own_x1, none)));
  return cudaGetLastError();
}

cudaError_t launch_dual_cells_iso(int logb, Locator loc, const int* nbr, const int* order, long long n_bricks,
                                  uint4* duals, long long cap, Scratch* sc, float iso, float* tris,
                                  long long tri_cap, const McConst& mc, cudaStream_t st) {
  if (n_bricks <= 0) return cudaSuccess;
  const int grid = (int)(n_bricks < (1ll << 30) ? n_bricks : (1ll << 30));
  AMR_DISPATCH(logb, (k_dual_cells<LB, true><<<grid, DualShape<LB>::kThreads, 0, st>>>(
                         loc, nbr, order, n_bricks, duals, cap, sc, iso, tris, tri_cap, INT_MIN, INT_MAX, mc)));
  return cudaGetLastError();
}

cudaError_t launch_mc(int logb, Locator loc, const uint4* duals, long long nd, float iso, float* tris,
                      long long cap, unsigned long long* counter, unsigned char* cases,
                      unsigned char* ntri, const McConst& mc, int grid, cudaStream_t st, long long* tags) {
  if (nd <= 0) return cudaSuccess;
  // dynamic shared memory above the 48 KB default (an attribute of the
  // current device's context, so set on every launch)
  if (cases || ntri) {
    AMR_DISPATCH(logb, (k_mc<LB, false, true><<<grid, 256, 0, st>>>(loc, duals, nd, iso, tris, cap, counter,
                                                                     cases, ntri, nullptr, mc)));
  } else if (tags) {
    AMR_DISPATCH(logb, ({
      const cudaError_t e = cudaFuncSetAttribute(k_mc<LB, true, false, false, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kMcSmemBytes);
      if (e != cudaSuccess) return e;
      k_mc<LB, true, false, false, true><<<grid, 256, kMcSmemBytes, st>>>(loc, duals, nd, iso, tris, cap, counter,
                                                                         nullptr, nullptr, tags, mc);
    }));
  } else {
    AMR_DISPATCH(logb, ({
      const cudaError_t e =
          cudaFuncSetAttribute(k_mc<LB, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMcSmemBytes);
      if (e != cudaSuccess) return e;
      k_mc<LB, true, false><<<grid, 256, kMcSmemBytes, st>>>(loc, duals, nd, iso, tris, cap, counter, cases, ntri,
                                                             nullptr, mc);
    }));
  }
  return cudaGetLastError();
}

cudaError_t launch_mc_keys(int logb, Locator loc, const uint4* duals, long long nd, float iso,
                           unsigned long long* tkeys, long long cap, unsigned long long* counter, const McConst& mc,
                           int grid, cudaStream_t st) {
  if (nd <= 0) return cudaSuccess;
  AMR_DISPATCH(logb, ({
    const cudaError_t e =
        cudaFuncSetAttribute(k_mc<LB, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMcSmemBytes);
    if (e != cudaSuccess) return e;
    k_mc<LB, true, false, true><<<grid, 256, kMcSmemBytes, st>>>(loc, duals, nd, iso, reinterpret_cast<float*>(tkeys),
                                                                  cap, counter, nullptr, nullptr, nullptr, mc);
  }));
  return cudaGetLastError();
}

cudaError_t launch_weld_insert(int logb, Locator loc, const unsigned long long* tkeys, long long n_keys,
                               ulonglong2* wtab, unsigned long long wmask, float iso, float* vtx, int* vkeys,
                               long long vcap, Scratch* sc, int grid, cudaStream_t st) {
  if (n_keys <= 0) return cudaSuccess;
  AMR_DISPATCH(logb, (k_weld_insert<LB><<<grid, 256, 0, st>>>(loc, tkeys, n_keys, wtab, wmask, iso, vtx, vkeys, vcap,
                                                               sc)));
  return cudaGetLastError();
}

cudaError_t launch_weld_index(const unsigned long long* tkeys, long long n_tri, const ulonglong2* wtab,
                              unsigned long long wmask, int* tri, int grid, cudaStream_t st) {
  if (n_tri <= 0) return cudaSuccess;
  k_weld_index<<<grid, 256, 0, st>>>(tkeys, n_tri, wtab, wmask, tri);
  return cudaGetLastError();
}

int batch_tile(long long nd) {
  int t = kBTile;
  while (t > 256 && nd < 16384ll * t) t >>= 1;
  return t;
}

void batch_add_job(BatchTable& T, const uint4* duals, const float* scal, const int4* bricks, long long nd, int logb,
                   int n_iso) {
  BatchJob& J = T.job[T.n_jobs];
  J.duals = duals;
  J.scal = scal;
  J.bricks = bricks;
  J.nd = nd;
  J.logb = logb;
  J.tile0 = T.n_tiles;
  J.tile = batch_tile(nd);
  J.tiles = (nd + J.tile - 1) / J.tile;
  J.cbase = T.n_counters;
  J.q0 = T.n_q;
  J.n_iso = n_iso;
  T.n_tiles += J.tiles;
  T.n_counters += J.tiles * n_iso;
  T.n_q += n_iso;
  T.n_jobs += 1;
}

size_t batch_workspace_bytes(long long n_counters) { return (size_t)n_counters * 12 + 8 * (kMaxIso + 1); }

namespace {
struct BatchWs {
  unsigned* counts;
  long long* rel;
  long long* totals;
};
BatchWs batch_ws(const BatchTable& T, void* ws) {
  long long* rel = static_cast<long long*>(ws);
  long long* totals = rel + T.n_counters;
  unsigned* counts = reinterpret_cast<unsigned*>(totals + kMaxIso + 1);
  return BatchWs{counts, rel, totals};
}
}  // namespace

cudaError_t launch_batch_count(const BatchTable& T, const float* isos, void* ws, const McConst& mc, int grid,
                               cudaStream_t st) {
  if (T.n_tiles <= 0) return cudaSuccess;
  const BatchWs W = batch_ws(T, ws);
  k_batch_count<<<(unsigned)std::min<long long>(grid, T.n_tiles), 256, 0, st>>>(T, isos, W.counts, mc);
  return cudaGetLastError();
}

cudaError_t launch_batch_scan(const BatchTable& T, void* ws, long long* off, cudaStream_t st) {
  const BatchWs W = batch_ws(T, ws);
  if (T.n_tiles > 0) {
    k_batch_scan<<<(unsigned)T.n_q, kScanThreads, 0, st>>>(T, W.counts, W.rel, W.totals);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else {
    const cudaError_t e = cudaMemsetAsync(W.totals, 0, sizeof(long long) * (kMaxIso + 1), st);
    if (e != cudaSuccess) return e;
  }
  k_batch_bases<<<1, 32, 0, st>>>(T.n_q, W.totals, off);
  return cudaGetLastError();
}

cudaError_t launch_batch_emit(const BatchTable& T, const float* isos, const void* ws, const long long* off,
                              float* tris, long long cap, const McConst& mc, int grid, cudaStream_t st) {
  if (T.n_tiles <= 0) return cudaSuccess;
  const BatchWs W = batch_ws(T, const_cast<void*>(ws));
  k_batch_emit<<<(unsigned)std::min<long long>(grid, T.n_tiles), 256, 0, st>>>(T, isos, W.rel, off, tris, cap, mc);
  return cudaGetLastError();
}

cudaError_t launch_get_duals(const uint4* duals, long long nd, const unsigned long long* rec, int* out,
                             int grid, cudaStream_t st) {
  if (nd <= 0) return cudaSuccess;
  k_get_duals<<<grid, 256, 0, st>>>(duals, nd, rec, out);
  return cudaGetLastError();
}

}  // namespace amriso
