// kdt_internal.cuh -- device-side types and helpers of the CUDA k-d tree build.
//
// The build follows the level structure of the canonical k-d tree (paper,
// Sec. 1 and Sec. 2): level l splits each of its cells along one key
// coordinate, children of heap node h are 2h+1 and 2h+2. Each cell's split is
// combined from per-subset medians (the subsets of Sec. 3.2 / App. C.2); the
// per-subset statistic is the lower median and the combination is the
// count-weighted lower median of those medians.
//
// Layout invariant of the multi-CTA pipeline: inside every cell the points are
// ordered by subset, so each (cell, subset) segment is one contiguous range.
// The root is reordered once by subset (a counting pass; closed form for
// subsets by index mod r; nothing to do for contiguous subsets), and the
// stable two-way partition of every level keeps the order. The medians, the
// splits and the cell sizes do not depend on the order of points inside a
// cell; the one output that does, the order of the permutation inside each
// leaf, is ascending original index in the sequential definition (stable
// partitions of the identity), and a final per-leaf sort restores it.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kdt {

// ----------------------------------------------------------------- limits

constexpr int kMaxDims = 64;          // d <= 64
constexpr int kMaxSubsets = 4096;     // r <= 4096 on the CUDA path
constexpr int kMaxLevels = 30;        // depth / max_levels <= 30
constexpr int kTile = 2048;           // points per tile of the multi-CTA pipeline
constexpr int kTileThreads = 256;     // threads of the tile kernels
constexpr int kSelTinyMax = 64;       // segments up to this size: one thread per segment
constexpr int kSelSmallMax = 4096;    // largest warp-select segment (kdt_tuning warp_max)
constexpr int kSelWarpMin = 1024;     // smallest warp_max: sizes the list of CTA-select segments
constexpr int kSubtreeThreads = 256;  // threads of a CTA of the in-shared-memory subtree kernel
constexpr int kSubtreeWarps = kSubtreeThreads / 32;

// status codes (mirror include/kdt.h)
enum : int32_t {
  ST_OK = 0,
  ST_INVALID_ARG = 1,
  ST_NAN_INPUT = 2,
  ST_OOM = 3,
  ST_CUDA = 4,
  ST_CAPACITY = 5,
  ST_TIMEOUT = 6,
  ST_LEVEL_CAP = 7,
  ST_INTERNAL = 9,  // an internal table was inconsistent (reported as a CUDA error)
};

enum : int32_t { KEY_CYCLIC = 0, KEY_WIDEST = 1 };
enum : int32_t { SUB_MOD = 0, SUB_CONTIG = 1, SUB_EXPLICIT = 2 };

// --------------------------------------------------------- data structures

// Everything a kernel needs to know about one tree. Level l reads its points
// from src(l) and the multi-CTA partition writes them to dst(l):
//   src(0) = the root reordered by subset in buf[1] (presorted trees), else
//            the caller's input (perm = identity);
//   src(l>0) = buf[(l-1)&1], dst(l) = buf[l&1].
struct TreeDev {
  int64_t n;
  int32_t d, r, subset_mode, key_rule;
  int32_t depth;       // > 0 depth mode
  int32_t leaf_size;   // leaf mode
  int32_t max_levels;  // leaf mode level cap
  int32_t stall_limit; // d (cyclic) or 1 (widest)
  int32_t sid_bytes;   // explicit mode: 1 or 2
  int32_t small_max;   // cells up to this size finish in the subtree kernel
  int32_t presorted;   // root reordered by subset into buf[1]; leaves sorted at the end
  const float* x_in;
  const void* sid_in;
  float* xbuf[2];
  uint32_t* pbuf[2];
  void* sbuf[2];
  uint32_t* root_off;    // [r+1] subset offsets of the root (level 0)
  uint32_t* root_cur;    // [r] subset counts, then fill cursors of the presort
  uint32_t* huge;        // [huge_cap] terminal records too large for one CTA's leaf sort
  uint32_t* huge_count;  // device word
  uint32_t huge_cap;
  int32_t fourier_j;     // > 0: splits by the Fourier-moment estimator with this many harmonics
  int32_t combine_rule;  // 0: count-weighted median of the subset medians; 1: every subset counts once
  int32_t sub_wide;      // small cells run in the subtree kernel's wide shape (else the narrow one)
  uint32_t* out_perm;
  float* out_vals;
  int8_t* out_dims;
  int64_t* out_offs;
  struct TermRec* terms; // terminal cells
  uint32_t term_cap;
  uint32_t pad1;
  uint32_t* term_count;
  int32_t* status;
  int32_t* levels;       // L (max terminal level in leaf mode)
  int32_t* live;         // cells of this tree still waiting to be split (0: the tree is done)
};

// A cell of the tree: a contiguous position range [begin, begin+count) of its
// tree's current order.
struct Cell {
  uint32_t begin;
  uint32_t count;
  uint32_t heap;
  int32_t tree;
  int8_t level;
  int8_t stall;   // consecutive splits on this path that left the right child empty
  int16_t dim;    // widest-spread key coordinate if already known, else -1
};

// A terminal cell (leaf of the real tree); finalize turns these into offsets
// and sentinels below them.
struct TermRec {
  uint32_t begin;
  uint32_t count;
  uint32_t heap;
  int32_t level;
};

// Per-step arrays of the multi-CTA pipeline (one entry per big cell / tile /
// (cell, subset) segment).
struct StepDev {
  const Cell* cells;      // big cells of this step
  uint32_t ncells;              // cells of this step (steps driven by the host)
  const uint32_t* ncells_dev;   // if set: the device word that holds it (steps inside a graph)
  uint32_t pad;
  uint32_t* tile_base;    // [ncells+1] first tile of each cell (exclusive scan)
  uint32_t* seg_base;     // [ncells+1] first segment of each cell
  uint2* tiles;           // [ntiles] (cell, offset within cell)
  uint32_t* ntiles_total; // device word
  uint32_t* kdim;         // [ncells] key coordinate
  uint32_t* mkey;         // [ncells] split key
  uint32_t* lcount;       // [ncells] left child size
  uint32_t* tile_mm;      // [ntiles][2][kMaxDims][2] per-tile min/max keys of a root (widest; side 0)
  uint32_t* child_mm;     // [ncells][2][kMaxDims][2] per-child min/max keys (widest), reduced
                          // by the scatter with atomics
  uint32_t* seg_w;        // [nseg] points per (cell, subset)
  const uint32_t** seg_key; // [nseg] first key of the segment (raw float bits, key column)
  uint32_t* seg_med;      // [nseg] lower median key
  uint32_t* bigseg;       // [bigseg_cap] segments larger than kSelSmallMax
  uint32_t* bigseg_count; // device word
  uint32_t* midseg;       // [midseg_cap] segments of kSelTinyMax+1 .. kSelSmallMax points
  uint32_t* midseg_count; // device word
  uint32_t* tile_left;    // [ntiles]
  uint32_t* tile_loff;    // [ntiles]
  Cell* next_big;         // children that stay in the multi-CTA pipeline
  uint32_t* next_big_count;
  Cell* small;            // children that finish in the subtree kernel: cells of narrow-shape
                          // trees from the front, of wide-shape trees from the back
  uint32_t* small_count;  // cells at the front
  uint32_t* small_count_w;  // cells at the back (small[small_cap - 1 - j])
  uint32_t* small_total;    // both (appends past small_cap fail)
  uint32_t next_big_cap;
  uint32_t small_cap;
  uint32_t* next_big_points;  // points in next_big (for bandwidth accounting)
  uint32_t* small_points;     // points appended to small
  // subset offsets (relative to the cell's begin, r+1 per cell) of this
  // step's cells: rows of off_cur at obase_cur[c]; level-0 cells use their
  // tree's root_off. The scatter fills the rows of the big children.
  const uint32_t* off_cur;
  const uint32_t* obase_cur;  // [ncells]
  uint32_t* off_next;
  uint32_t* obase_next;       // [next_big_cap]
  uint32_t* off_used;         // device word: words of off_next handed out
  uint32_t off_cap;
  uint32_t bigseg_cap;
  // select paths by segment size (kdt_tuning): one thread up to tiny_max keys,
  // a warp's bitonic network up to bitonic_max, a warp's radix select up to
  // warp_max, a CTA above
  uint32_t tiny_max, bitonic_max, warp_max;
  uint32_t midseg_cap;
  uint32_t pad4;
  uint2* crow;                // [ncells][2] (slot, row of off_next) of each big child; (kNoRow, slot in
                              // small) of a child queued for the subtree kernel; else (kNoRow, kNoRow)
  // Sharded build (0 shards: off). The forest's trees 0..shards-1 are the
  // shards of one tree, each owning the subsets s with s % shards == its
  // slot, all at the same level in every step.
  uint32_t shards;
  uint32_t shard_span;        // 2^(levels - 1): entries per shard of shard_idx
  uint32_t* shard_idx;        // [shards][shard_span] step cell of (shard, heap - (2^level - 1)), or kNoRow
  uint32_t* wcount;           // [ncells] points of the cell over all shards (the combine's weight)
  uint32_t* mm_tmp;           // [ncells][2][d][2] children's min / max over all shards
};

constexpr uint32_t kNoRow = 0xffffffffu;

// ------------------------------------------------------------- key transform

// Order-preserving map float -> uint32: unsigned comparison of keys equals
// the float order, with -0.0 below +0.0.
__device__ __forceinline__ uint32_t ord_key(float x) {
  uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_float(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k ^ 0x80000000u) : ~k;
  return __uint_as_float(u);
}

__device__ __forceinline__ bool is_nan_bits(float x) {
  return (__float_as_uint(x) & 0x7fffffffu) > 0x7f800000u;
}

// -------------------------------------------------------------- tree views

__device__ __forceinline__ const float* src_cols(const TreeDev& t, int level) {
  return (level == 0 && !t.presorted) ? t.x_in : t.xbuf[(level - 1) & 1];
}
__device__ __forceinline__ const uint32_t* src_perm(const TreeDev& t, int level) {
  return (level == 0 && !t.presorted) ? nullptr : t.pbuf[(level - 1) & 1];
}
__device__ __forceinline__ const void* src_sid(const TreeDev& t, int level) {
  return (level == 0 && !t.presorted) ? t.sid_in : t.sbuf[(level - 1) & 1];
}

__device__ __forceinline__ void set_status(const TreeDev& t, int32_t code) {
  atomicCAS(t.status, ST_OK, code);
}

// Subset of the point at position pos whose original index is orig. An
// explicit id >= r is reported as an invalid argument and replaced by 0 so
// that no table is indexed out of range.
__device__ __forceinline__ uint32_t subset_of(const TreeDev& t, const void* sidcol, uint32_t orig,
                                              int64_t pos) {
  if (t.subset_mode == SUB_MOD) return orig % (uint32_t)t.r;
  if (t.subset_mode == SUB_CONTIG)
    return (uint32_t)(((uint64_t)orig * (uint64_t)t.r) / (uint64_t)t.n);
  const uint32_t s = t.sid_bytes == 1 ? (uint32_t)((const uint8_t*)sidcol)[pos]
                                      : (uint32_t)((const uint16_t*)sidcol)[pos];
  if (s >= (uint32_t)t.r) {
    set_status(t, ST_INVALID_ARG);
    return 0;
  }
  return s;
}

// Subset of a point from its original index (modes that define it so).
__device__ __forceinline__ uint32_t subset_from_orig(const TreeDev& t, uint32_t orig) {
  if (t.subset_mode == SUB_MOD) return orig % (uint32_t)t.r;
  return (uint32_t)(((uint64_t)orig * (uint64_t)t.r) / (uint64_t)t.n);
}

// Subset of the point at position pos of the order level `level` reads
// (explicit ids there are already checked and below r).
__device__ __forceinline__ uint32_t subset_at(const TreeDev& t, int level, int64_t pos) {
  if (t.subset_mode == SUB_EXPLICIT) {
    const void* S = src_sid(t, level);
    const uint32_t v = t.sid_bytes == 1 ? (uint32_t)((const uint8_t*)S)[pos] : (uint32_t)((const uint16_t*)S)[pos];
    return min(v, (uint32_t)t.r - 1u);
  }
  const uint32_t* P = src_perm(t, level);
  return subset_from_orig(t, P ? P[pos] : (uint32_t)pos);
}

// Terminal test for a cell about to be processed at `level` (reading R8 in
// leaf mode; empty cells and the last level in depth mode).
// Cells of a step: the host's count, or the device word a graph-driven step
// reads (clamped to the capacity of the cell lists).
__device__ __forceinline__ uint32_t ncells_of(const StepDev& s) {
  return s.ncells_dev ? min(*s.ncells_dev, s.next_big_cap) : s.ncells;
}

// Points of step cell c whose split is being combined: its own count, or in a
// sharded build the cell's count over all shards.
__device__ __forceinline__ uint32_t cell_weight(const StepDev& s, uint32_t c, const Cell& cell) {
  return s.shards ? s.wcount[c] : cell.count;
}

__device__ __forceinline__ bool is_terminal(const TreeDev& t, uint32_t count, int level, int stall) {
  if (t.depth > 0) return count == 0 || level >= t.depth;
  return count <= (uint32_t)t.leaf_size || stall >= t.stall_limit;
}

__device__ __forceinline__ void record_terminal(const TreeDev& t, uint32_t begin, uint32_t count,
                                                uint32_t heap, int level) {
  uint32_t slot = atomicAdd(t.term_count, 1u);
  if (slot < t.term_cap) {
    t.terms[slot] = TermRec{begin, count, heap, level};
  } else {
    set_status(t, ST_CAPACITY);
  }
  atomicMax(t.levels, level);
}

// ------------------------------------------------------------ warp helpers

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ uint32_t warp_min(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ uint32_t warp_max(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Given a 256-bin histogram in shared memory (counts or weights) and a
// 0-based target rank, the whole warp finds the digit whose bin holds that
// rank; returns the digit and, in *below, the total of the lower bins.
__device__ __forceinline__ uint32_t warp_find_digit(const uint32_t* hist, uint32_t rank,
                                                    uint32_t* below) {
  const int lane = threadIdx.x & 31;
  uint32_t local[8];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    local[i] = hist[lane * 8 + i];
    s += local[i];
  }
  uint32_t incl = warp_incl_scan(s);
  uint32_t excl = incl - s;
  // the lane whose range [excl, incl) contains rank
  unsigned ballot = __ballot_sync(0xffffffffu, rank >= excl && rank < incl);
  int owner = ballot ? __ffs(ballot) - 1 : 31;
  uint32_t digit = 0, b = 0;
  if (lane == owner) {
    uint32_t acc = excl;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (rank < acc + local[i]) {
        digit = lane * 8 + i;
        b = acc;
        break;
      }
      acc += local[i];
    }
  }
  digit = __shfl_sync(0xffffffffu, digit, owner);
  *below = __shfl_sync(0xffffffffu, b, owner);
  return digit;
}

// Like warp_find_digit for a histogram of nb = 2^bits bins (1 <= bits <= 8).
__device__ __forceinline__ uint32_t warp_find_digit_n(const uint32_t* hist, uint32_t nb, uint32_t rank,
                                                      uint32_t* below) {
  const int lane = threadIdx.x & 31;
  const uint32_t per = nb >= 32u ? nb / 32u : 1u;
  const uint32_t first = lane * per;
  uint32_t local[8];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    local[i] = ((uint32_t)i < per && first + i < nb) ? hist[first + i] : 0u;
    s += local[i];
  }
  const uint32_t incl = warp_incl_scan(s);
  const uint32_t excl = incl - s;
  const unsigned ballot = __ballot_sync(0xffffffffu, rank >= excl && rank < incl);
  const int owner = ballot ? __ffs(ballot) - 1 : 31;
  uint32_t digit = 0, b = 0;
  if (lane == owner) {
    uint32_t acc = excl;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if ((uint32_t)i < per && rank < acc + local[i]) {
        digit = first + i;
        b = acc;
        break;
      }
      acc += local[i];
    }
  }
  digit = __shfl_sync(0xffffffffu, digit, owner);
  *below = __shfl_sync(0xffffffffu, b, owner);
  return digit;
}

// Exact key of 0-based weighted rank `rank` among cnt items (key_of(j),
// w_of(j)), j < cnt, one warp: the smallest key m whose items with key <= m
// weigh more than `rank`. MSD radix select over the bits where the keys
// differ (the common prefix of their min and max is known from the start, so
// no pass is spent on bits every key shares), 8-bit digits, histogram `hist`
// of 256 words owned by the warp.
template <bool kUnit = false, class KeyOf, class WOf, class ValidOf>
__device__ uint32_t warp_weighted_select(uint32_t cnt, uint32_t rank, uint32_t* hist, KeyOf key_of, WOf w_of,
                                         ValidOf valid_of) {
  const int lane = threadIdx.x & 31;
  uint32_t lo = 0xffffffffu, hi = 0u;
  for (uint32_t j = lane; j < cnt; j += 32)
    if (valid_of(j)) {
      const uint32_t k = key_of(j);
      lo = min(lo, k);
      hi = max(hi, k);
    }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if (lo >= hi) return lo;
  int rem = 32 - __clz(lo ^ hi);  // low bits still unknown
  uint32_t prefix = rem == 32 ? 0u : (lo & ~((1u << rem) - 1u));
  while (rem > 0) {
    const int bits = rem < 8 ? rem : 8;
    const int shift = rem - bits;
    const uint32_t nb = 1u << bits;
    const uint32_t hmask = rem == 32 ? 0u : ~((1u << rem) - 1u);
    for (uint32_t i = lane; i < nb; i += 32) hist[i] = 0;
    __syncwarp();
    for (uint32_t j = lane; j < cnt; j += 32) {
      if (!valid_of(j)) continue;
      const uint32_t k = key_of(j);
      if ((k & hmask) == prefix) atomicAdd(&hist[(k >> shift) & (nb - 1u)], kUnit ? 1u : w_of(j));
    }
    __syncwarp();
    uint32_t below;
    const uint32_t digit = warp_find_digit_n(hist, nb, rank, &below);
    rank -= below;
    prefix |= digit << shift;
    rem = shift;
    __syncwarp();
  }
  return prefix;
}

template <bool kUnit = false, class KeyOf, class WOf>
__device__ uint32_t warp_weighted_select(uint32_t cnt, uint32_t rank, uint32_t* hist, KeyOf key_of, WOf w_of) {
  return warp_weighted_select<kUnit>(cnt, rank, hist, key_of, w_of, [](uint32_t) { return true; });
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total. `tmp` holds 33 words.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* tmp, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  uint32_t incl = warp_incl_scan(v);
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nwarps ? tmp[lane] : 0u;
    uint32_t wi = warp_incl_scan(w);
    if (lane < nwarps) tmp[lane] = wi - w;
    if (lane == nwarps - 1) tmp[32] = wi;
  }
  __syncthreads();
  uint32_t r = tmp[warp] + incl - v;
  *total = tmp[32];
  __syncthreads();
  return r;
}

}  // namespace kdt
