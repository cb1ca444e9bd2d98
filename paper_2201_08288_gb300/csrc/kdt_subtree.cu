// kdt_subtree.cu -- finish every remaining level of a small cell inside one
// CTA, and turn the terminal cells into the output offsets.
//
// A cell with at most subtree_capacity(d) points is staged once into shared
// memory with bulk asynchronous copies (cp.async.bulk, completion on an
// mbarrier): all d coordinate columns. Its points are in
// subset order (the layout invariant of kdt_internal.cuh; the root of a small
// tree is put in that order here by a counting sort), and the local order is
// kept by stable partitions, so every (cell, subset) segment is a contiguous
// run of positions. Then, level by level (paper, Sec. 2: each level splits
// every cell of the previous one along its key), for all live local cells at
// once:
//   1. key coordinate (cyclic, or widest range);
//   2. the key of every position on its cell's coordinate, and the segment
//      starts (a cell's first position, or a change of subset), numbered by
//      one block-wide scan;
//   3. the lower median of every segment: rank counting inside the segment
//      (at most kRankMax points), else a warp radix select over the bits
//      where its keys differ;
//   4. per cell, the count-weighted lower median of its segments' medians;
//   5. a stable partition of the local order around the split (ties left);
//   6. children: terminal cells are recorded, the others form the next level.
// The permutation is written once, at the end, gathered from the cell's
// incoming permutation in global memory. The kernel is persistent: each CTA
// pulls cells from a queue. It is compiled for the two shapes of
// kdt_launch.h (positions per thread, CTAs per SM, cell-table size).
#include <algorithm>
#include <type_traits>

#include "kdt_internal.cuh"
#include "kdt_launch.h"
#include "kdt_ptx.cuh"
#include "kdt_trace.h"

namespace kdt {

namespace {

constexpr int T = kSubtreeThreads;
constexpr int NW = kSubtreeWarps;
constexpr uint16_t kNoCell = 0xffff;
constexpr uint32_t kRankMax = 32;

// -------------------------------------------------------- shared layout

struct Smem {
  uint32_t* whist;    // NW * 256 words: warp histograms, tables of few cells, root subset counts
  uint16_t* biglist;  // kSubtreeBigCap segments above kRankMax points
  LCell* tab;         // 2 * cells: the cell tables of two levels
  uint32_t* cols;     // d key columns at stride `stride`
  uint32_t* gk;       // N: key of each position on its cell's coordinate
  uint32_t* smed;     // N: median of each segment
  uint16_t* sid;      // N: subset of each local point
  uint16_t* ordA;     // N: local point at each position
  uint16_t* ordB;     // N
  uint16_t* cellid;   // N: live cell of each position (kNoCell: finished)
  uint16_t* pre;      // N + 1: exclusive prefix of the segment starts, then of the left flags
  uint16_t* segs;     // N + 1: first position of each segment
};

__device__ __forceinline__ uint32_t al16(uint32_t off) { return (off + 15u) & ~15u; }

// Carve the dynamic shared memory with plain byte offsets from its base (no
// pointer is stored through another pointer), so that the compiler keeps
// every array in the shared address space.
__device__ __forceinline__ Smem carve(uint8_t* base, uint32_t N, int d, int cells) {
  Smem s;
  uint32_t off = 0;
  s.whist = (uint32_t*)(base + off);
  off += (uint32_t)NW * 256u * 4u;
  s.biglist = (uint16_t*)(base + off);
  off += (uint32_t)kSubtreeBigCap * 2u;
  s.tab = (LCell*)(base + off);
  off += 2u * (uint32_t)cells * (uint32_t)sizeof(LCell);
  s.cols = (uint32_t*)(base + off);
  off += (uint32_t)d * subtree_stride(N) * 4u;
  s.gk = (uint32_t*)(base + off);
  off = al16(off + N * 4u);
  s.smed = (uint32_t*)(base + off);
  off = al16(off + N * 4u);
  const uint32_t a = (N + 1u) * 2u;
  s.sid = (uint16_t*)(base + off);
  off = al16(off + a);
  s.ordA = (uint16_t*)(base + off);
  off = al16(off + a);
  s.ordB = (uint16_t*)(base + off);
  off = al16(off + a);
  s.cellid = (uint16_t*)(base + off);
  off = al16(off + a);
  s.pre = (uint16_t*)(base + off);
  off = al16(off + a);
  s.segs = (uint16_t*)(base + off);
  return s;
}

__device__ __forceinline__ double key_range(uint32_t lo, uint32_t hi) {
  return (lo == hi) ? 0.0 : (double)key_float(hi) - (double)key_float(lo);
}

// Widest coordinate of one cell from its per-coordinate min and max keys
// (coordinate l in lane l % 32, slot l / 32): the largest range
// (double)max - (double)min, 0 for equal keys, lowest coordinate on ties.
// A range is never negative, so the bit patterns of two ranges order like the
// ranges as unsigned integers: the argmax is taken on the high word, then the
// low word, then the lowest coordinate, with integer warp reductions (the only
// double arithmetic is the one subtraction per range).
__device__ __forceinline__ int warp_pick_widest(const uint32_t (&lo)[2], const uint32_t (&hi)[2], int d) {
  const int lane = threadIdx.x & 31;
  uint64_t rb = lane < d ? (uint64_t)__double_as_longlong(key_range(lo[0], hi[0])) : 0ull;
  uint32_t ib = lane < d ? (uint32_t)lane : 0xffffffffu;
  if (lane + 32 < d) {
    const uint64_t r1 = (uint64_t)__double_as_longlong(key_range(lo[1], hi[1]));
    if (r1 > rb) {
      rb = r1;
      ib = (uint32_t)lane + 32u;
    }
  }
  const uint32_t rh = (uint32_t)(rb >> 32), rl = (uint32_t)rb;
  const uint32_t mh = __reduce_max_sync(0xffffffffu, rh);
  const uint32_t ml = __reduce_max_sync(0xffffffffu, rh == mh ? rl : 0u);
  return (int)__reduce_min_sync(0xffffffffu, (rh == mh && rl == ml) ? ib : 0xffffffffu);
}

// Exclusive prefix, over all positions, of the flags whose warp ballots are
// bal[q] (position tid + q T, block q NW + warp), given the popcount of every
// block in cnt[kQ NW] (block order = position order; at most 64 blocks);
// *total is the sum.
template <int kQ>
__device__ __forceinline__ void block_counts_scan(const unsigned (&bal)[kQ], const uint32_t* cnt, int lane,
                                                  int warp, uint32_t (&excl)[kQ], uint32_t* total) {
  static_assert(kQ * NW <= 64, "two block counts per lane at most");
  const uint32_t c0 = lane < kQ * NW ? cnt[lane] : 0u, c1 = lane + 32 < kQ * NW ? cnt[lane + 32] : 0u;
  const uint32_t i0 = warp_incl_scan(c0);
  const uint32_t i1 = warp_incl_scan(c1) + __shfl_sync(0xffffffffu, i0, 31);
  *total = __shfl_sync(0xffffffffu, i1, 31);
  const uint32_t e0 = i0 - c0, e1 = i1 - c1;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int src = (q * NW + warp) & 31;
    const uint32_t v0 = __shfl_sync(0xffffffffu, e0, src), v1 = __shfl_sync(0xffffffffu, e1, src);
    excl[q] = (q * NW < 32 ? v0 : v1) + (uint32_t)__popc(bal[q] & lt);
  }
}

// Block-wide exclusive scan of one value per thread with one barrier; wtot
// (NW words) must not be reused before the next barrier.
__device__ __forceinline__ uint32_t block_excl_scan_1bar(uint32_t v, uint32_t* wtot, int lane, int warp,
                                                         uint32_t* total) {
  const uint32_t incl = warp_incl_scan(v);
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t x = wtot[w];
    all += x;
    before += w < warp ? x : 0u;
  }
  *total = all;
  return before + incl - v;
}

// Weighted select by one warp with the items in registers (K per lane, cnt <=
// 32 K, total weight below 2^20): the smallest key m whose items with key <= m
// weigh more than `rank`. Starting below the bits where every key agrees, each
// step sums, over the remaining candidates whose next bit is 0, their weight
// and their number (one warp sum of (w << 12) | 1) and fixes that bit. The
// answer is the key of a remaining candidate, so once a single candidate is
// left its key is the answer and the lower bits need no steps.
template <int K, class KeyOf, class WOf>
__device__ __forceinline__ uint32_t warp_wsel_bits(uint32_t cnt, uint32_t rank, KeyOf key_of, WOf w_of) {
  const int lane = threadIdx.x & 31;
  uint32_t key[K], pw[K];
  uint32_t lo = 0xffffffffu, hi = 0u;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const uint32_t j = (uint32_t)lane + 32u * q;
    const bool ok = j < cnt;
    key[q] = ok ? key_of(j) : 0u;
    pw[q] = ok ? (w_of(j) << 12) | 1u : 0u;
    if (ok) {
      lo = min(lo, key[q]);
      hi = max(hi, key[q]);
    }
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if (lo >= hi) return lo;
  int bit = 31 - __clz(lo ^ hi);                    // highest bit where the keys differ
  uint32_t prefix = lo & ~((2u << bit) - 1u);       // the bits above it (none when bit = 31)
  uint32_t ncand = cnt;                             // items matching the fixed bits
  for (; bit >= 0; --bit) {
    const uint32_t fixed = ~((1u << bit) - 1u);     // bits above `bit`, and `bit` itself
    uint32_t acc = 0;
#pragma unroll
    for (int q = 0; q < K; ++q) acc += ((key[q] ^ prefix) & fixed) == 0u ? pw[q] : 0u;
    acc = __reduce_add_sync(0xffffffffu, acc);
    const uint32_t w0 = acc >> 12, n0 = acc & 0xfffu;
    if (rank >= w0) {
      rank -= w0;
      prefix |= 1u << bit;
      ncand -= n0;
    } else {
      ncand = n0;
    }
    if (ncand == 1u) {  // the one item whose key matches the fixed bits
      uint32_t m = 0;
#pragma unroll
      for (int q = 0; q < K; ++q)
        if (pw[q] != 0u && ((key[q] ^ prefix) & fixed) == 0u) m = key[q];
      return __reduce_max_sync(0xffffffffu, m);
    }
  }
  return prefix;
}

// kWide: compiled for the wide shape, else the narrow one (kdt_launch.h).
template <bool kWide>
__global__ void __launch_bounds__(T, (kWide ? kSubWide : kSubNarrow).ctas)
k_subtree(const TreeDev* trees, const Cell* list, uint32_t count, const uint32_t* count_dev, uint32_t reversed,
          uint32_t* head, LCell* slices, uint32_t slice_cells, uint32_t probe_tries) {
  constexpr SubtreeShape kSh = kWide ? kSubWide : kSubNarrow;
  constexpr int kQ = kSh.q, kCells = kSh.cells;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  const uint32_t count_cap = count;
  if (count_dev) count = min(*count_dev, count);  // a graph-driven step: the queue's length, capped
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t s_item, s_ncur, s_nbig, s_where, s_fail;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_colbase[kMaxDims];
  __shared__ uint32_t s_bcnt[kQ * NW];  // per-block counts of a level's position flags
  __shared__ uint32_t s_wtot[NW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // this CTA's two global cell tables (for levels with too many cells for
  // shared memory); tables are picked by offset, never by an indexed array,
  // so that no pointer array of this kernel lives in local memory
  LCell* const gslice = slices + (size_t)blockIdx.x * 2 * slice_cells;
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    mbar_init_fence();
    s_fail = 0;
  }
  uint32_t phase = 0;

  for (;;) {
    fence_proxy_async_smem();  // earlier generic writes before the next bulk copies
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(head, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= count) break;
    const Cell c = list[reversed ? count_cap - 1u - item : item];
    const TreeDev& t = trees[c.tree];
    if (probe_tries && tid == 0) {
      // injected fault (kdt_fault_inject): wait on a phase that nothing
      // completes, with no copy in flight, until the bound gives up; each CTA
      // probes once
      const uint32_t tries = probe_tries;
      probe_tries = 0;
      if (!mbar_wait_bounded_n(&s_bar, phase, tries)) {
        set_status(t, ST_TIMEOUT);
        s_fail = 1;
      }
    }
    __syncthreads();
    if (s_fail) {
      // a bounded wait of this CTA gave up: the cells it still pulls fail
      // without being touched, so that every tree's count of cells left
      // reaches zero and its caller gets the status
      if (tid == 0) {
        set_status(t, ST_TIMEOUT);
        atomicSub(t.live, 1);
      }
      continue;
    }
    const uint32_t N = c.count;
    const int d = t.d, r = t.r;
    const int64_t n = t.n;
    if (N > (uint32_t)(kQ * T) || subtree_fixed_bytes(kCells) + subtree_point_bytes(N, d) > kSh.smem) {
      // a queue holds only cells within its shape's capacity
      if (tid == 0) {
        set_status(t, ST_INTERNAL);
        atomicSub(t.live, 1);
      }
      continue;
    }
    const uint32_t stride = subtree_stride(N);
    Smem S = carve(smem_raw, N, d, kCells);
    // Column l of the cell sits at S.cols + s_colbase[l]. Each column's
    // offset absorbs the 16-byte alignment phase of its global source so that
    // the bulk copies are aligned on both sides.
    const uint32_t* P = src_perm(t, c.level);  // incoming permutation (null: the identity)

    // ---- 0. stage the cell: bulk copies of the aligned middle, plain loads at the edges
    {
      const float* X = src_cols(t, c.level);
      const uint32_t b0 = c.begin, e0 = c.begin + N;
      const int ncols = d;
      auto src_of = [&](int l) -> const uint32_t* { return (const uint32_t*)(X + (int64_t)l * n); };
      // phase of element b0 of column l: elements past the previous 16-byte boundary
      auto phase_of = [&](int l) -> uint32_t {
        return (uint32_t)(((uintptr_t)(src_of(l) + b0) >> 2) & 3u);
      };
      if (tid < d) s_colbase[tid] = (uint32_t)tid * stride + phase_of(tid);
      if (tid == 0) {
        uint32_t total = 0;
        for (int l = 0; l < ncols; ++l) {
          const uint32_t ph = phase_of(l);
          const uint32_t a0 = min(b0 + ((4u - ph) & 3u), e0);
          const uint32_t a1 = a0 + ((e0 - a0) & ~3u);
          total += (a1 - a0) * 4u;
        }
        mbar_arrive_expect_tx(&s_bar, total);
        for (int l = 0; l < ncols; ++l) {
          const uint32_t ph = phase_of(l);
          const uint32_t a0 = min(b0 + ((4u - ph) & 3u), e0);
          const uint32_t a1 = a0 + ((e0 - a0) & ~3u);
          if (a1 > a0)
            bulk_g2s(S.cols + (size_t)l * stride + ph + (a0 - b0), src_of(l) + a0, (a1 - a0) * 4u, &s_bar);
        }
        if (P) {
          // the incoming permutation is gathered at the end: bring the cell's
          // range into L2 now (whole 16-byte blocks; buffers are 256-byte
          // aligned and padded to a multiple of 256 bytes)
          const uintptr_t p0 = (uintptr_t)(P + b0) & ~(uintptr_t)15, p1 = ((uintptr_t)(P + e0) + 15) & ~(uintptr_t)15;
          bulk_prefetch_l2((const void*)p0, (uint32_t)(p1 - p0));
        }
      }
      for (int j = tid; j < ncols * 8; j += T) {
        const int l = j >> 3, e = j & 7;
        const uint32_t ph = phase_of(l);
        const uint32_t a0 = min(b0 + ((4u - ph) & 3u), e0);
        const uint32_t a1 = a0 + ((e0 - a0) & ~3u);
        const uint32_t idx = e < 4 ? b0 + e : a1 + (e - 4);
        const bool ok = e < 4 ? (idx < a0) : (idx < e0);
        if (ok) S.cols[(size_t)l * stride + ph + (idx - b0)] = src_of(l)[idx];
      }
      __syncthreads();
      // explicit subset ids are read from global memory while the bulk copies
      // run (neither touches the other's shared memory), eight loads in
      // flight per thread
      const void* SID = src_sid(t, c.level);
      const bool expl = t.subset_mode == SUB_EXPLICIT;
      for (uint32_t i0 = tid; i0 < N; i0 += 8 * T) {
        uint32_t v[8];
        if (expl) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const uint32_t i = i0 + (uint32_t)q * T;
            v[q] = i >= N ? 0u
                          : (t.sid_bytes == 1 ? (uint32_t)((const uint8_t*)SID)[(int64_t)b0 + i]
                                              : (uint32_t)((const uint16_t*)SID)[(int64_t)b0 + i]);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint32_t i = i0 + (uint32_t)q * T;
          if (i >= N) break;
          if (expl) {
            if (v[q] >= (uint32_t)r) {  // an id outside [0, r): reported, replaced by 0
              set_status(t, ST_INVALID_ARG);
              v[q] = 0;
            }
            S.sid[i] = (uint16_t)v[q];
          }
          S.cellid[i] = 0;
        }
      }
      // one thread waits for the copies (a waiting thread keeps issuing
      // try_wait); the barrier after it parks the others without issue slots
      // and makes what the copies wrote visible to them
      if (tid == 0 && !mbar_wait_bounded(&s_bar, phase)) {
        set_status(t, ST_TIMEOUT);
        s_fail = 1;
      }
      phase ^= 1u;
      __syncthreads();
      if (s_fail) {  // copies in flight: wait once more (bounded), then fail this cell and drain
        if (tid == 0) {
          mbar_wait_bounded(&s_bar, phase ^ 1u);
          atomicSub(t.live, 1);
        }
        continue;
      }
      // keys in place; NaN is looked for in the roots of small trees only (the
      // multi-CTA pipeline checked every point of a larger tree at its root)
      bool nan = false;
      const bool check_nan = c.level == 0;
      for (int l = 0; l < d; ++l) {
        uint32_t* col = S.cols + s_colbase[l];
#pragma unroll 4
        for (uint32_t i = tid; i < N; i += T) {
          const float x = __uint_as_float(col[i]);
          nan |= check_nan && is_nan_bits(x);
          col[i] = ord_key(x);
        }
      }
      if (nan) set_status(t, ST_NAN_INPUT);
      if (!expl)
        for (uint32_t i = tid; i < N; i += T)
          S.sid[i] = (uint16_t)subset_of(t, SID, P ? P[b0 + i] : b0 + i, (int64_t)b0 + i);
      // The root of a small tree arrives in index order: put it in subset
      // order (counting sort; order inside a subset is immaterial). Every
      // other cell is in subset order already.
      const bool sort_root = c.level == 0 && t.subset_mode != SUB_CONTIG && r > 1;
      if (sort_root) {
        for (int j = tid; j < r; j += T) S.whist[j] = 0;
        __syncthreads();
        for (uint32_t i = tid; i < N; i += T) S.ordB[i] = (uint16_t)atomic_add_shared(&S.whist[S.sid[i]], 1u);
        __syncthreads();
        uint32_t run = 0;
        for (int j0 = 0; j0 < r; j0 += T) {
          const int j = j0 + tid;
          const uint32_t v = j < r ? S.whist[j] : 0u;
          uint32_t tot;
          const uint32_t ex = block_excl_scan(v, tmp, &tot);
          if (j < r) S.whist[j] = run + ex;
          run += tot;
        }
        __syncthreads();
        for (uint32_t i = tid; i < N; i += T) S.ordA[S.whist[S.sid[i]] + S.ordB[i]] = (uint16_t)i;
      } else {
        for (uint32_t i = tid; i < N; i += T) S.ordA[i] = (uint16_t)i;
      }
      if (tid == 0) {
        S.tab[0] = LCell{c.heap, 0u, 0, (uint16_t)N, 0, 0, (uint8_t)c.stall};
        s_ncur = 1;
        s_where = 0;
      }
    }
    __syncthreads();

    uint16_t* ordA = S.ordA;
    uint16_t* ordB = S.ordB;
    int which = 0;
    int level = c.level;
    int prev_global = 0;  // the previous level's cell table lives in the global slice
    for (;;) {
      const uint32_t ncur = s_ncur;
      if (ncur == 0) break;
      // The body of a level is compiled twice: for a cell table in shared
      // memory (the usual case, accessed with shared-memory loads) and for one
      // that outgrew it and lives in this CTA's global slice.
      auto level_body = [&](auto in_global) {
        LCell* cc = decltype(in_global)::value ? gslice + (size_t)which * slice_cells
                                               : S.tab + which * kCells;
        // the previous level's table: its cells' mkey holds the numbers of
        // their live children (kNoCell for a finished one), low half left
        const LCell* cprev = prev_global ? gslice + (size_t)(which ^ 1) * slice_cells : S.tab + (which ^ 1) * kCells;
        const bool first = level == (int)c.level;

        // ---- 1. key coordinate of every live cell
        if (t.key_rule == KEY_CYCLIC) {
          for (uint32_t k = tid; k < ncur; k += T) cc[k].dim = (uint8_t)(level % d);
        } else if (level == (int)c.level && c.dim >= 0) {
          if (tid == 0) cc[0].dim = (uint8_t)c.dim;  // picked from the parent's partition
        } else {
          // per (cell, part): min and max key of every coordinate, coordinate l
          // ending in lane l % 32; G warps share a cell when there are few cells
          const uint32_t G = ncur >= (uint32_t)NW ? 1u : (uint32_t)NW / ncur;
          uint32_t* tab = S.whist;  // few cells: [ncur][d][2]
          if (G > 1) {
            for (uint32_t j = tid; j < ncur * (uint32_t)d; j += T) {
              tab[2 * j] = 0xffffffffu;
              tab[2 * j + 1] = 0u;
            }
            __syncthreads();
          }
          for (uint32_t w0 = warp; w0 < ncur * G; w0 += NW) {
            const uint32_t k = w0 / G, part = w0 % G;
            const uint32_t b = cc[k].begin, cnt = cc[k].count;
            const uint32_t i0 = b + (cnt * part) / G, i1 = b + (cnt * (part + 1)) / G;
            uint32_t lo2[2] = {0xffffffffu, 0xffffffffu}, hi2[2] = {0u, 0u};
            for (int c0 = 0; c0 < d; c0 += 8) {
              const int nc = min(8, d - c0);
              uint32_t base[8], lo[8], hi[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                base[q] = q < nc ? s_colbase[c0 + q] : 0u;
                lo[q] = 0xffffffffu;
                hi[q] = 0u;
              }
              for (uint32_t i = i0 + lane; i < i1; i += 32) {
                const uint32_t o = ordA[i];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                  if (q < nc) {
                    const uint32_t kk = S.cols[base[q] + o];
                    lo[q] = min(lo[q], kk);
                    hi[q] = max(hi[q], kk);
                  }
              }
#pragma unroll
              for (int q = 0; q < 8; ++q)
                if (q < nc) {
                  const uint32_t l = __reduce_min_sync(0xffffffffu, lo[q]);
                  const uint32_t h = __reduce_max_sync(0xffffffffu, hi[q]);
                  const int col = c0 + q;
                  if (lane == (col & 31)) {
                    if (col < 32) {
                      lo2[0] = l;
                      hi2[0] = h;
                    } else {
                      lo2[1] = l;
                      hi2[1] = h;
                    }
                  }
                }
            }
            if (G == 1) {
              const int best = warp_pick_widest(lo2, hi2, d);
              if (lane == 0) cc[k].dim = (uint8_t)best;
            } else {
              for (int h2 = 0; h2 < 2; ++h2) {
                const int col = lane + 32 * h2;
                if (col < d) {
                  atomic_min_shared(&tab[(k * d + col) * 2], lo2[h2]);
                  atomic_max_shared(&tab[(k * d + col) * 2 + 1], hi2[h2]);
                }
              }
            }
          }
          if (G > 1) {
            __syncthreads();
            for (uint32_t k = warp; k < ncur; k += NW) {
              uint32_t lo2[2], hi2[2];
              for (int h2 = 0; h2 < 2; ++h2) {
                const int col = lane + 32 * h2;
                lo2[h2] = col < d ? tab[(k * d + col) * 2] : 0u;
                hi2[h2] = col < d ? tab[(k * d + col) * 2 + 1] : 0u;
              }
              const int best = warp_pick_widest(lo2, hi2, d);
              if (lane == 0) cc[k].dim = (uint8_t)best;
            }
          }
        }
        __syncthreads();

        // ---- 2. keys in local order, segment starts, their numbering.
        // Thread tid owns positions i = tid + q T (q < kQ); the 32 positions of
        // (q, warp) form block q NW + warp, and blocks are in position order,
        // so one scan over the kQ NW block counts of the start flags (warp
        // ballots) numbers every segment.
        uint32_t kq[kQ], keyq[kQ], segq[kQ];
        unsigned balq[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          const uint32_t i = (uint32_t)tid + (uint32_t)q * T;
          uint32_t k = kNoCell, key = 0u;
          bool f = false;
          if (i < N) {
            k = S.cellid[i];
            if (!first && k != kNoCell) {
              // the position's cell at this level: a child of its previous cell
              const LCell& pc = cprev[k];
              k = (pc.mkey >> ((i - pc.begin) >= pc.lcount ? 16u : 0u)) & 0xffffu;
              S.cellid[i] = (uint16_t)k;
            }
            if (k != kNoCell) {
              const uint32_t o = ordA[i];
              const uint32_t cb = cc[k].begin;
              key = S.cols[s_colbase[cc[k].dim] + o];
              f = (i == cb) || S.sid[o] != S.sid[ordA[i - 1]];
              S.gk[i] = key;
            }
          }
          kq[q] = k;
          keyq[q] = key;
          balq[q] = __ballot_sync(0xffffffffu, f);
          if (lane == 0) s_bcnt[q * NW + warp] = (uint32_t)__popc(balq[q]);
        }
        if (tid == 0) s_nbig = 0;
        __syncthreads();
        {
          uint32_t total;
          block_counts_scan(balq, s_bcnt, lane, warp, segq, &total);
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const uint32_t i = (uint32_t)tid + (uint32_t)q * T;
            const bool f = (balq[q] >> lane) & 1u;
            if (i < N) {
              S.pre[i] = (uint16_t)segq[q];  // starts before position i
              if (f) S.segs[segq[q]] = (uint16_t)i;
            }
            segq[q] = segq[q] + (f ? 1u : 0u) - 1u;  // the segment of position i
          }
          if (tid == 0) {
            S.segs[total] = (uint16_t)N;
            S.pre[N] = (uint16_t)total;
          }
        }
        __syncthreads();

        // ---- 3. lower median of every segment: rank counting inside the
        // segment, or (more than kRankMax points) a warp radix select
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          const uint32_t i = (uint32_t)tid + (uint32_t)q * T;
          const uint32_t k = kq[q];
          if (i >= N || k == kNoCell) continue;
          const uint32_t sx = segq[q];
          const uint32_t b = S.segs[sx], e = min((uint32_t)S.segs[sx + 1], (uint32_t)cc[k].begin + cc[k].count);
          const uint32_t w = e - b;
          if (w > kRankMax) {
            if (i == b) {
              const uint32_t slot = atomicAdd(&s_nbig, 1u);
              if (slot < (uint32_t)kSubtreeBigCap) S.biglist[slot] = (uint16_t)sx; else set_status(t, ST_INTERNAL);
            }
            continue;
          }
          const uint32_t key = keyq[q];
          uint32_t rk = 0;
          for (uint32_t j = b; j < e; ++j) {
            const uint32_t kj = S.gk[j];
            rk += (kj < key) | ((kj == key) & (j < i));
          }
          if (rk == (w - 1) / 2) S.smed[sx] = key;
        }
        __syncthreads();
        if (s_nbig) {
          const uint32_t nbig = min(s_nbig, (uint32_t)kSubtreeBigCap);
          for (uint32_t j = warp; j < nbig; j += NW) {
            const uint32_t sx = S.biglist[j];
            const uint32_t b = S.segs[sx];
            const uint16_t k = S.cellid[b];
            const uint32_t e = min((uint32_t)S.segs[sx + 1], (uint32_t)cc[k].begin + cc[k].count);
            const uint32_t* g = S.gk + b;
            const uint32_t m = warp_weighted_select<true>(e - b, (e - b - 1) / 2, S.whist + warp * 256,
                                                          [&](uint32_t jj) { return g[jj]; },
                                                          [](uint32_t) { return 1u; });
            if (lane == 0) S.smed[sx] = m;
          }
          __syncthreads();
        }

        // ---- 4. weighted lower median per cell: the smallest segment median m
        // whose segments with median <= m hold >= ceil(W/2) points, i.e. the
        // key of weighted rank (W-1)/2. A cell's segments are [pre[begin],
        // pre[end]). One warp per cell, no block barrier: up to 256 segments
        // are held in registers and the key is settled one bit per step by a
        // warp sum; more segments go through the warp's radix histogram.
        for (uint32_t k = warp; k < ncur; k += NW) {
          const uint32_t b = cc[k].begin, e = b + cc[k].count;
          const uint32_t s0 = S.pre[b], s1 = S.pre[e], ns = s1 - s0;
          const bool unit = t.combine_rule == 1;  // every subset counts once (segments are non-empty)
          const uint32_t rank = unit ? (ns - 1u) / 2u : (cc[k].count - 1u) / 2u;
          auto key_of = [&](uint32_t j) { return S.smed[s0 + j]; };
          auto w_of = [&](uint32_t j) {
            return unit ? 1u : min((uint32_t)S.segs[s0 + j + 1], e) - S.segs[s0 + j];
          };
          uint32_t m;
          if (ns <= 32u)
            m = warp_wsel_bits<1>(ns, rank, key_of, w_of);
          else if (ns <= 64u)
            m = warp_wsel_bits<2>(ns, rank, key_of, w_of);
          else if (ns <= 128u)
            m = warp_wsel_bits<4>(ns, rank, key_of, w_of);
          else if (ns <= 256u)
            m = warp_wsel_bits<8>(ns, rank, key_of, w_of);
          else
            m = warp_weighted_select(ns, rank, S.whist + warp * 256, key_of, w_of);
          if (lane == 0) cc[k].mkey = m;
        }
        __syncthreads();
        for (uint32_t k = tid; k < ncur; k += T) {
          t.out_vals[cc[k].heap] = key_float(cc[k].mkey);
          t.out_dims[cc[k].heap] = (int8_t)cc[k].dim;
        }

        // ---- 5. stable partition of the local order (key <= split to the
        // left): left ranks from warp ballots and one scan of the block counts
        {
          unsigned lbq[kQ];
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const uint32_t i = (uint32_t)tid + (uint32_t)q * T;
            const uint32_t k = kq[q];
            const bool left = i < N && k != kNoCell && keyq[q] <= cc[k].mkey;
            lbq[q] = __ballot_sync(0xffffffffu, left);
            if (lane == 0) s_bcnt[q * NW + warp] = (uint32_t)__popc(lbq[q]);
          }
          __syncthreads();
          uint32_t lpre[kQ], tot;
          block_counts_scan(lbq, s_bcnt, lane, warp, lpre, &tot);
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const uint32_t i = (uint32_t)tid + (uint32_t)q * T;
            if (i < N) S.pre[i] = (uint16_t)lpre[q];  // left points before position i
          }
          if (tid == 0) S.pre[N] = (uint16_t)tot;
          __syncthreads();
          for (uint32_t k = tid; k < ncur; k += T)
            cc[k].lcount = (uint16_t)(S.pre[cc[k].begin + cc[k].count] - S.pre[cc[k].begin]);
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const uint32_t i = (uint32_t)tid + (uint32_t)q * T;
            if (i >= N) continue;
            const uint32_t k = kq[q];
            const uint16_t o = ordA[i];
            if (k == kNoCell) {
              ordB[i] = o;
              continue;
            }
            const uint32_t b = cc[k].begin;
            const uint32_t pb = S.pre[b];
            const uint32_t L = (uint32_t)S.pre[b + cc[k].count] - pb;
            const uint32_t lb = lpre[q] - pb;
            const uint32_t dst = ((lbq[q] >> lane) & 1u) ? b + lb : b + L + (i - b - lb);
            ordB[dst] = o;
          }
        }
        __syncthreads();
        {
          uint16_t* x = ordA;
          ordA = ordB;
          ordB = x;
        }

        // ---- 6. children: a scan over the cells numbers the live children
        // (their number is parked in the parent's mkey); every position takes
        // its child's number when the next level reads its cell (step 2)
        const int nlevel = level + 1;
        uint32_t run_out = 0;
        int nwhere = 0;
        if (ncur <= (uint32_t)T) {
          // a cell per thread: one scan with a single barrier
          const uint32_t k = tid;
          LCell ch[2] = {};
          bool live[2] = {false, false};
          if (k < ncur) {
            const LCell p = cc[k];
            const uint32_t L = p.lcount, R = p.count - L;
            const int stall = (R == 0) ? p.stall + 1 : 0;
            const uint32_t cbeg[2] = {p.begin, p.begin + L};
            const uint32_t cn[2] = {L, R};
#pragma unroll
            for (int side = 0; side < 2; ++side) {
              const uint32_t heap = 2u * p.heap + 1u + (uint32_t)side;
              if (is_terminal(t, cn[side], nlevel, stall)) {
                record_terminal(t, c.begin + cbeg[side], cn[side], heap, nlevel);
              } else if (t.depth == 0 && nlevel >= t.max_levels) {
                set_status(t, ST_LEVEL_CAP);
              } else {
                ch[side] = LCell{heap, 0u, (uint16_t)cbeg[side], (uint16_t)cn[side], 0, 0, (uint8_t)stall};
                live[side] = true;
              }
            }
          }
          const uint32_t nlive = (uint32_t)live[0] + (uint32_t)live[1];
          const uint32_t ex = block_excl_scan_1bar(nlive, s_wtot, lane, warp, &run_out);
          nwhere = run_out <= (uint32_t)kCells ? 0 : 1;
          LCell* nc = nwhere ? gslice + (size_t)(which ^ 1) * slice_cells : S.tab + (which ^ 1) * kCells;
          if (k < ncur) {
            const uint32_t li = live[0] ? ex : kNoCell;
            const uint32_t ri = live[1] ? ex + (live[0] ? 1u : 0u) : kNoCell;
            if (live[0]) nc[li] = ch[0];
            if (live[1]) nc[ri] = ch[1];
            cc[k].mkey = li | (ri << 16);
          }
        } else {
          uint32_t total_live = 0;
          {
            // count the live children first to choose where the next table lives
            uint32_t sum = 0;
            for (uint32_t k = tid; k < ncur; k += T) {
              const LCell p = cc[k];
              const uint32_t L = p.lcount, R = p.count - L;
              const int stall = (R == 0) ? p.stall + 1 : 0;
              const bool cap = t.depth == 0 && nlevel >= t.max_levels;
              sum += (!is_terminal(t, L, nlevel, stall) && !cap) + (!is_terminal(t, R, nlevel, stall) && !cap);
            }
            block_excl_scan(sum, tmp, &total_live);
          }
          nwhere = total_live <= (uint32_t)kCells ? 0 : 1;
          LCell* nc = nwhere ? gslice + (size_t)(which ^ 1) * slice_cells : S.tab + (which ^ 1) * kCells;
          for (uint32_t k0 = 0; k0 < ncur; k0 += T) {
            const uint32_t k = k0 + tid;
            LCell ch[2] = {};
            bool live[2] = {false, false};
            if (k < ncur) {
              const LCell p = cc[k];
              const uint32_t L = p.lcount, R = p.count - L;
              const int stall = (R == 0) ? p.stall + 1 : 0;
              const uint32_t cbeg[2] = {p.begin, p.begin + L};
              const uint32_t cn[2] = {L, R};
#pragma unroll
              for (int side = 0; side < 2; ++side) {
                const uint32_t heap = 2u * p.heap + 1u + (uint32_t)side;
                if (is_terminal(t, cn[side], nlevel, stall)) {
                  record_terminal(t, c.begin + cbeg[side], cn[side], heap, nlevel);
                } else if (t.depth == 0 && nlevel >= t.max_levels) {
                  set_status(t, ST_LEVEL_CAP);
                } else {
                  ch[side] = LCell{heap, 0u, (uint16_t)cbeg[side], (uint16_t)cn[side], 0, 0, (uint8_t)stall};
                  live[side] = true;
                }
              }
            }
            const uint32_t nlive = (uint32_t)live[0] + (uint32_t)live[1];
            uint32_t tot;
            const uint32_t ex = block_excl_scan(nlive, tmp, &tot);
            if (k < ncur) {
              const uint32_t li = live[0] ? run_out + ex : kNoCell;
              const uint32_t ri = live[1] ? run_out + ex + (live[0] ? 1u : 0u) : kNoCell;
              if (live[0]) nc[li] = ch[0];
              if (live[1]) nc[ri] = ch[1];
              cc[k].mkey = li | (ri << 16);
            }
            run_out += tot;
          }
        }
        if (tid == 0) {
          s_ncur = run_out;
          s_where = (uint32_t)nwhere;
        }
        // every position takes its child's number at the start of the next
        // level (from this table's mkey); the barrier publishes the table
        __syncthreads();
        prev_global = decltype(in_global)::value ? 1 : 0;
        which ^= 1;
        level = nlevel;
      };
      if (s_where)
        level_body(std::true_type{});
      else
        level_body(std::false_type{});
    }

    // ---- write the permutation in final order
    for (uint32_t i = tid; i < N; i += T) {
      const uint32_t o = c.begin + ordA[i];
      t.out_perm[(int64_t)c.begin + i] = P ? P[o] : o;
    }
    if (tid == 0) atomicSub(t.live, 1);
  }
}

// One warp per terminal cell: offsets of the leaves at level L below it and
// sentinels (dim -1, value +inf) on its own node and every node below it.
__global__ void k_finalize(const TreeDev* tree, const uint32_t* term_count) {
  const TreeDev& t = *tree;
  const uint32_t nrec = min(*term_count, t.term_cap);
  const int L = t.depth > 0 ? t.depth : *t.levels;
  const int lane = threadIdx.x & 31;
  const uint32_t rec = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0) t.out_offs[(int64_t)1 << L] = t.n;
  if (rec >= nrec) return;
  const TermRec tr = t.terms[rec];
  const int lv = tr.level;
  if (lv > L) return;
  const int64_t k = (int64_t)tr.heap - (((int64_t)1 << lv) - 1);
  const int64_t span = (int64_t)1 << (L - lv);
  const int64_t leaf0 = k * span;
  for (int64_t j = lane; j < span; j += 32)
    t.out_offs[leaf0 + j] = (j == 0) ? (int64_t)tr.begin : (int64_t)tr.begin + tr.count;
  for (int l2 = lv; l2 < L; ++l2) {
    const int64_t width = (int64_t)1 << (l2 - lv);
    const int64_t first = ((int64_t)tr.heap + 1) * width - 1;
    for (int64_t j = lane; j < width; j += 32) {
      t.out_dims[first + j] = -1;
      t.out_vals[first + j] = __int_as_float(0x7f800000);
    }
  }
}

// Finalize of several trees: grid (chunks, trees); each warp takes terminal
// records of its tree in turn (same per-record work as k_finalize).
__global__ void k_finalize_many(const TreeDev* trees, const uint32_t* slots, uint32_t nslots) {
  const uint32_t si = blockIdx.y;
  if (si >= nslots) return;
  const TreeDev& t = trees[slots[si]];
  const uint32_t nrec = min(*t.term_count, t.term_cap);
  const int L = t.depth > 0 ? t.depth : *t.levels;
  const int lane = threadIdx.x & 31;
  const uint32_t wpb = blockDim.x >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) t.out_offs[(int64_t)1 << L] = t.n;
  for (uint32_t rec = blockIdx.x * wpb + (threadIdx.x >> 5); rec < nrec; rec += gridDim.x * wpb) {
    const TermRec tr = t.terms[rec];
    const int lv = tr.level;
    if (lv > L) continue;
    const int64_t k = (int64_t)tr.heap - (((int64_t)1 << lv) - 1);
    const int64_t span = (int64_t)1 << (L - lv);
    const int64_t leaf0 = k * span;
    for (int64_t j = lane; j < span; j += 32)
      t.out_offs[leaf0 + j] = (j == 0) ? (int64_t)tr.begin : (int64_t)tr.begin + tr.count;
    for (int l2 = lv; l2 < L; ++l2) {
      const int64_t width = (int64_t)1 << (l2 - lv);
      const int64_t first = ((int64_t)tr.heap + 1) * width - 1;
      for (int64_t j = lane; j < width; j += 32) {
        t.out_dims[first + j] = -1;
        t.out_vals[first + j] = __int_as_float(0x7f800000);
      }
    }
  }
}

__global__ void k_iota(uint32_t* out, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = i;
}

}  // namespace

void launch_iota(uint32_t* out, uint32_t n, cudaStream_t st) {
  if (n == 0) return;
  TraceScope ts(K_IOTA, st, n);
  k_iota<<<std::min<uint32_t>((n + 255) / 256, 4096u), 256, 0, st>>>(out, n);
}

// The kernel instance of a shape.
using SubtreeKernel = void (*)(const TreeDev*, const Cell*, uint32_t, const uint32_t*, uint32_t, uint32_t*, LCell*,
                               uint32_t, uint32_t);
SubtreeKernel subtree_kernel(const SubtreeShape& sh) {
  return sh.q == kSubWide.q ? k_subtree<true> : k_subtree<false>;
}

cudaError_t prepare_subtree_kernel() {
  for (const SubtreeShape* sh : {&kSubNarrow, &kSubWide}) {
    const cudaError_t e = cudaFuncSetAttribute(subtree_kernel(*sh), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sh->smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void launch_subtree(const SubtreeShape& sh, const TreeDev* trees, const Cell* list, uint32_t count,
                    const uint32_t* count_dev, bool reversed, uint32_t* head, LCell* slices, uint32_t slice_cells,
                    uint32_t grid, uint64_t points, cudaStream_t st) {
  if (count == 0 || grid == 0) return;
  cudaMemsetAsync(head, 0, sizeof(uint32_t), st);
  const uint32_t probe = fault_take(KDT_FAULT_WAIT) ? 1024u : 0u;
  TraceScope ts(K_SUBTREE, st, points);
  subtree_kernel(sh)<<<grid, T, sh.smem, st>>>(trees, list, count, count_dev, reversed ? 1u : 0u, head, slices,
                                               slice_cells, probe);
}

void launch_finalize_many(const TreeDev* trees, const uint32_t* slots, uint32_t nslots, uint32_t max_records,
                          cudaStream_t st) {
  if (nslots == 0) return;
  TraceScope ts(K_FINALIZE, st);
  const uint32_t chunks = std::max<uint32_t>(1, std::min<uint32_t>((max_records + 7) / 8, 8192));
  k_finalize_many<<<dim3(chunks, nslots), 256, 0, st>>>(trees, slots, nslots);
}

void launch_finalize(const TreeDev* tree, const uint32_t* term_count, uint32_t max_terms, cudaStream_t st) {
  const uint32_t blocks = (max_terms + 7) / 8 + 1;
  TraceScope ts(K_FINALIZE, st);
  k_finalize<<<blocks, 256, 0, st>>>(tree, term_count);
}

}  // namespace kdt
