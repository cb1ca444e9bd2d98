// kdt_step.cu -- one level of the multi-CTA pipeline for cells too large to
// finish in shared memory.
//
// For every big cell c of the step (paper, Sec. 2: a level splits each of its
// cells along the key coordinate t at a median):
//   0. (roots only) the points are reordered by subset (counting pass, or
//      closed form for subsets by index mod r), so that every (cell, subset)
//      segment is contiguous from then on;
//   1. key coordinate: cyclic (Sec. 1) or widest range (Sec. 1, Friedman
//      rule; computed for the root here, for every other cell by the parent's
//      scatter, which reduces each child's per-coordinate min and max while it
//      moves the columns);
//   2. per (cell, subset) segment (the subsets of Sec. 3.2 / App. C.2): its
//      position range, from the cell's subset offsets;
//   3. per segment: the exact lower median (8-bit MSD radix select) read in
//      place from the key column;
//   4. per cell: the count-weighted lower median of the segment medians;
//   5. children sizes from per-tile counts and a per-cell scan of them; the
//      children are classified (terminal / small / big) before the move;
//   6. stable partition of all d columns, the permutation and the subset ids
//      around the split (key <= split to the left); the scatter also writes
//      the big children's subset offsets.
// Work is split into tiles of kTile points of one cell; a thread owns kItems
// points of a tile (strided by the block size, so every load is coalesced)
// and issues all of its loads before it uses any of them.
#include <algorithm>

#include "kdt_internal.cuh"
#include "kdt_launch.h"
#include "kdt_ptx.cuh"
#include "kdt_trace.h"

namespace kdt {

namespace {

constexpr int kItems = kTile / kTileThreads;
constexpr int kWarps = kTileThreads / 32;
constexpr int kPsGroup = 2;                       // tiles per block of the root presort
constexpr int kPsPoints = kPsGroup * kTile;
constexpr int kPsThreads = 512;
constexpr int kPsItems = kPsPoints / kPsThreads;
constexpr size_t kPsSmemBytes = (size_t)kPsPoints * 6;  // one word and one u16 subset per point

__device__ __forceinline__ bool tile_of(const StepDev& s, uint32_t tile, uint2* out) {
  if (tile >= *s.ntiles_total) return false;
  *out = s.tiles[tile];
  return true;
}

// ---------------------------------------------------------------- prep

// Single CTA: per-cell tile and segment counts, exclusive scans, key dims
// that are already known. Each thread takes kPrepItems consecutive cells per
// round, so a deep level's many cells cost few block scans.
constexpr int kPrepItems = 4;

__global__ void k_prep(const TreeDev* trees, StepDev s) {
  __shared__ uint32_t tmp[33];
  uint32_t tile_run = 0, seg_run = 0;
  const uint32_t ncells = ncells_of(s);
  for (uint32_t c0 = 0; c0 < ncells; c0 += blockDim.x * kPrepItems) {
    const uint32_t cb = c0 + threadIdx.x * kPrepItems;
    uint32_t nt[kPrepItems], ns[kPrepItems], st = 0, ss = 0;
#pragma unroll
    for (int q = 0; q < kPrepItems; ++q) {
      const uint32_t c = cb + q;
      nt[q] = 0;
      ns[q] = 0;
      if (c < ncells) {
        const Cell cell = s.cells[c];
        const TreeDev& t = trees[cell.tree];
        nt[q] = (cell.count + kTile - 1) / kTile;
        ns[q] = (uint32_t)t.r;
        if (t.key_rule == KEY_CYCLIC)
          s.kdim[c] = (uint32_t)(cell.level % t.d);
        else if (cell.dim >= 0)
          s.kdim[c] = (uint32_t)cell.dim;
      }
      st += nt[q];
      ss += ns[q];
    }
    uint32_t tot_t, tot_s;
    uint32_t et = block_excl_scan(st, tmp, &tot_t);
    uint32_t es = block_excl_scan(ss, tmp, &tot_s);
#pragma unroll
    for (int q = 0; q < kPrepItems; ++q) {
      const uint32_t c = cb + q;
      if (c < ncells) {
        s.tile_base[c] = tile_run + et;
        s.seg_base[c] = seg_run + es;
      }
      et += nt[q];
      es += ns[q];
    }
    tile_run += tot_t;
    seg_run += tot_s;
  }
  if (threadIdx.x == 0) {
    s.tile_base[ncells] = tile_run;
    s.seg_base[ncells] = seg_run;
    *s.ntiles_total = tile_run;
    *s.bigseg_count = 0;
    *s.midseg_count = 0;
  }
}

// One warp per cell: tile list entries; zeroed subset counts of a presorted
// root, and (widest spread, coordinate not known yet) the identities in its
// first tile's min / max record, which the presort's groups reduce into.
// (Most cells of a deep level have one to three tiles.)
__device__ __forceinline__ void tiles_cell(const TreeDev* trees, const StepDev& s, uint32_t c) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t tb = s.tile_base[c], te = s.tile_base[c + 1];
  for (uint32_t j = tb + lane; j < te; j += 32u) s.tiles[j] = make_uint2(c, (j - tb) * (uint32_t)kTile);
  const Cell cell = s.cells[c];
  if (cell.level == 0) {
    const TreeDev& t = trees[cell.tree];
    if (t.presorted) {
      for (uint32_t j = lane; j < (uint32_t)t.r; j += 32u) t.root_cur[j] = 0;
      if (t.key_rule == KEY_WIDEST && cell.dim < 0 && tb < te)
        for (uint32_t j = lane; j < 2u * (uint32_t)t.d; j += 32u)
          s.tile_mm[((size_t)tb * 2 * kMaxDims + j / 2) * 2 + (j & 1)] = (j & 1) ? 0u : 0xffffffffu;
    }
  }
}

__global__ void k_tiles(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  const uint32_t wpb = blockDim.x >> 5;
  for (uint32_t c = blockIdx.x * wpb + (threadIdx.x >> 5); c < nc; c += gridDim.x * wpb) tiles_cell(trees, s, c);
}

// ------------------------------------------------------ root presort

__device__ __forceinline__ bool presort_tile(const TreeDev* trees, const StepDev& s, uint32_t tile, uint2* tl,
                                             Cell* cell) {
  if (!tile_of(s, tile, tl)) return false;
  *cell = s.cells[tl->x];
  return cell->level == 0 && trees[cell->tree].presorted;
}

// Points per subset of every presorted root with explicit subset ids. Each
// CTA counts a contiguous range of tiles into a shared histogram and adds it
// to the root's totals (root_cur) when the range moves to another tree and at
// its end.
__global__ void __launch_bounds__(kTileThreads) k_ps_count(const TreeDev* trees, StepDev s) {
  __shared__ uint32_t hist[kMaxSubsets];
  const uint32_t ntiles = *s.ntiles_total;
  const uint32_t t_begin = (uint32_t)(((uint64_t)blockIdx.x * ntiles) / gridDim.x);
  const uint32_t t_end = (uint32_t)(((uint64_t)(blockIdx.x + 1) * ntiles) / gridDim.x);
  int32_t cur = -1;  // tree whose counts hist holds
  auto flush = [&]() {
    __syncthreads();
    if (cur >= 0) {
      const TreeDev& t = trees[cur];
      for (int j = threadIdx.x; j < t.r; j += blockDim.x)
        if (hist[j]) atomicAdd(&t.root_cur[j], hist[j]);
    }
    __syncthreads();
  };
  for (uint32_t tile = t_begin; tile < t_end; ++tile) {
    const uint2 tl = s.tiles[tile];
    const Cell cell = s.cells[tl.x];
    const TreeDev& t = trees[cell.tree];
    if (cell.level != 0 || !t.presorted || t.subset_mode != SUB_EXPLICIT) continue;
    if (cell.tree != cur) {
      flush();
      for (int j = threadIdx.x; j < t.r; j += blockDim.x) hist[j] = 0;
      cur = cell.tree;
      __syncthreads();
    }
    const uint32_t end = min(tl.y + (uint32_t)kTile, cell.count);
    uint32_t sub[kItems];
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      const uint32_t i = tl.y + threadIdx.x + q * kTileThreads;
      sub[q] = i < end ? subset_of(t, t.sid_in, 0u, (int64_t)i) : 0xffffffffu;
    }
#pragma unroll
    for (int q = 0; q < kItems; ++q)
      if (sub[q] != 0xffffffffu) atomic_add_shared(&hist[sub[q]], 1u);
  }
  flush();
}

// One CTA per root cell: its subset offsets (r + 1 entries). Explicit ids:
// exclusive scan of the counts (which also become the fill cursors); subsets
// by index mod r: r_j = floor(n/r) + [j < n mod r] points each; contiguous
// subsets (already in order): subset j starts at ceil(j n / r).
__device__ __forceinline__ void ps_offsets_cell(const TreeDev* trees, const StepDev& s, uint32_t c) {
  __shared__ uint32_t tmp[33];
  const Cell cell = s.cells[c];
  if (cell.level != 0) return;
  const TreeDev& t = trees[cell.tree];
  const uint32_t r = (uint32_t)t.r, n = cell.count;
  if (t.subset_mode == SUB_EXPLICIT) {
    uint32_t run = 0;
    for (uint32_t j0 = 0; j0 < r; j0 += blockDim.x) {
      const uint32_t j = j0 + threadIdx.x;
      const uint32_t v = j < r ? t.root_cur[j] : 0u;
      uint32_t tot;
      const uint32_t ex = block_excl_scan(v, tmp, &tot);
      if (j < r) {
        t.root_off[j] = run + ex;
        t.root_cur[j] = run + ex;
      }
      run += tot;
    }
    if (threadIdx.x == 0) {
      t.root_off[r] = run;
      if (run != n) set_status(t, ST_INTERNAL);
    }
  } else if (t.subset_mode == SUB_MOD) {
    const uint32_t q = n / r, rem = n % r;
    for (uint32_t j = threadIdx.x; j <= r; j += blockDim.x) t.root_off[j] = j * q + min(j, rem);
  } else {
    for (uint32_t j = threadIdx.x; j <= r; j += blockDim.x)
      t.root_off[j] = (uint32_t)(((uint64_t)j * n + r - 1) / r);
  }
}

__global__ void k_ps_offsets(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  for (uint32_t c = blockIdx.x; c < nc; c += gridDim.x) {
    ps_offsets_cell(trees, s, c);
    __syncthreads();  // the cell's shared memory is free for the next one
  }
}

// Per group of kPsGroup consecutive tiles of a presorted root (kPsPoints
// points): every point gets a rank inside its subset within the group
// (shared-memory counter; order inside a subset is immaterial, see
// kdt_internal.cuh), each subset of the group reserves a run of its place in
// subset order (explicit ids: from the fill cursors; index mod r: closed
// form), and every column passes through shared memory in subset order so
// that the stores are contiguous runs of about kPsPoints / r points.
__global__ void __launch_bounds__(kPsThreads) k_ps_move(const TreeDev* trees, StepDev s) {
  uint2 tl;
  Cell cell;
  if (!presort_tile(trees, s, blockIdx.x, &tl, &cell)) return;
  const TreeDev& t = trees[cell.tree];
  // widest spread: the group's min / max key per coordinate go by atomics into
  // the record of the root's first tile, the other tiles' records hold the
  // identities
  const bool want_mm = t.key_rule == KEY_WIDEST && cell.dim < 0;
  if ((tl.y / (uint32_t)kTile) % (uint32_t)kPsGroup != 0u) {  // the group's first tile runs it
    if (want_mm)
      for (int j = threadIdx.x; j < 2 * t.d; j += blockDim.x)
        s.tile_mm[((size_t)blockIdx.x * 2 * kMaxDims + j / 2) * 2 + (j & 1)] = (j & 1) ? 0u : 0xffffffffu;
    return;
  }
  extern __shared__ __align__(16) uint32_t ps_buf[];  // kPsPoints words, then kPsPoints u16 subsets
  uint16_t* lsub = (uint16_t*)(ps_buf + kPsPoints);
  __shared__ uint32_t loff[kMaxSubsets];   // counts, then local offsets
  __shared__ uint32_t gbase[kMaxSubsets];  // global start of each subset's run
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t gmm[kMaxDims][2];
  const uint32_t r = (uint32_t)t.r, i0 = tl.y, end = min(i0 + (uint32_t)kPsPoints, cell.count);
  const uint32_t m = end - i0;
  const bool expl = t.subset_mode == SUB_EXPLICIT;
  for (uint32_t j = threadIdx.x; j < r; j += kPsThreads) loff[j] = 0;
  for (int j = threadIdx.x; j < 2 * t.d; j += kPsThreads) gmm[j / 2][j & 1] = (j & 1) ? 0u : 0xffffffffu;
  __syncthreads();
  uint32_t sub[kPsItems], lp[kPsItems];
#pragma unroll
  for (int q = 0; q < kPsItems; ++q) {
    const uint32_t i = i0 + threadIdx.x + q * kPsThreads;
    sub[q] = i < end ? (expl ? subset_of(t, t.sid_in, 0u, (int64_t)i) : i % r) : 0xffffffffu;
  }
#pragma unroll
  for (int q = 0; q < kPsItems; ++q) lp[q] = sub[q] != 0xffffffffu ? atomic_add_shared(&loff[sub[q]], 1u) : 0u;
  __syncthreads();
  uint32_t run = 0;
  for (uint32_t j0 = 0; j0 < r; j0 += kPsThreads) {
    const uint32_t j = j0 + threadIdx.x;
    const uint32_t c = j < r ? loff[j] : 0u;
    if (j < r) {
      if (expl)
        gbase[j] = c ? atomicAdd(&t.root_cur[j], c) : 0u;
      else  // indices below i0 in subset j: floor(i0 / r) + [j < i0 mod r]
        gbase[j] = t.root_off[j] + i0 / r + (j < i0 % r ? 1u : 0u);
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan(c, tmp, &tot);
    if (j < r) loff[j] = run + ex;
    run += tot;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kPsItems; ++q)
    if (sub[q] != 0xffffffffu) {
      lp[q] += loff[sub[q]];
      lsub[lp[q]] = (uint16_t)sub[q];
    }
  __syncthreads();
  // place a value per point in subset order, then store the runs
  auto pass = [&](auto value_of, auto store) {
#pragma unroll
    for (int q = 0; q < kPsItems; ++q)
      if (sub[q] != 0xffffffffu) ps_buf[lp[q]] = value_of(q);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < m; j += kPsThreads) {
      const uint32_t sj = lsub[j];
      const uint32_t dst = gbase[sj] + (j - loff[sj]);
      if (dst < cell.count) store(dst, ps_buf[j]); else set_status(t, ST_INTERNAL);
    }
    __syncthreads();
  };
  const int64_t n = t.n;
  // each column's loads are issued before the previous column's passes
  uint32_t x[kPsItems], xn[kPsItems];
  auto load = [&](int l, uint32_t (&v)[kPsItems]) {
    const uint32_t* X = (const uint32_t*)(t.x_in + (int64_t)l * n);
#pragma unroll
    for (int q = 0; q < kPsItems; ++q) {
      const uint32_t i = i0 + threadIdx.x + q * kPsThreads;
      v[q] = i < end ? __ldg(X + i) : 0u;
    }
  };
  // the input's NaN check (the scatter of a presorted root skips it): a NaN
  // key lies above +inf's or below -inf's
  bool nan = false;
  load(0, x);
  for (int l = 0; l < t.d; ++l) {
    if (l + 1 < t.d) load(l + 1, xn);
    if (want_mm) {
      uint32_t lo = 0xffffffffu, hi = 0u;
#pragma unroll
      for (int q = 0; q < kPsItems; ++q)
        if (sub[q] != 0xffffffffu) {
          const uint32_t k = ord_key(__uint_as_float(x[q]));
          lo = min(lo, k);
          hi = max(hi, k);
        }
      nan |= hi > 0xff800000u || lo < 0x007fffffu;
      lo = __reduce_min_sync(0xffffffffu, lo);
      hi = __reduce_max_sync(0xffffffffu, hi);
      if ((threadIdx.x & 31) == 0) {
        atomic_min_shared(&gmm[l][0], lo);
        atomic_max_shared(&gmm[l][1], hi);
      }
    } else {
#pragma unroll
      for (int q = 0; q < kPsItems; ++q) nan |= sub[q] != 0xffffffffu && is_nan_bits(__uint_as_float(x[q]));
    }
    uint32_t* out = (uint32_t*)(t.xbuf[1] + (int64_t)l * n);
    pass([&](int q) { return x[q]; }, [&](uint32_t dst, uint32_t v) { out[dst] = v; });
#pragma unroll
    for (int q = 0; q < kPsItems; ++q) x[q] = xn[q];
  }
  if (nan) set_status(t, ST_NAN_INPUT);
  if (want_mm) {  // the passes' barriers order the shared-memory reductions before this
    // into the root's first tile record (identities set by k_tiles); this
    // tile's own record, if another, holds the identities
    const uint32_t tb = s.tile_base[tl.x];
    for (int j = threadIdx.x; j < 2 * t.d; j += kPsThreads) {
      uint32_t* acc = &s.tile_mm[((size_t)tb * 2 * kMaxDims + j / 2) * 2 + (j & 1)];
      if (j & 1) atomicMax(acc, gmm[j / 2][1]); else atomicMin(acc, gmm[j / 2][0]);
      if (blockIdx.x != tb)
        s.tile_mm[((size_t)blockIdx.x * 2 * kMaxDims + j / 2) * 2 + (j & 1)] = (j & 1) ? 0u : 0xffffffffu;
    }
  }
  pass([&](int q) { return i0 + threadIdx.x + q * kPsThreads; },
       [&](uint32_t dst, uint32_t v) { t.pbuf[1][dst] = v; });
  if (expl) {
    if (t.sid_bytes == 1)
      pass([&](int q) { return sub[q]; }, [&](uint32_t dst, uint32_t v) { ((uint8_t*)t.sbuf[1])[dst] = (uint8_t)v; });
    else
      pass([&](int q) { return sub[q]; },
           [&](uint32_t dst, uint32_t v) { ((uint16_t*)t.sbuf[1])[dst] = (uint16_t)v; });
  }
}

// ------------------------------------------------------- widest spread

// Per tile and coordinate of a cell whose key coordinate is not known yet
// (the root): min and max key, reduced per cell by k_pick_dim.
__global__ void __launch_bounds__(kTileThreads) k_minmax(const TreeDev* trees, StepDev s) {
  uint2 tl;
  if (!tile_of(s, blockIdx.x, &tl)) return;
  const Cell cell = s.cells[tl.x];
  const TreeDev& t = trees[cell.tree];
  if (t.key_rule != KEY_WIDEST || cell.dim >= 0 || t.presorted) return;  // presorted: from k_ps_move
  __shared__ uint32_t red[2][kWarps];
  const float* X = src_cols(t, cell.level) + cell.begin;
  const int64_t n = t.n;
  const uint32_t end = min(tl.y + (uint32_t)kTile, cell.count);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool nan = false;
  for (int l = 0; l < t.d; ++l) {
    float x[kItems];
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      const uint32_t i = tl.y + threadIdx.x + q * kTileThreads;
      x[q] = i < end ? X[(int64_t)l * n + i] : 0.0f;
    }
    uint32_t lo = 0xffffffffu, hi = 0u;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      const uint32_t i = tl.y + threadIdx.x + q * kTileThreads;
      if (i < end) {
        nan |= is_nan_bits(x[q]);
        const uint32_t k = ord_key(x[q]);
        lo = min(lo, k);
        hi = max(hi, k);
      }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
      red[0][warp] = lo;
      red[1][warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kWarps; ++w) {
        lo = min(lo, red[0][w]);
        hi = max(hi, red[1][w]);
      }
      s.tile_mm[((size_t)blockIdx.x * 2 * kMaxDims + l) * 2 + 0] = lo;
      s.tile_mm[((size_t)blockIdx.x * 2 * kMaxDims + l) * 2 + 1] = hi;
    }
    __syncthreads();
  }
  if (nan) set_status(t, ST_NAN_INPUT);
}

// Range of a coordinate from its min and max keys: (double)max - (double)min,
// 0 when both are the same key.
__device__ __forceinline__ double key_range(uint32_t lo, uint32_t hi) {
  return (lo == hi) ? 0.0 : (double)key_float(hi) - (double)key_float(lo);
}

// One CTA per cell with an unknown widest coordinate: reduce the tile
// partials and pick the coordinate of largest range (lowest on ties). Every
// thread walks its own tiles, eight coordinates at a time (four 16-byte loads
// per tile: a tile's record holds min, max of each coordinate in turn).
__device__ __forceinline__ void pick_dim_cell(const TreeDev* trees, const StepDev& s, uint32_t c) {
  const Cell cell = s.cells[c];
  const TreeDev& t = trees[cell.tree];
  if (t.key_rule != KEY_WIDEST || cell.dim >= 0) return;
  __shared__ uint32_t slo[kMaxDims], shi[kMaxDims];
  for (int l = threadIdx.x; l < t.d; l += blockDim.x) {
    slo[l] = 0xffffffffu;
    shi[l] = 0u;
  }
  __syncthreads();
  // the roots of a sharded build's shards are parts of one root: every one
  // of them reduces the tiles of all
  const uint32_t tb = s.shards ? 0u : s.tile_base[c];
  // a presorted root's presort gathered its min / max in its first tile's
  // record; other roots' are spread over their tiles
  const uint32_t te = s.shards ? s.tile_base[ncells_of(s)] : (t.presorted ? tb + 1u : s.tile_base[c + 1]);
  const int lane = threadIdx.x & 31;
  for (int c0 = 0; c0 < t.d; c0 += 8) {
    const int nc = min(8, t.d - c0);
    uint32_t lo[8], hi[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      lo[q] = 0xffffffffu;
      hi[q] = 0u;
    }
    for (uint32_t j = tb + threadIdx.x; j < te; j += blockDim.x) {
      // 16-byte aligned: a record is 2 * kMaxDims * 2 words, c0 a multiple of 8
      const uint4* p = (const uint4*)(s.tile_mm + ((size_t)j * 2 * kMaxDims + c0) * 2);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        if (2 * h >= nc) break;
        const uint4 v = p[h];
        lo[2 * h] = min(lo[2 * h], v.x);
        hi[2 * h] = max(hi[2 * h], v.y);
        lo[2 * h + 1] = min(lo[2 * h + 1], v.z);
        hi[2 * h + 1] = max(hi[2 * h + 1], v.w);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < nc) {
        const uint32_t l2 = __reduce_min_sync(0xffffffffu, lo[q]);
        const uint32_t h2 = __reduce_max_sync(0xffffffffu, hi[q]);
        if (lane == 0) {
          atomic_min_shared(&slo[c0 + q], l2);
          atomic_max_shared(&shi[c0 + q], h2);
        }
      }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    double best_range = -1.0;
    for (int l = 0; l < t.d; ++l) {
      const double range = key_range(slo[l], shi[l]);
      if (range > best_range) {
        best_range = range;
        best = l;
      }
    }
    s.kdim[c] = (uint32_t)best;
  }
}

__global__ void __launch_bounds__(1024) k_pick_dim(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  for (uint32_t c = blockIdx.x; c < nc; c += gridDim.x) {
    pick_dim_cell(trees, s, c);
    __syncthreads();  // the cell's shared memory is free for the next one
  }
}

// ------------------------------------------------------------ segments

// Key column of a cell (raw float bits; ord_key is applied on every load).
__device__ __forceinline__ const uint32_t* key_column(const TreeDev& t, const Cell& cell, uint32_t dim) {
  return (const uint32_t*)(src_cols(t, cell.level) + (int64_t)dim * t.n);
}

__device__ __forceinline__ uint32_t kload(const uint32_t* p) { return ord_key(__uint_as_float(__ldg(p))); }


// One CTA per cell (after its key coordinate is known): size and first key
// of every (cell, subset) segment from the cell's subset offsets, and the
// lists of segments for the warp and CTA selects. Offsets are clamped to the
// cell, so a damaged table cannot send a later kernel outside it (it is
// reported instead).
__device__ __forceinline__ void segs_cell(const TreeDev* trees, const StepDev& s, uint32_t c) {
  const Cell cell = s.cells[c];
  const TreeDev& t = trees[cell.tree];
  const uint32_t r = (uint32_t)t.r;
  const uint32_t* off = cell.level == 0 ? t.root_off : s.off_cur + s.obase_cur[c];
  const uint32_t g0 = s.seg_base[c];
  const uint32_t* kc = key_column(t, cell, s.kdim[c]) + cell.begin;
  if (threadIdx.x == 0 && (off[0] != 0u || off[r] != cell.count)) set_status(t, ST_INTERNAL);
  for (uint32_t j = threadIdx.x; j < r; j += blockDim.x) {
    const uint32_t a = min(off[j], cell.count), b = min(off[j + 1], cell.count);
    if (b < a) set_status(t, ST_INTERNAL);
    const uint32_t w = b >= a ? b - a : 0u;
    s.seg_key[g0 + j] = kc + a;
    s.seg_w[g0 + j] = w;
    if (w > s.warp_max) {
      const uint32_t k = atomicAdd(s.bigseg_count, 1u);
      if (k < s.bigseg_cap) s.bigseg[k] = g0 + j; else set_status(t, ST_INTERNAL);
    } else if (w > s.tiny_max) {
      const uint32_t k = atomicAdd(s.midseg_count, 1u);
      if (k < s.midseg_cap) s.midseg[k] = g0 + j; else set_status(t, ST_INTERNAL);
    }
  }
}

__global__ void k_segs(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  for (uint32_t c = blockIdx.x; c < nc; c += gridDim.x) {
    segs_cell(trees, s, c);
    __syncthreads();  // the cell's shared memory is free for the next one
  }
}

// ------------------------------------------------------------ selection

// Batcher's odd-even merge sort of v[0, M) ascending, M a power of two. In
// the round of merge width 2p and distance k, position x is compared with
// x + k when x lies in an even block of k positions counted from k mod p and
// both lie in one block of 2p; every comparator is fixed at compile time.
template <int M>
__device__ __forceinline__ void oddeven_sort(uint32_t (&v)[M]) {
#pragma unroll
  for (int p = 1; p < M; p <<= 1)
#pragma unroll
    for (int k = p; k >= 1; k >>= 1)
#pragma unroll
      for (int x = 0; x < M; ++x) {
        const int j0 = k % p;
        if (x >= j0 && ((x - j0) / k) % 2 == 0 && x + k < M && x / (2 * p) == (x + k) / (2 * p)) {
          const uint32_t a = v[x], b = v[x + k];
          v[x] = min(a, b);
          v[x + k] = max(a, b);
        }
      }
}

// Lower median (rank (w-1)/2) of a segment of 1 <= w <= 2M keys by one
// thread. The keys are padded to 2M: M - 1 - (w-1)/2 copies of the smallest
// key 0, the rest the largest key ~0, so that the median has rank M - 1 among
// the 2M (padding keys equal to a real key would not change the element at
// that rank). Both halves are sorted; A ascending followed by B reversed is
// bitonic, so min(A[i], B[M-1-i]) over i are the M smallest of the 2M, and
// the largest of them is the element of rank M - 1.
template <int M>
__device__ __forceinline__ uint32_t thread_lower_median(const uint32_t* keys, uint32_t w) {
  const uint32_t zeros_end = w + (uint32_t)(M - 1) - (w - 1u) / 2u;  // [w, zeros_end) hold 0
  uint32_t a[M], b[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const uint32_t e = (uint32_t)i, f = (uint32_t)(i + M);
    a[i] = e < w ? kload(keys + e) : (e < zeros_end ? 0u : 0xffffffffu);
    b[i] = f < w ? kload(keys + f) : (f < zeros_end ? 0u : 0xffffffffu);
  }
  oddeven_sort<M>(a);
  oddeven_sort<M>(b);
  uint32_t med = 0u;
#pragma unroll
  for (int i = 0; i < M; ++i) med = max(med, min(a[i], b[M - 1 - i]));
  return med;
}

// One thread per segment of at most tiny_max <= kSelTinyMax points (the
// threads stride over the segments of the step). The network's size is
// chosen per warp, by the warp's largest segment, so a warp never runs two.
// Five CTAs per SM by a register bound (48 registers): the path waits on its
// loads, and the extra warps hide that better than keeping the larger
// networks in registers does (they spill about 300 bytes per thread to local
// memory; measured faster than four or six CTAs per SM).
__global__ void __launch_bounds__(256, 5) k_select_tiny(const TreeDev* trees, StepDev s) {
  const uint32_t nseg = s.seg_base[ncells_of(s)];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t g0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); g0 < nseg; g0 += stride) {
    const uint32_t g = g0 + lane;
    uint32_t w = g < nseg ? s.seg_w[g] : 0u;
    if (w > s.tiny_max) w = 0u;
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, w);
    if (wmax == 0u) continue;
    const uint32_t* keys = w ? s.seg_key[g] : nullptr;
    uint32_t med;
    if (wmax <= 8u)
      med = thread_lower_median<4>(keys, w);
    else if (wmax <= 16u)
      med = thread_lower_median<8>(keys, w);
    else if (wmax <= 32u)
      med = thread_lower_median<16>(keys, w);
    else
      med = thread_lower_median<32>(keys, w);
    if (w) s.seg_med[g] = med;
  }
}

// Lower median of 1 <= w <= 32K keys by one warp, element e = k * 32 + lane
// in register k of a lane. As in thread_lower_median the keys are padded to
// N = 32K with the smallest and the largest key so that the median has rank
// N/2 - 1; the bitonic network runs its stages up to size N/2 only, which
// leaves the first half ascending and the second descending: a bitonic
// sequence whose half-cleaner min(v[k], v[k + K/2]) holds the N/2 smallest
// keys, the largest of which (over the warp) is the median.
template <int K>
__device__ uint32_t warp_bitonic_median(const uint32_t* keys, uint32_t w) {
  static_assert(K >= 2 && (K & (K - 1)) == 0, "K: a power of two of at least 2");
  const int lane = threadIdx.x & 31;
  constexpr int N = 32 * K;
  const uint32_t zeros_end = w + (uint32_t)(N / 2 - 1) - (w - 1u) / 2u;  // [w, zeros_end) hold 0
  uint32_t v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t e = (uint32_t)(k * 32 + lane);
    v[k] = e < w ? kload(keys + e) : (e < zeros_end ? 0u : 0xffffffffu);
  }
#pragma unroll
  for (int size = 2; size <= N / 2; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int e = k * 32 + lane;
        const bool asc = (e & size) == 0;
        if (j >= 32) {
          const int kk = k ^ (j >> 5);
          if (k < kk) {
            const uint32_t lo = min(v[k], v[kk]), hi = max(v[k], v[kk]);
            v[k] = asc ? lo : hi;
            v[kk] = asc ? hi : lo;
          }
        } else {
          const uint32_t o = __shfl_xor_sync(0xffffffffu, v[k], j);
          const bool lower = (lane & j) == 0;
          v[k] = (lower == asc) ? min(v[k], o) : max(v[k], o);
        }
      }
    }
  }
  uint32_t m = 0u;
#pragma unroll
  for (int k = 0; k < K / 2; ++k) m = max(m, min(v[k], v[k + K / 2]));
  return __reduce_max_sync(0xffffffffu, m);
}

// State of a warp's radix select: the key bits found so far (`prefix`, all
// bits above `rem`) and the rank still sought below them.
struct RadixState {
  uint32_t prefix, rank;
  int rem;
};

__device__ __forceinline__ bool radix_start(uint32_t lo, uint32_t hi, uint32_t rank, RadixState* st) {
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  st->rank = rank;
  if (lo >= hi) {
    st->prefix = lo;
    st->rem = 0;
    return false;
  }
  st->rem = 32 - __clz(lo ^ hi);
  st->prefix = st->rem == 32 ? 0u : (lo & ~((1u << st->rem) - 1u));
  return true;
}

// Lower median (rank (w-1)/2) of w keys by one warp: MSD radix select with
// 8-bit digits over the bits where the keys differ (histogram of 256 words
// owned by the warp), the keys read on every pass from global memory (raw
// float bits, turned into order keys), 8 loads per lane issued together, or
// from a shared-memory copy (order keys already).
template <bool kGlobal>
__device__ uint32_t warp_select_stream(const uint32_t* keys, uint32_t w, uint32_t* hist) {
  constexpr int U = 8;
  const int lane = threadIdx.x & 31;
  auto load = [&](uint32_t i) -> uint32_t { return kGlobal ? kload(keys + i) : keys[i]; };
  uint32_t lo = 0xffffffffu, hi = 0u;
  for (uint32_t b0 = 0; b0 < w; b0 += 32 * U) {
    uint32_t x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = b0 + (uint32_t)(u * 32 + lane);
      x[u] = i < w ? load(i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (b0 + (uint32_t)(u * 32 + lane) < w) {
        lo = min(lo, x[u]);
        hi = max(hi, x[u]);
      }
  }
  RadixState st;
  if (!radix_start(lo, hi, (w - 1) / 2, &st)) return st.prefix;
  while (st.rem > 0) {
    const int bits = st.rem < 8 ? st.rem : 8, shift = st.rem - bits;
    const uint32_t nb = 1u << bits, hmask = st.rem == 32 ? 0u : ~((1u << st.rem) - 1u);
    for (uint32_t i = lane; i < nb; i += 32) hist[i] = 0;
    __syncwarp();
    for (uint32_t b0 = 0; b0 < w; b0 += 32 * U) {
      uint32_t x[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = b0 + (uint32_t)(u * 32 + lane);
        x[u] = i < w ? load(i) : 0u;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (b0 + (uint32_t)(u * 32 + lane) < w && (x[u] & hmask) == st.prefix)
          atomicAdd(&hist[(x[u] >> shift) & (nb - 1u)], 1u);
    }
    __syncwarp();
    uint32_t below;
    const uint32_t digit = warp_find_digit_n(hist, nb, st.rank, &below);
    st.rank -= below;
    st.prefix |= digit << shift;
    st.rem = shift;
    __syncwarp();
  }
  return st.prefix;
}

// One warp per listed segment of tiny_max+1 .. warp_max points: up to
// bitonic_max keys sorted in registers; up to 1024 keys staged once in shared
// memory for a radix select; larger segments read from global memory on every
// pass.
__global__ void __launch_bounds__(256) k_select_small(const TreeDev* trees, StepDev s) {
  __shared__ uint32_t hist[8][256];
  __shared__ uint32_t stage[8][1024];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t cnt = min(*s.midseg_count, s.midseg_cap);
  for (uint32_t j = blockIdx.x * 8u + (uint32_t)warp; j < cnt; j += gridDim.x * 8u) {
    const uint32_t g = s.midseg[j];
    const uint32_t w = s.seg_w[g];
    const uint32_t* keys = s.seg_key[g];
    uint32_t med;
    if (w <= s.bitonic_max && w <= 64u) {
      med = warp_bitonic_median<2>(keys, w);
    } else if (w <= s.bitonic_max && w <= 128u) {
      med = warp_bitonic_median<4>(keys, w);
    } else if (w <= s.bitonic_max) {
      med = warp_bitonic_median<8>(keys, w);
    } else if (w <= 1024u) {
      uint32_t* st = stage[warp];
      for (uint32_t b0 = 0; b0 < w; b0 += 256) {
        uint32_t x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const uint32_t i = b0 + (uint32_t)(u * 32 + lane);
          x[u] = i < w ? kload(keys + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const uint32_t i = b0 + (uint32_t)(u * 32 + lane);
          if (i < w) st[i] = x[u];
        }
      }
      __syncwarp();
      med = warp_select_stream<false>(st, w, hist[warp]);
    } else {
      med = warp_select_stream<true>(keys, w, hist[warp]);
    }
    if (lane == 0) s.seg_med[g] = med;
    __syncwarp();
  }
}

// CTAs of kThreads stride over the listed segments above the warp-select
// size: MSD radix select with kBits-bit digits (8: four passes, one histogram
// per warp, which suits the few bins that the top digits of clustered data
// fall into; 11: three passes over a CTA-wide 2048-bin histogram), keys read
// from global memory 16 bytes at a time (the unaligned head and tail of the
// segment by single words).
template <int kThreads, int kBits>
__global__ void __launch_bounds__(kThreads) k_select_big(const TreeDev* trees, StepDev s) {
  constexpr int kW = kThreads / 32;
  constexpr bool kWarpHist = kBits == 8;
  constexpr int kBins = 1 << kBits;
  constexpr int kHist = kWarpHist ? kW * kBins : kBins;
  constexpr int kPer = kBins >= kThreads ? kBins / kThreads : 1;  // bins per thread in the digit search
  __shared__ uint32_t hist[kHist];
  __shared__ uint32_t tot_w[kWarpHist ? kBins : 1];
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t bcast[2];
  const int warp = threadIdx.x >> 5;
  uint32_t* tot = kWarpHist ? tot_w : hist;
  const uint32_t cnt = min(*s.bigseg_count, s.bigseg_cap);
  for (uint32_t jb = blockIdx.x; jb < cnt; jb += gridDim.x) {
    const uint32_t g = s.bigseg[jb];
    const uint32_t w = s.seg_w[g];
    const uint32_t* keys = s.seg_key[g];
    const uint32_t head = min(w, (4u - (uint32_t)(((uintptr_t)keys >> 2) & 3u)) & 3u);
    const uint4* kv = (const uint4*)(keys + head);  // 16-byte aligned
    const uint32_t nv = (w - head) >> 2, tail0 = head + nv * 4u;
    uint32_t rank = (w - 1) / 2, prefix = 0;
    for (int top = 32; top > 0;) {  // bits [top, 32) are known
      const int bits = top < kBits ? top : kBits, shift = top - bits;
      const uint32_t mask = top == 32 ? 0u : ~((1u << top) - 1u), nb = 1u << bits;
      for (int i = threadIdx.x; i < kHist; i += kThreads) hist[i] = 0;
      __syncthreads();
      uint32_t* wh = kWarpHist ? hist + warp * kBins : hist;
      auto add = [&](uint32_t u) {
        const uint32_t k = ord_key(__uint_as_float(u));
        if ((k & mask) == prefix) atomicAdd(&wh[(k >> shift) & (nb - 1u)], 1u);
      };
      uint32_t v = threadIdx.x;
      for (; v + 3 * kThreads < nv; v += 4 * kThreads) {
        uint4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = __ldg(kv + v + u * kThreads);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          add(q[u].x);
          add(q[u].y);
          add(q[u].z);
          add(q[u].w);
        }
      }
      for (; v < nv; v += kThreads) {
        const uint4 q = __ldg(kv + v);
        add(q.x);
        add(q.y);
        add(q.z);
        add(q.w);
      }
      if (threadIdx.x < head) add(__ldg(keys + threadIdx.x));
      if (threadIdx.x < w - tail0) add(__ldg(keys + tail0 + threadIdx.x));
      __syncthreads();
      if (kWarpHist) {
        for (int b = threadIdx.x; b < kBins; b += kThreads) {
          uint32_t sum = 0;
#pragma unroll
          for (int q = 0; q < kW; ++q) sum += hist[q * kBins + b];
          tot[b] = sum;
        }
        __syncthreads();
      }
      // the bin holding `rank`: each thread scans kPer consecutive bins
      const uint32_t first = (uint32_t)threadIdx.x * kPer;
      uint32_t loc[kPer], sum = 0;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        loc[q] = first + q < nb ? tot[first + q] : 0u;
        sum += loc[q];
      }
      uint32_t all;
      const uint32_t ex = block_excl_scan(sum, tmp, &all);
      if (rank >= ex && rank < ex + sum) {
        uint32_t acc = ex;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          if (rank < acc + loc[q]) {
            bcast[0] = first + q;
            bcast[1] = acc;
            break;
          }
          acc += loc[q];
        }
      }
      __syncthreads();
      rank -= bcast[1];
      prefix |= bcast[0] << shift;
      top = shift;
      __syncthreads();
    }
    if (threadIdx.x == 0) s.seg_med[g] = prefix;
  }
}

// One CTA per cell: count-weighted lower median of the segment medians: the
// smallest median m whose segments with median <= m hold at least
// ceil(W/2) of the W points (weighted 8-bit MSD radix select).
__device__ __forceinline__ void combine_cell(const TreeDev* trees, const StepDev& s, uint32_t c) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t bcast[2];
  const Cell cell = s.cells[c];
  const TreeDev& t = trees[cell.tree];
  const int r = t.r;
  const uint32_t g0 = s.seg_base[c];
  const bool unit = t.combine_rule == 1;  // every non-empty subset counts once
  uint32_t rank = (cell_weight(s, c, cell) - 1) / 2, prefix = 0, mask = 0;
  if (unit) {  // rank (m - 1) / 2 among the m non-empty segments
    if (threadIdx.x == 0) bcast[0] = 0;
    __syncthreads();
    uint32_t m = 0;
    for (int j = threadIdx.x; j < r; j += blockDim.x) m += s.seg_w[g0 + j] != 0u;
    m = warp_sum(m);
    if ((threadIdx.x & 31) == 0) atomicAdd(&bcast[0], m);
    __syncthreads();
    rank = (bcast[0] - 1u) / 2u;
    __syncthreads();
  }
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
      const uint32_t w = s.seg_w[g0 + j];
      if (!w) continue;
      const uint32_t k = s.seg_med[g0 + j];
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], unit ? 1u : w);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t below;
      const uint32_t digit = warp_find_digit(hist, rank, &below);
      if (threadIdx.x == 0) {
        bcast[0] = digit;
        bcast[1] = below;
      }
    }
    __syncthreads();
    rank -= bcast[1];
    prefix |= bcast[0] << shift;
    mask |= 255u << shift;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    s.mkey[c] = prefix;
    t.out_vals[cell.heap] = key_float(prefix);
    t.out_dims[cell.heap] = (int8_t)s.kdim[c];
  }
}

__global__ void __launch_bounds__(256) k_combine(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  for (uint32_t c = blockIdx.x; c < nc; c += gridDim.x) {
    combine_cell(trees, s, c);
    __syncthreads();  // the cell's shared memory is free for the next one
  }
}

// One warp per cell (steps with many cells): the same weighted lower median
// by the warp radix select, which starts at the first bit where the cell's
// segment medians differ.
__device__ __forceinline__ void combine_warp_cell(const TreeDev* trees, const StepDev& s, uint32_t c) {
  __shared__ uint32_t hist[8][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Cell cell = s.cells[c];
  const TreeDev& t = trees[cell.tree];
  const uint32_t g0 = s.seg_base[c];
  const uint32_t* med = s.seg_med + g0;
  const uint32_t* wt = s.seg_w + g0;
  const bool unit = t.combine_rule == 1;  // every non-empty subset counts once
  uint32_t rank = (cell_weight(s, c, cell) - 1) / 2;
  if (unit) {
    uint32_t nz = 0;
    for (uint32_t j = lane; j < (uint32_t)t.r; j += 32) nz += wt[j] != 0u;
    rank = (warp_sum(nz) - 1u) / 2u;
  }
  const uint32_t m = warp_weighted_select(
      (uint32_t)t.r, rank, hist[warp], [&](uint32_t j) { return med[j]; },
      [&](uint32_t j) { return unit ? 1u : wt[j]; }, [&](uint32_t j) { return wt[j] != 0u; });
  if (lane == 0) {
    s.mkey[c] = m;
    t.out_vals[cell.heap] = key_float(m);
    t.out_dims[cell.heap] = (int8_t)s.kdim[c];
  }
}

__global__ void __launch_bounds__(256, 1) k_combine_warp(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  for (uint32_t c = blockIdx.x * 8u + (threadIdx.x >> 5); c < nc; c += gridDim.x * 8u) combine_warp_cell(trees, s, c);
}

// ------------------------------------------- the paper's estimator (Sec. 3)

constexpr int kFourierTerms = 2 * KDT_FOURIER_MAX_J + 1;
constexpr int kTileRecWords = 2 * kMaxDims * 2;  // words of a tile's record in tile_mm
static_assert(kFourierTerms * 2 <= kTileRecWords, "a tile's sums fit its record");

// The sums over a cell's points of the basis terms of Lemma 1 on its key
// coordinate, c_0 = 1, c_{2j-1} = cos((2j-1)x), c_{2j} = sin((2j-1)x) for
// j = 1..J (the additive statistics of Sec. 3.2). The kernel is persistent:
// CTA k takes the tiles [k T / G, (k+1) T / G) of the step (T tiles, G
// CTAs). Each thread holds 8 points of a tile and runs the odd harmonics
// for all of them at once (h(k+2) = 2 cos(2x) h(k) - h(k-2), from one sincosf
// per point), adding each harmonic's terms in float, then over the warp by
// a shuffle tree in float (double arithmetic is scarce on this GPU); the CTA
// adds the warps' sums in double in a fixed order into a running total per
// term, written to the record of the run's first tile when the
// CTA's run of the cell's tiles ends. The split kernel adds a cell's run
// records in order, so the result does not depend on scheduling. A
// coordinate outside (0,1) is reported.
__global__ void __launch_bounds__(256, 2) k_fourier_moments(const TreeDev* trees, StepDev s) {
  constexpr int kPer = kTile / 256;
  __shared__ float red[8][kFourierTerms];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ntiles = *s.ntiles_total;
  const uint32_t t_begin = (uint32_t)(((uint64_t)blockIdx.x * ntiles) / gridDim.x);
  const uint32_t t_end = (uint32_t)(((uint64_t)(blockIdx.x + 1) * ntiles) / gridDim.x);
  // a tile's record, cell and this thread's points (loaded one tile ahead)
  struct Ahead {
    uint2 tl;
    int32_t tree;
    uint32_t end;
    float x[kPer];
  };
  auto fetch = [&](uint32_t tile, Ahead& a) {
    a.tl = s.tiles[tile];
    const Cell cell = s.cells[a.tl.x];
    const TreeDev& t = trees[cell.tree];
    const float* X = (const float*)key_column(t, cell, s.kdim[a.tl.x]) + cell.begin;
    a.tree = cell.tree;
    a.end = min(a.tl.y + (uint32_t)kTile, cell.count);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const uint32_t i = a.tl.y + threadIdx.x + 256u * q;
      a.x[q] = i < a.end ? __ldg(X + i) : 0.5f;
    }
  };
  double run = 0.0;  // thread j: term j of the current run
  uint32_t run_first = t_begin;
  Ahead cur, nxt;
  if (t_begin < t_end) fetch(t_begin, cur);
  for (uint32_t tile = t_begin; tile < t_end; ++tile) {
    if (tile + 1 < t_end) fetch(tile + 1, nxt);  // in flight while this tile is summed
    const TreeDev& t = trees[cur.tree];
    const int J = t.fourier_j;
    float c2[kPer], cp[kPer], sp[kPer], cc[kPer], sc[kPer];
    bool outside = false, nan = false;
    uint32_t cnt = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const uint32_t i = cur.tl.y + threadIdx.x + 256u * q;
      const bool ok = i < cur.end;
      const float x = cur.x[q];
      nan |= ok && x != x;
      outside |= ok && !(x > 0.f && x < 1.f);
      float sx, cx;
      sincosf(x, &sx, &cx);
      const float w = ok ? 1.f : 0.f;  // a missing point adds nothing
      c2[q] = 2.f * (cx * cx - sx * sx);
      cp[q] = w * cx;  // harmonic -1
      sp[q] = -w * sx;
      cc[q] = w * cx;  // harmonic 1
      sc[q] = w * sx;
      cnt += ok ? 1u : 0u;
    }
    if (outside) set_status(t, nan ? ST_NAN_INPUT : ST_INVALID_ARG);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) red[warp][0] = (float)cnt;
    for (int k = 1; k <= J; ++k) {
      float ac = 0.f, as = 0.f;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        ac += cc[q];
        as += sc[q];
        const float cn = fmaf(c2[q], cc[q], -cp[q]), sn = fmaf(c2[q], sc[q], -sp[q]);
        cp[q] = cc[q];
        sp[q] = sc[q];
        cc[q] = cn;
        sc[q] = sn;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ac += __shfl_down_sync(0xffffffffu, ac, o);
        as += __shfl_down_sync(0xffffffffu, as, o);
      }
      if (lane == 0) {
        red[warp][2 * k - 1] = ac;
        red[warp][2 * k] = as;
      }
    }
    __syncthreads();
    if ((int)threadIdx.x <= 2 * J) {
      double v = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) v += (double)red[w][threadIdx.x];
      run += v;
    }
    // the CTA's run of this cell's tiles ends here: write its record
    if (tile + 1 == t_end || nxt.tl.x != cur.tl.x) {
      if ((int)threadIdx.x <= 2 * J) ((double*)(s.tile_mm + (size_t)run_first * kTileRecWords))[threadIdx.x] = run;
      run = 0.0;
      run_first = tile + 1;
    }
    __syncthreads();
    cur = nxt;
  }
}

// Per cell, one warp: the cell's sums C_j (its tiles' records added in tile
// order; lane l holds terms l, l + 32, l + 64), its bounds (a, b) on its key
// coordinate (the splits of its ancestors on that coordinate, (0,1) at the
// root), and the root of Eq. (kd:eq:b) by 60 bisection steps in double on
// (a, b) of F(m) = 1_J(a, m) - 1_J(m, b) = sum_j C_j (g_j(a, m) - g_j(m, b)),
// with g_j of Lemma 1: the term of j = 0 is (1(b<1) - 1(a>0)) / 2, of
// j = 2k-1 q (2 sin(Km) - 1(a>0) sin(Ka) - 1(b<1) sin(Kb)) and of j = 2k
// q (1(a>0) cos(Ka) + 1(b<1) cos(Kb) - 2 cos(Km)), K = 2k-1, q = 2 / (pi K).
// The lower end moves up while F < 0; the split is the last midpoint
// rounded to float, and a point goes left when its coordinate is <= it. The
// harmonics of the midpoint are evaluated in float (their error moves the
// root by about 1e-7 of the cell's width), the sums in double.
__global__ void __launch_bounds__(256) k_fourier_split(const TreeDev* trees, StepDev s, uint32_t mgrid) {
  const int lane = threadIdx.x & 31;
  const uint32_t nc = ncells_of(s);
  const uint32_t ntiles = *s.ntiles_total;
  auto range_start = [&](uint32_t k) { return (uint32_t)(((uint64_t)k * ntiles) / mgrid); };
  for (uint32_t c = blockIdx.x * 8u + (threadIdx.x >> 5); c < nc; c += gridDim.x * 8u) {
    const Cell cell = s.cells[c];
    const TreeDev& t = trees[cell.tree];
    const int nt = 2 * t.fourier_j + 1;
    const uint32_t tb = s.tile_base[c], te = s.tile_base[c + 1];
    // the moments kernel's runs of this cell start at tb and at every start
    // of a CTA's tile range inside (tb, te)
    uint64_t k0 = ((uint64_t)tb * mgrid) / (ntiles > 0u ? ntiles : 1u);
    uint32_t k = (uint32_t)(k0 < (uint64_t)mgrid ? k0 : (uint64_t)(mgrid - 1u));
    while (k > 0u && range_start(k) > tb) --k;
    while (k + 1u < mgrid && range_start(k + 1u) <= tb) ++k;
    double C[3] = {0.0, 0.0, 0.0};
    uint32_t r0 = tb;
    for (uint32_t kk = k + 1u;; ++kk) {
      const double* rec = (const double*)(s.tile_mm + (size_t)r0 * kTileRecWords);
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (lane + 32 * q < nt) C[q] += rec[lane + 32 * q];
      uint32_t nxt = te;
      while (kk < mgrid && (nxt = range_start(kk)) <= r0) ++kk;  // CTAs with empty ranges
      if (kk >= mgrid || nxt >= te) break;
      r0 = nxt;
    }
    const uint32_t dim = s.kdim[c];
    double a = 0.0, b = 1.0;
    if (lane == 0)
      for (uint32_t h = cell.heap; h > 0;) {
        const uint32_t par = (h - 1u) / 2u;
        const uint32_t plevel = 31u - (uint32_t)__clz(par + 1u);
        if (plevel % (uint32_t)t.d == dim) {
          const double v = (double)t.out_vals[par];
          if (h == 2u * par + 1u)
            b = fmin(b, v);
          else
            a = fmax(a, v);
        }
        h = par;
      }
    a = __shfl_sync(0xffffffffu, a, 0);
    b = __shfl_sync(0xffffffffu, b, 0);
    const double ia = a > 0.0 ? 1.0 : 0.0, ib = b < 1.0 ? 1.0 : 0.0;
    // per term: F_j(m) = base + slope * (sin or cos)(K m)
    double base[3], slope[3], K[3];
    bool use_sin[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int j = lane + 32 * q;
      base[q] = slope[q] = 0.0;
      K[q] = 0.0;
      use_sin[q] = true;
      if (j >= nt) continue;
      if (j == 0) {
        base[q] = C[q] * 0.5 * (ib - ia);
        continue;
      }
      const double k = (double)(2 * ((j + 1) / 2) - 1);
      const double qk = 2.0 / (3.14159265358979323846 * k);
      K[q] = k;
      if (j & 1) {
        base[q] = -C[q] * qk * (ia * sin(k * a) + ib * sin(k * b));
        slope[q] = 2.0 * C[q] * qk;
      } else {
        base[q] = C[q] * qk * (ia * cos(k * a) + ib * cos(k * b));
        slope[q] = -2.0 * C[q] * qk;
        use_sin[q] = false;
      }
    }
    double lo = a, hi = b;
    for (int it = 0; it < 60; ++it) {
      const double mid = 0.5 * (lo + hi);
      double f = 0.0;
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (slope[q] != 0.0 || base[q] != 0.0)
          f += base[q] + (slope[q] != 0.0
                              ? slope[q] * (double)(use_sin[q] ? sinf((float)(K[q] * mid)) : cosf((float)(K[q] * mid)))
                              : 0.0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
      f = __shfl_sync(0xffffffffu, f, 0);  // lane 0's sum decides for the warp
      if (f < 0.0)
        lo = mid;
      else
        hi = mid;
    }
    if (lane == 0) {
      const float m32 = (float)(0.5 * (lo + hi));
      s.mkey[c] = ord_key(m32);
      t.out_vals[cell.heap] = m32;
      t.out_dims[cell.heap] = (int8_t)dim;
    }
  }
}

// ------------------------------------------------------------ partition

// Per tile: number of points with key <= split. One warp per tile: the
// tile's key range is read 16 bytes at a time with all of a lane's loads in
// flight together (its unaligned head and tail by single words).
__device__ __forceinline__ void part_count_tile(const TreeDev* trees, const StepDev& s, uint32_t tile, uint2 tl) {
  constexpr int kV = kTile / 4 / 32;  // 16-byte vectors per lane of a full tile
  const int lane = threadIdx.x & 31;
  const Cell cell = s.cells[tl.x];
  const TreeDev& t = trees[cell.tree];
  const float* X = src_cols(t, cell.level) + (int64_t)s.kdim[tl.x] * t.n + cell.begin + tl.y;
  const uint32_t m = s.mkey[tl.x];
  const uint32_t cnt_pts = min((uint32_t)kTile, cell.count - tl.y);
  const uint32_t head = min(cnt_pts, (4u - (uint32_t)(((uintptr_t)X >> 2) & 3u)) & 3u);
  const uint32_t nv = (cnt_pts - head) >> 2, tail0 = head + nv * 4u;
  const float4* xv = (const float4*)(X + head);  // 16-byte aligned
  float4 v[kV];
#pragma unroll
  for (int q = 0; q < kV; ++q) {
    const uint32_t i = (uint32_t)(lane + q * 32);
    v[q] = i < nv ? __ldg(xv + i) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  uint32_t cnt = 0;
#pragma unroll
  for (int q = 0; q < kV; ++q)
    if ((uint32_t)(lane + q * 32) < nv)
      cnt += (ord_key(v[q].x) <= m) + (ord_key(v[q].y) <= m) + (ord_key(v[q].z) <= m) + (ord_key(v[q].w) <= m);
  if ((uint32_t)lane < head) cnt += ord_key(__ldg(X + lane)) <= m;
  if ((uint32_t)lane < cnt_pts - tail0) cnt += ord_key(__ldg(X + tail0 + lane)) <= m;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) s.tile_left[tile] = cnt;
}

// Warps stride over the tiles; three CTAs per SM by a register bound (80
// registers: a lane's sixteen 16-byte loads still fit, with a few words of
// spill).
__global__ void __launch_bounds__(256, 3) k_part_count(const TreeDev* trees, StepDev s) {
  const uint32_t ntiles = *s.ntiles_total;
  for (uint32_t tile = blockIdx.x * 8u + (threadIdx.x >> 5); tile < ntiles; tile += gridDim.x * 8u)
    part_count_tile(trees, s, tile, s.tiles[tile]);
}

// One CTA per cell: exclusive scan of its tiles' left counts.
__device__ __forceinline__ void part_scan_cell(const StepDev& s, uint32_t c) {
  __shared__ uint32_t tmp[33];
  const uint32_t tb = s.tile_base[c], te = s.tile_base[c + 1];
  uint32_t run = 0;
  for (uint32_t j0 = tb; j0 < te; j0 += blockDim.x) {
    const uint32_t j = j0 + threadIdx.x;
    const uint32_t v = j < te ? s.tile_left[j] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, tmp, &tot);
    if (j < te) s.tile_loff[j] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) s.lcount[c] = run;
}

__global__ void k_part_scan(StepDev s) {
  const uint32_t nc = ncells_of(s);
  for (uint32_t c = blockIdx.x; c < nc; c += gridDim.x) {
    part_scan_cell(s, c);
    __syncthreads();  // the cell's shared memory is free for the next one
  }
}

// One warp per cell (steps with many cells, few tiles each).
__device__ __forceinline__ void part_scan_warp_cell(const StepDev& s, uint32_t c) {
  const int lane = threadIdx.x & 31;
  const uint32_t tb = s.tile_base[c], te = s.tile_base[c + 1];
  uint32_t run = 0;
  for (uint32_t j0 = tb; j0 < te; j0 += 32) {
    const uint32_t j = j0 + (uint32_t)lane;
    const uint32_t v = j < te ? s.tile_left[j] : 0u;
    const uint32_t inc = warp_incl_scan(v);
    if (j < te) s.tile_loff[j] = run + inc - v;
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (lane == 0) s.lcount[c] = run;
}

__global__ void __launch_bounds__(256) k_part_scan_warp(StepDev s) {
  const uint32_t nc = ncells_of(s);
  for (uint32_t c = blockIdx.x * 8u + (threadIdx.x >> 5); c < nc; c += gridDim.x * 8u) part_scan_warp_cell(s, c);
}

// One warp per cell (widest spread): the key coordinate of each big child,
// and of each child queued for the subtree kernel (its first level), from its
// min and max key per coordinate (reduced by the scatter): the
// largest range (double)max - (double)min, 0 for equal keys, lowest
// coordinate on ties. A range is never negative, so the bit patterns of two
// ranges order like the ranges as unsigned integers: the argmax runs on the
// high word, then the low word, then the lowest coordinate, by integer warp
// reductions (double arithmetic, slow on this part, only for the one
// subtraction per range).
__device__ __forceinline__ void child_dims_cell(const TreeDev* trees, const StepDev& s, uint32_t c) {
  const int lane = threadIdx.x & 31;
  const Cell cell = s.cells[c];
  const TreeDev& t = trees[cell.tree];
  if (t.key_rule != KEY_WIDEST) return;
  const int d = t.d;
  for (int side = 0; side < 2; ++side) {
    const uint2 cr = s.crow[2 * c + side];
    if (cr.x == kNoRow && cr.y == kNoRow) continue;  // terminal
    uint64_t rb = 0ull;
    uint32_t ib = 0xffffffffu;
    for (int l = lane; l < d; l += 32) {  // l ascending: the first of equal ranges is kept
      const uint2 mm = *(const uint2*)&s.child_mm[(((size_t)c * 2 + side) * kMaxDims + l) * 2];
      const uint64_t range = (uint64_t)__double_as_longlong(key_range(mm.x, mm.y));
      if (ib == 0xffffffffu || range > rb) {
        rb = range;
        ib = (uint32_t)l;
      }
    }
    const uint32_t rh = (uint32_t)(rb >> 32), rl = (uint32_t)rb;
    const uint32_t mh = __reduce_max_sync(0xffffffffu, ib != 0xffffffffu ? rh : 0u);
    const uint32_t ml = __reduce_max_sync(0xffffffffu, (ib != 0xffffffffu && rh == mh) ? rl : 0u);
    ib = __reduce_min_sync(0xffffffffu, (ib != 0xffffffffu && rh == mh && rl == ml) ? ib : 0xffffffffu);
    if (lane == 0) {
      if (cr.x != kNoRow)
        s.next_big[cr.x].dim = (int16_t)ib;
      else
        s.small[cr.y].dim = (int16_t)ib;  // the subtree kernel's first level
    }
  }
}

__global__ void __launch_bounds__(256, 1) k_child_dims(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  for (uint32_t c = blockIdx.x * 8u + (threadIdx.x >> 5); c < nc; c += gridDim.x * 8u) child_dims_cell(trees, s, c);
}

// ------------------------------------------------------------- children

// One thread per cell, after the children's sizes are known and before the
// move: terminal children are recorded, small ones queued for the subtree
// kernel, big ones get a slot of the next step and a row of its subset
// offsets (which the scatter fills).
__device__ __forceinline__ void classify_cell(const TreeDev* trees, const StepDev& s, uint32_t c) {
  const Cell cell = s.cells[c];
  const TreeDev& t = trees[cell.tree];
  const uint32_t L = s.lcount[c], R = cell.count - L;
  const int level = cell.level + 1;
  const int stall = (R == 0) ? cell.stall + 1 : 0;
  const uint32_t cb[2] = {cell.begin, cell.begin + L};
  const uint32_t cc[2] = {L, R};
  int live_delta = -1;  // this cell is done; each child that still needs splitting adds one
  if (t.key_rule == KEY_WIDEST)  // identities for the scatter's min / max reductions
    for (int j = 0; j < 4 * t.d; ++j) {
      const int side = j / (2 * t.d), l = (j / 2) % t.d, which = j & 1;
      s.child_mm[(((size_t)c * 2 + side) * kMaxDims + l) * 2 + which] = which ? 0u : 0xffffffffu;
    }
  for (int side = 0; side < 2; ++side) {
    uint2 cr = make_uint2(kNoRow, kNoRow);
    const uint32_t heap = 2u * cell.heap + 1u + (uint32_t)side;
    if (is_terminal(t, cc[side], level, stall)) {
      record_terminal(t, cb[side], cc[side], heap, level);
    } else if (t.depth == 0 && level >= t.max_levels) {
      set_status(t, ST_LEVEL_CAP);
    } else {
      ++live_delta;
      const Cell child{cb[side], cc[side], heap, cell.tree, (int8_t)level, (int8_t)stall, (int16_t)-1};
      if (cc[side] <= (uint32_t)t.small_max) {
        if (atomicAdd(s.small_total, 1u) < s.small_cap) {
          // the two ends of the queue never meet: at most small_cap cells get a slot
          const uint32_t slot = t.sub_wide ? s.small_cap - 1u - atomicAdd(s.small_count_w, 1u)
                                           : atomicAdd(s.small_count, 1u);
          s.small[slot] = child;
          cr = make_uint2(kNoRow, slot);  // its widest coordinate is picked with the big children's
        } else {
          set_status(t, ST_CAPACITY);
        }
        atomicAdd(s.small_points, cc[side]);
      } else {
        const uint32_t slot = atomicAdd(s.next_big_count, 1u);
        const uint32_t row = atomicAdd(s.off_used, (uint32_t)t.r + 1u);
        if (slot < s.next_big_cap && row <= s.off_cap - ((uint32_t)t.r + 1u)) {
          s.next_big[slot] = child;
          s.obase_next[slot] = row;
          cr = make_uint2(slot, row);
        } else {
          set_status(t, ST_CAPACITY);
        }
        atomicAdd(s.next_big_points, cc[side]);
      }
    }
    s.crow[2 * c + side] = cr;
  }
  if (live_delta) atomicAdd(t.live, live_delta);
}

__global__ void k_classify(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
    classify_cell(trees, s, c);
}

}  // namespace

// ------------------------------------------------------------ launcher

constexpr uint32_t kManyCells = 1024;  // from here on: a warp per cell in combine and scan

cudaError_t prepare_step_kernels() {
  return cudaFuncSetAttribute(k_ps_move, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPsSmemBytes);
}

void launch_big_step(const TreeDev* trees, const StepDev& s, uint32_t max_tiles, uint32_t nseg,
                     uint32_t max_bigseg, bool has_roots, bool need_root_dims, bool any_widest, int max_d, int uniform_d,
                     const SelectTuning& tune, uint64_t points, uint32_t sms, cudaStream_t st, bool fourier) {
  // s.ncells: the step's cells, or (s.ncells_dev set: a step inside a graph)
  // their capacity; per-cell kernels stride over the cells, so their grids
  // cover the cells exactly here and are capped there
  const uint32_t nc = s.ncells;
  if (nc == 0) return;
  const bool dev = s.ncells_dev != nullptr;
  auto cells_grid = [&](uint32_t per_block, uint32_t cap) {
    const uint32_t g = (nc + per_block - 1) / per_block;
    return std::max<uint32_t>(1, dev ? std::min(g, cap) : g);
  };
  { TraceScope ts(K_PREP, st); k_prep<<<1, 1024, 0, st>>>(trees, s); }
  { TraceScope ts(K_TILES, st); k_tiles<<<cells_grid(8, sms * 8u), 256, 0, st>>>(trees, s); }
  if (s.shards) launch_shard_index(s, nc, st);
  if (has_roots) {
    {
      TraceScope ts(K_PS_COUNT, st, points);
      k_ps_count<<<std::max<uint32_t>(1, std::min(max_tiles, sms * 4u)), kTileThreads, 0, st>>>(trees, s);
    }
    { TraceScope ts(K_PS_OFFSETS, st); k_ps_offsets<<<nc, 1024, 0, st>>>(trees, s); }
    { TraceScope ts(K_PS_MOVE, st, points); k_ps_move<<<max_tiles, kPsThreads, kPsSmemBytes, st>>>(trees, s); }
  }
  if (need_root_dims) {
    { TraceScope ts(K_MINMAX, st, points); k_minmax<<<max_tiles, kTileThreads, 0, st>>>(trees, s); }
    { TraceScope ts(K_PICK_DIM, st); k_pick_dim<<<nc, 1024, 0, st>>>(trees, s); }
  }
  // a CTA per cell while cells are few (large subset counts, deep scans),
  // a warp per cell once they are many (and in a graph, where the count is
  // not known when the launch is recorded)
  const bool many = dev || nc >= kManyCells;
  if (fourier) {  // the paper's estimator: per-run sums, then the root per cell
    const uint32_t mgrid = std::max<uint32_t>(1, std::min(max_tiles, sms * 2u));
    {
      TraceScope ts(K_FOURIER_MOMENTS, st, points);
      k_fourier_moments<<<mgrid, 256, 0, st>>>(trees, s);
    }
    { TraceScope ts(K_FOURIER_SPLIT, st); k_fourier_split<<<cells_grid(8, sms * 8u), 256, 0, st>>>(trees, s, mgrid); }
  } else {
    { TraceScope ts(K_SEGS, st); k_segs<<<cells_grid(1, sms * 8u), 256, 0, st>>>(trees, s); }
    {
      TraceScope ts(K_SELECT_TINY, st, points);
      k_select_tiny<<<std::max<uint32_t>(1, std::min<uint32_t>((nseg + 255) / 256, sms * 16u)), 256, 0, st>>>(trees, s);
    }
    {
      TraceScope ts(K_SELECT_SMALL, st, points);
      k_select_small<<<std::max<uint32_t>(1, std::min<uint32_t>((nseg + 7) / 8, sms * 8u)), 256, 0, st>>>(trees, s);
    }
    if (max_bigseg) {
      TraceScope ts(K_SELECT_BIG, st);
      // nseg bounds the big segments too; with few of them (the first levels
      // of a large tree) a CTA's loads in flight set the rate, so they take
      // 512 threads whatever the tuning
      const uint32_t grid = std::max<uint32_t>(1, std::min<uint32_t>(std::min(max_bigseg, nseg), sms * 4u));
      if (tune.cta_threads == 512 || nseg <= sms * 4u) {
        if (tune.digit_bits == 8)
          k_select_big<512, 8><<<grid, 512, 0, st>>>(trees, s);
        else
          k_select_big<512, 11><<<grid, 512, 0, st>>>(trees, s);
      } else {
        if (tune.digit_bits == 8)
          k_select_big<256, 8><<<grid, 256, 0, st>>>(trees, s);
        else
          k_select_big<256, 11><<<grid, 256, 0, st>>>(trees, s);
      }
    }
    if (s.shards) launch_shard_medians(trees, s, nc, st);  // the all-gather of the segment statistics
    {
      TraceScope ts(K_COMBINE, st);
      if (many)
        k_combine_warp<<<cells_grid(8, sms * 8u), 256, 0, st>>>(trees, s);
      else
        k_combine<<<nc, 256, 0, st>>>(trees, s);
    }
  }
  {
    TraceScope ts(K_PART_COUNT, st, points);
    k_part_count<<<std::max<uint32_t>(1, std::min((max_tiles + 7) / 8, sms * 16u)), 256, 0, st>>>(trees, s);
  }
  {
    TraceScope ts(K_PART_SCAN, st);
    if (many)
      k_part_scan_warp<<<cells_grid(8, sms * 8u), 256, 0, st>>>(s);
    else
      k_part_scan<<<nc, 1024, 0, st>>>(s);
  }
  { TraceScope ts(K_CLASSIFY, st); k_classify<<<cells_grid(256, sms * 4u), 256, 0, st>>>(trees, s); }
  launch_scatter(trees, s, max_tiles, 2 * sms, points, uniform_d, st);
  if (any_widest && s.shards) launch_shard_minmax(trees, s, nc, st);
  if (any_widest) {
    TraceScope ts(K_CHILD_DIMS, st);
    k_child_dims<<<cells_grid(8, sms * 8u), 256, 0, st>>>(trees, s);
  }
}

namespace {

// Last node of a graph's loop body: count the iteration and keep looping
// while the next step has cells (at most `limit` iterations).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const uint32_t* ncells_next, uint32_t* iters,
                            uint32_t limit) {
  const uint32_t it = *iters + 1u;
  *iters = it;
  cudaGraphSetConditional(h, (*ncells_next > 0u && it < limit) ? 1u : 0u);
}

}  // namespace

void launch_loop_cond(cudaGraphConditionalHandle h, const uint32_t* ncells_next, uint32_t* iters, uint32_t limit,
                      cudaStream_t st) {
  k_loop_cond<<<1, 1, 0, st>>>(h, ncells_next, iters, limit);
}

}  // namespace kdt
