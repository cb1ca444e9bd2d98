// kdt_step.cu -- one level of the multi-CTA pipeline for cells too large to
// finish in shared memory.
//
// For every big cell c of the step (paper, Sec. 2: a level splits each of its
// cells along the key coordinate t at a median):
//   1. key coordinate: cyclic (Sec. 1) or widest range (Sec. 1, Friedman rule)
//   2. per (cell, subset) segment: count, then the keys grouped by segment
//      into a scratch array (the subsets of Sec. 3.2 / App. C.2)
//   3. per segment: the exact lower median (8-bit MSD radix select)
//   4. per cell: the count-weighted lower median of the segment medians
//   5. stable partition of all d columns, the permutation and the subset ids
//      around the split (key <= split to the left), via per-tile counts and a
//      per-cell scan of them
//   6. children: terminal / small (subtree kernel) / big (next step)
// Work is split into tiles of kTile points of one cell.
#include "kdt_internal.cuh"
#include "kdt_launch.h"

namespace kdt {

namespace {

__device__ __forceinline__ bool tile_of(const StepDev& s, uint32_t tile, uint2* out) {
  if (tile >= *s.ntiles_total) return false;
  *out = s.tiles[tile];
  return true;
}

// ---------------------------------------------------------------- prep

// Single CTA: per-cell tile and segment counts, exclusive scans, key dim for
// cyclic keys.
__global__ void k_prep(const TreeDev* trees, StepDev s) {
  __shared__ uint32_t tmp[33];
  uint32_t tile_run = 0, seg_run = 0;
  for (uint32_t c0 = 0; c0 < s.ncells; c0 += blockDim.x) {
    const uint32_t c = c0 + threadIdx.x;
    uint32_t nt = 0, ns = 0;
    if (c < s.ncells) {
      const Cell cell = s.cells[c];
      const TreeDev& t = trees[cell.tree];
      nt = (cell.count + kTile - 1) / kTile;
      ns = (uint32_t)t.r;
      if (t.key_rule == KEY_CYCLIC) s.kdim[c] = (uint32_t)(cell.level % t.d);
    }
    uint32_t tot_t, tot_s;
    const uint32_t et = block_excl_scan(nt, tmp, &tot_t);
    const uint32_t es = block_excl_scan(ns, tmp, &tot_s);
    if (c < s.ncells) {
      s.tile_base[c] = tile_run + et;
      s.seg_base[c] = seg_run + es;
    }
    tile_run += tot_t;
    seg_run += tot_s;
  }
  if (threadIdx.x == 0) {
    s.tile_base[s.ncells] = tile_run;
    s.seg_base[s.ncells] = seg_run;
    *s.ntiles_total = tile_run;
    *s.bigseg_count = 0;
  }
}

// One CTA per cell: tile list entries and zeroed segment counts.
__global__ void k_tiles(const TreeDev* trees, StepDev s) {
  const uint32_t c = blockIdx.x;
  const Cell cell = s.cells[c];
  const uint32_t tb = s.tile_base[c], te = s.tile_base[c + 1];
  for (uint32_t j = tb + threadIdx.x; j < te; j += blockDim.x)
    s.tiles[j] = make_uint2(c, (j - tb) * (uint32_t)kTile);
  const uint32_t sb = s.seg_base[c], se = s.seg_base[c + 1];
  for (uint32_t g = sb + threadIdx.x; g < se; g += blockDim.x) s.seg_w[g] = 0;
  (void)trees;
  (void)cell;
}

// ------------------------------------------------------- widest spread

// Per tile and coordinate: min and max key (partials; reduced per cell below).
__global__ void __launch_bounds__(kTileThreads) k_minmax(const TreeDev* trees, StepDev s) {
  uint2 tl;
  if (!tile_of(s, blockIdx.x, &tl)) return;
  __shared__ uint32_t red[2][kTileThreads / 32];
  const Cell cell = s.cells[tl.x];
  const TreeDev& t = trees[cell.tree];
  const float* X = src_cols(t, cell.level);
  const int64_t n = t.n;
  const uint32_t end = min(tl.y + (uint32_t)kTile, cell.count);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int l = 0; l < t.d; ++l) {
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (uint32_t i = tl.y + threadIdx.x; i < end; i += blockDim.x) {
      const float x = X[(int64_t)l * n + cell.begin + i];
      if (is_nan_bits(x)) set_status(t, ST_NAN_INPUT);
      const uint32_t k = ord_key(x);
      lo = min(lo, k);
      hi = max(hi, k);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (lane == 0) {
      red[0][warp] = lo;
      red[1][warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        lo = min(lo, red[0][w]);
        hi = max(hi, red[1][w]);
      }
      s.tile_mm[((size_t)blockIdx.x * kMaxDims + l) * 2 + 0] = lo;
      s.tile_mm[((size_t)blockIdx.x * kMaxDims + l) * 2 + 1] = hi;
    }
    __syncthreads();
  }
}

// One CTA per cell: reduce the tile partials and pick the widest coordinate
// (range (double)max - (double)min; 0 when max and min are the same key;
// lowest coordinate on ties).
__global__ void k_pick_dim(const TreeDev* trees, StepDev s) {
  const uint32_t c = blockIdx.x;
  const Cell cell = s.cells[c];
  const TreeDev& t = trees[cell.tree];
  if (t.key_rule != KEY_WIDEST) return;
  __shared__ uint32_t slo[kMaxDims], shi[kMaxDims];
  const uint32_t tb = s.tile_base[c], te = s.tile_base[c + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int l = warp; l < t.d; l += nw) {
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (uint32_t j = tb + lane; j < te; j += 32) {
      lo = min(lo, s.tile_mm[((size_t)j * kMaxDims + l) * 2 + 0]);
      hi = max(hi, s.tile_mm[((size_t)j * kMaxDims + l) * 2 + 1]);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (lane == 0) {
      slo[l] = lo;
      shi[l] = hi;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    double best_range = -1.0;
    for (int l = 0; l < t.d; ++l) {
      const double range =
          (slo[l] == shi[l]) ? 0.0 : (double)key_float(shi[l]) - (double)key_float(slo[l]);
      if (range > best_range) {
        best_range = range;
        best = l;
      }
    }
    s.kdim[c] = (uint32_t)best;
  }
}

// ------------------------------------------------------------ segments

// Per tile: points per subset -> seg_w (shared-memory histogram, then one
// global atomic per non-empty subset of the tile).
__global__ void __launch_bounds__(kTileThreads) k_seg_count(const TreeDev* trees, StepDev s) {
  uint2 tl;
  if (!tile_of(s, blockIdx.x, &tl)) return;
  __shared__ uint32_t hist[kMaxSubsets];
  const Cell cell = s.cells[tl.x];
  const TreeDev& t = trees[cell.tree];
  const int r = t.r;
  const uint32_t* P = src_perm(t, cell.level);
  const void* S = src_sid(t, cell.level);
  for (int j = threadIdx.x; j < r; j += blockDim.x) hist[j] = 0;
  __syncthreads();
  const uint32_t end = min(tl.y + (uint32_t)kTile, cell.count);
  for (uint32_t i = tl.y + threadIdx.x; i < end; i += blockDim.x) {
    const int64_t p = (int64_t)cell.begin + i;
    const uint32_t orig = P ? P[p] : (uint32_t)p;
    atomicAdd(&hist[subset_of(t, S, orig, p)], 1u);
  }
  __syncthreads();
  uint32_t* w = s.seg_w + s.seg_base[tl.x];
  for (int j = threadIdx.x; j < r; j += blockDim.x)
    if (hist[j]) atomicAdd(&w[j], hist[j]);
}

// One CTA per cell: segment start positions (exclusive scan over subsets) and
// the list of segments too large for a single warp.
__global__ void k_seg_scan(const TreeDev* trees, StepDev s) {
  __shared__ uint32_t tmp[33];
  const uint32_t c = blockIdx.x;
  const Cell cell = s.cells[c];
  const int r = trees[cell.tree].r;
  const uint32_t g0 = s.seg_base[c];
  uint32_t run = 0;
  for (int j0 = 0; j0 < r; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    const uint32_t w = j < r ? s.seg_w[g0 + j] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(w, tmp, &tot);
    if (j < r) {
      const uint32_t beg = cell.begin + run + ex;
      s.seg_beg[g0 + j] = beg;
      s.seg_cur[g0 + j] = beg;
      s.seg_cell[g0 + j] = c;
      if (w > (uint32_t)kSelSmallMax) s.bigseg[atomicAdd(s.bigseg_count, 1u)] = g0 + j;
    }
    run += tot;
  }
}

// Per tile: copy the keys of the tile's points into the scratch array grouped
// by subset (order inside a segment is irrelevant to its median).
constexpr int kPerThread = kTile / kTileThreads;
__global__ void __launch_bounds__(kTileThreads) k_group(const TreeDev* trees, StepDev s) {
  uint2 tl;
  if (!tile_of(s, blockIdx.x, &tl)) return;
  __shared__ uint32_t cnt[kMaxSubsets];
  const Cell cell = s.cells[tl.x];
  const TreeDev& t = trees[cell.tree];
  const int r = t.r;
  const uint32_t dim = s.kdim[tl.x];
  const float* X = src_cols(t, cell.level) + (int64_t)dim * t.n;
  const uint32_t* P = src_perm(t, cell.level);
  const void* S = src_sid(t, cell.level);
  for (int j = threadIdx.x; j < r; j += blockDim.x) cnt[j] = 0;
  __syncthreads();
  const uint32_t end = min(tl.y + (uint32_t)kTile, cell.count);
  uint32_t key[kPerThread], sub[kPerThread], lr[kPerThread];
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    const uint32_t i = tl.y + threadIdx.x + q * blockDim.x;
    sub[q] = 0xffffffffu;
    if (i < end) {
      const int64_t p = (int64_t)cell.begin + i;
      const uint32_t orig = P ? P[p] : (uint32_t)p;
      sub[q] = subset_of(t, S, orig, p);
      key[q] = ord_key(X[p]);
      lr[q] = atomicAdd(&cnt[sub[q]], 1u);
    }
  }
  __syncthreads();
  uint32_t* cur = s.seg_cur + s.seg_base[tl.x];
  for (int j = threadIdx.x; j < r; j += blockDim.x)
    if (cnt[j]) cnt[j] = atomicAdd(&cur[j], cnt[j]);  // now: base position of this tile's run
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kPerThread; ++q)
    if (sub[q] != 0xffffffffu) t.keys[cnt[sub[q]] + lr[q]] = key[q];
}

// ------------------------------------------------------------ selection

// Exact key of 0-based rank `rank` among keys[0..w) by 8-bit MSD radix select,
// one warp, histogram `hist` (256 words of shared memory owned by the warp).
__device__ uint32_t warp_radix_select(const uint32_t* keys, uint32_t w, uint32_t rank, uint32_t* hist) {
  const int lane = threadIdx.x & 31;
  uint32_t prefix = 0, mask = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = lane; i < 256; i += 32) hist[i] = 0;
    __syncwarp();
    for (uint32_t i = lane; i < w; i += 32) {
      const uint32_t k = keys[i];
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
    }
    __syncwarp();
    uint32_t below;
    const uint32_t digit = warp_find_digit(hist, rank, &below);
    rank -= below;
    prefix |= digit << shift;
    mask |= 255u << shift;
    __syncwarp();
  }
  return prefix;
}

// Lower median of one small segment (w <= 32) by counting ranks in registers.
__device__ __forceinline__ uint32_t warp_rank_median(const uint32_t* keys, uint32_t w) {
  const int lane = threadIdx.x & 31;
  const uint32_t k = (uint32_t)lane < w ? keys[lane] : 0xffffffffu;
  const uint32_t want = (w - 1) / 2;
  uint32_t rk = 0;
  for (uint32_t j = 0; j < w; ++j) {
    const uint32_t kj = __shfl_sync(0xffffffffu, k, j);
    rk += (kj < k) || (kj == k && (int)j < lane);
  }
  const unsigned hit = __ballot_sync(0xffffffffu, (uint32_t)lane < w && rk == want);
  return __shfl_sync(0xffffffffu, k, __ffs(hit) - 1);
}

// One warp per segment of at most kSelSmallMax points.
__global__ void __launch_bounds__(256) k_select_small(const TreeDev* trees, StepDev s, uint32_t nseg) {
  __shared__ uint32_t hist[8][256];
  const int warp = threadIdx.x >> 5;
  const uint32_t g = blockIdx.x * 8u + (uint32_t)warp;
  if (g >= nseg) return;
  const uint32_t w = s.seg_w[g];
  if (w == 0 || w > (uint32_t)kSelSmallMax) return;
  const Cell cell = s.cells[s.seg_cell[g]];
  const uint32_t* keys = trees[cell.tree].keys + s.seg_beg[g];
  uint32_t med;
  if (w <= 32)
    med = warp_rank_median(keys, w);
  else
    med = warp_radix_select(keys, w, (w - 1) / 2, hist[warp]);
  if ((threadIdx.x & 31) == 0) s.seg_med[g] = med;
}

// One CTA per listed large segment: the same radix select with a CTA-wide
// histogram.
__global__ void __launch_bounds__(256) k_select_big(const TreeDev* trees, StepDev s) {
  if (blockIdx.x >= *s.bigseg_count) return;
  __shared__ uint32_t hist[256];
  __shared__ uint32_t bcast[2];
  const uint32_t g = s.bigseg[blockIdx.x];
  const uint32_t w = s.seg_w[g];
  const Cell cell = s.cells[s.seg_cell[g]];
  const uint32_t* keys = trees[cell.tree].keys + s.seg_beg[g];
  uint32_t rank = (w - 1) / 2, prefix = 0, mask = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < w; i += blockDim.x) {
      const uint32_t k = keys[i];
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
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
  if (threadIdx.x == 0) s.seg_med[g] = prefix;
}

// One CTA per cell: count-weighted lower median of the segment medians: the
// smallest median m whose segments with median <= m hold at least
// ceil(W/2) of the W points (weighted 8-bit MSD radix select).
__global__ void __launch_bounds__(256) k_combine(const TreeDev* trees, StepDev s) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t bcast[2];
  const uint32_t c = blockIdx.x;
  const Cell cell = s.cells[c];
  const TreeDev& t = trees[cell.tree];
  const int r = t.r;
  const uint32_t g0 = s.seg_base[c];
  uint32_t rank = (cell.count - 1) / 2, prefix = 0, mask = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
      const uint32_t w = s.seg_w[g0 + j];
      if (!w) continue;
      const uint32_t k = s.seg_med[g0 + j];
      if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], w);
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

// ------------------------------------------------------------ partition

// Per tile: number of points with key <= split.
__global__ void __launch_bounds__(kTileThreads) k_part_count(const TreeDev* trees, StepDev s) {
  uint2 tl;
  if (!tile_of(s, blockIdx.x, &tl)) return;
  const Cell cell = s.cells[tl.x];
  const TreeDev& t = trees[cell.tree];
  const float* X = src_cols(t, cell.level) + (int64_t)s.kdim[tl.x] * t.n + cell.begin;
  const uint32_t m = s.mkey[tl.x];
  const uint32_t end = min(tl.y + (uint32_t)kTile, cell.count);
  uint32_t cnt = 0;
  for (uint32_t i0 = tl.y; i0 < end; i0 += blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    const bool left = i < end && ord_key(X[i]) <= m;
    cnt += __syncthreads_count(left);
  }
  if (threadIdx.x == 0) s.tile_left[blockIdx.x] = cnt;
}

// One CTA per cell: exclusive scan of its tiles' left counts.
__global__ void k_part_scan(StepDev s) {
  __shared__ uint32_t tmp[33];
  const uint32_t c = blockIdx.x;
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

// Per tile: stable scatter of all columns, the permutation and the subset ids.
// Left points of the tile go to begin + (left points before the tile) + rank,
// right points to begin + L + (right points before the tile) + rank.
__global__ void __launch_bounds__(kTileThreads) k_part_scatter(const TreeDev* trees, StepDev s) {
  uint2 tl;
  if (!tile_of(s, blockIdx.x, &tl)) return;
  __shared__ uint32_t wsum[kTileThreads / 32];
  const Cell cell = s.cells[tl.x];
  const TreeDev& t = trees[cell.tree];
  const int level = cell.level;
  const int64_t n = t.n;
  const int d = t.d;
  const float* X = src_cols(t, level);
  const uint32_t* P = src_perm(t, level);
  const void* S = src_sid(t, level);
  float* Xo = t.xbuf[level & 1];
  uint32_t* Po = t.pbuf[level & 1];
  void* So = t.sbuf[level & 1];
  const bool explicit_sid = t.subset_mode == SUB_EXPLICIT;
  const uint32_t dim = s.kdim[tl.x];
  const uint32_t m = s.mkey[tl.x];
  const uint32_t loff = s.tile_loff[blockIdx.x];
  const uint32_t L = s.lcount[tl.x];
  uint32_t lnext = cell.begin + loff;
  uint32_t rnext = cell.begin + L + (tl.y - loff);
  // A child that is terminal is never read again: its points only need their
  // original index in the final order.
  const int child_stall = (cell.count == L) ? cell.stall + 1 : 0;
  const bool term_left = is_terminal(t, L, level + 1, child_stall);
  const bool term_right = is_terminal(t, cell.count - L, level + 1, child_stall);
  const uint32_t end = min(tl.y + (uint32_t)kTile, cell.count);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  bool saw_nan = false;
  for (uint32_t i0 = tl.y; i0 < end; i0 += blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    const bool valid = i < end;
    const int64_t p = (int64_t)cell.begin + i;
    bool left = false;
    if (valid) left = ord_key(X[(int64_t)dim * n + p]) <= m;
    const unsigned bal = __ballot_sync(0xffffffffu, left);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      const uint32_t v = wsum[w];
      before += (w < warp) ? v : 0u;
      total += v;
    }
    const uint32_t lrank = before + __popc(bal & lt_mask);
    const uint32_t nvalid = min((uint32_t)blockDim.x, end - i0);
    if (valid && (left ? term_left : term_right)) {
      const uint32_t dst = left ? lnext + lrank : rnext + (threadIdx.x - lrank);
      t.out_perm[dst] = P ? P[p] : (uint32_t)p;
      if (level == 0)
        for (int l = 0; l < d; ++l) saw_nan |= is_nan_bits(X[(int64_t)l * n + p]);
    } else if (valid) {
      const uint32_t dst = left ? lnext + lrank : rnext + (threadIdx.x - lrank);
      for (int l = 0; l < d; ++l) {
        const float x = X[(int64_t)l * n + p];
        saw_nan |= is_nan_bits(x);
        Xo[(int64_t)l * n + dst] = x;
      }
      Po[dst] = P ? P[p] : (uint32_t)p;
      if (explicit_sid) {
        if (t.sid_bytes == 1)
          ((uint8_t*)So)[dst] = ((const uint8_t*)S)[p];
        else
          ((uint16_t*)So)[dst] = ((const uint16_t*)S)[p];
      }
    }
    lnext += total;
    rnext += nvalid - total;
    __syncthreads();
  }
  if (saw_nan) set_status(t, ST_NAN_INPUT);
}

// ------------------------------------------------------------- children

// One thread per cell: classify the two children.
__global__ void k_next(const TreeDev* trees, StepDev s) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= s.ncells) return;
  const Cell cell = s.cells[c];
  const TreeDev& t = trees[cell.tree];
  const uint32_t L = s.lcount[c], R = cell.count - L;
  const int level = cell.level + 1;
  const int stall = (R == 0) ? cell.stall + 1 : 0;
  const uint32_t cb[2] = {cell.begin, cell.begin + L};
  const uint32_t cc[2] = {L, R};
  for (int side = 0; side < 2; ++side) {
    const uint32_t heap = 2u * cell.heap + 1u + (uint32_t)side;
    if (is_terminal(t, cc[side], level, stall)) {
      record_terminal(t, cb[side], cc[side], heap, level);
      continue;
    }
    if (t.depth == 0 && level >= t.max_levels) {
      set_status(t, ST_LEVEL_CAP);
      continue;
    }
    const Cell child{cb[side], cc[side], heap, cell.tree, (int16_t)level, (int16_t)stall};
    if (cc[side] <= (uint32_t)t.small_max) {
      const uint32_t slot = atomicAdd(s.small_count, 1u);
      if (slot < s.small_cap) s.small[slot] = child; else set_status(t, ST_CAPACITY);
    } else {
      const uint32_t slot = atomicAdd(s.next_big_count, 1u);
      if (slot < s.next_big_cap) s.next_big[slot] = child; else set_status(t, ST_CAPACITY);
    }
  }
}

}  // namespace

// ------------------------------------------------------------ launcher

void launch_big_step(const TreeDev* trees, const StepDev& s, uint32_t max_tiles, uint32_t nseg,
                     uint32_t max_bigseg, bool any_widest, cudaStream_t st) {
  const uint32_t nc = s.ncells;
  if (nc == 0) return;
  k_prep<<<1, 1024, 0, st>>>(trees, s);
  k_tiles<<<nc, 256, 0, st>>>(trees, s);
  if (any_widest) {
    k_minmax<<<max_tiles, kTileThreads, 0, st>>>(trees, s);
    k_pick_dim<<<nc, 256, 0, st>>>(trees, s);
  }
  k_seg_count<<<max_tiles, kTileThreads, 0, st>>>(trees, s);
  k_seg_scan<<<nc, 256, 0, st>>>(trees, s);
  k_group<<<max_tiles, kTileThreads, 0, st>>>(trees, s);
  k_select_small<<<(nseg + 7) / 8, 256, 0, st>>>(trees, s, nseg);
  if (max_bigseg) k_select_big<<<max_bigseg, 256, 0, st>>>(trees, s);
  k_combine<<<nc, 256, 0, st>>>(trees, s);
  k_part_count<<<max_tiles, kTileThreads, 0, st>>>(trees, s);
  k_part_scan<<<nc, 1024, 0, st>>>(s);
  k_part_scatter<<<max_tiles, kTileThreads, 0, st>>>(trees, s);
  k_next<<<(nc + 255) / 256, 256, 0, st>>>(trees, s);
}

}  // namespace kdt
