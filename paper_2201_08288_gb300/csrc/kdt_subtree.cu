// kdt_subtree.cu -- finish every remaining level of a small cell inside one
// CTA, and turn the terminal cells into the output offsets.
//
// A cell with at most subtree_capacity(d) points is loaded once into shared
// memory (all d coordinates as order-preserving keys, the permutation and the
// subset ids). Then, level by level (paper, Sec. 2: each level splits every
// cell of the previous one along its key), for all live local cells at once:
//   1. key coordinate (cyclic, or widest range);
//   2. counting sort of the points by (cell, subset) into bins, in batches of
//      at most kSubtreeBins bins; the lower median of every bin (rank counting
//      for bins of <= 16 points, a warp radix select above);
//   3. per cell, the count-weighted lower median of its bins' medians;
//   4. a stable partition of the local order around the split (ties left);
//   5. children: terminal cells are recorded, the others form the next level.
// The permutation is written once, at the end. The kernel is persistent: each
// CTA pulls cells from a queue and owns one slice of global memory for its
// local cell tables.
#include <algorithm>

#include "kdt_internal.cuh"
#include "kdt_launch.h"

namespace kdt {

namespace {

constexpr int T = kSubtreeThreads;
constexpr int NW = kSubtreeWarps;
constexpr uint16_t kNoCell = 0xffff;

// Radix select over keys reached through an index array (one warp).
__device__ uint32_t warp_select_indirect(const uint32_t* kbase, const uint16_t* idx, uint32_t w,
                                         uint32_t rank, uint32_t* hist) {
  const int lane = threadIdx.x & 31;
  uint32_t prefix = 0, mask = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = lane; i < 256; i += 32) hist[i] = 0;
    __syncwarp();
    for (uint32_t i = lane; i < w; i += 32) {
      const uint32_t k = kbase[idx[i]];
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

struct Smem {
  uint32_t* bins;    // kSubtreeBins + 1
  uint32_t* med;     // kSubtreeBins
  uint32_t* whist;   // NW * 256
  uint16_t* biglist; // kSubtreeBigBinCap
  uint32_t* keys;    // d * N
  uint32_t* perm;    // N
  uint16_t* sid;     // N
  uint16_t* ordA;    // N
  uint16_t* ordB;    // N
  uint16_t* cellid;  // N
  uint16_t* pre;     // N + 1
};

__device__ Smem carve(uint8_t* base, int N, int d) {
  Smem s;
  s.bins = (uint32_t*)base;
  s.med = s.bins + kSubtreeBins + 1;
  s.whist = s.med + kSubtreeBins;
  s.biglist = (uint16_t*)(s.whist + NW * 256);
  s.keys = (uint32_t*)(s.biglist + kSubtreeBigBinCap);
  s.perm = s.keys + (size_t)d * N;
  s.sid = (uint16_t*)(s.perm + N);
  s.ordA = s.sid + N;
  s.ordB = s.ordA + N;
  s.cellid = s.ordB + N;
  s.pre = s.cellid + N;
  return s;
}

__global__ void __launch_bounds__(T, 1)
k_subtree(const TreeDev* trees, const Cell* list, uint32_t count, uint32_t* head, LCell* slices,
          uint32_t slice_cells) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t s_item, s_ncur, s_nbig;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  LCell* cur = slices + (size_t)blockIdx.x * 2 * slice_cells;
  LCell* nxt = cur + slice_cells;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(head, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= count) break;
    const Cell c = list[item];
    const TreeDev& t = trees[c.tree];
    const int N = (int)c.count;
    const int d = t.d, r = t.r;
    const int64_t n = t.n;
    Smem S = carve(smem_raw, N, d);
    uint16_t* ordA = S.ordA;
    uint16_t* ordB = S.ordB;
    LCell* cc = cur;
    LCell* nc = nxt;

    // ---- load the cell
    {
      const float* X = src_cols(t, c.level) + c.begin;
      const uint32_t* P = src_perm(t, c.level);
      const void* SID = src_sid(t, c.level);
      bool nan = false;
      for (int l = 0; l < d; ++l) {
        const float* col = X + (int64_t)l * n;
        uint32_t* kd = S.keys + (size_t)l * N;
        for (int i = tid; i < N; i += T) {
          const float x = col[i];
          nan |= is_nan_bits(x);
          kd[i] = ord_key(x);
        }
      }
      if (nan) set_status(t, ST_NAN_INPUT);
      for (int i = tid; i < N; i += T) {
        const int64_t p = (int64_t)c.begin + i;
        const uint32_t orig = P ? P[p] : (uint32_t)p;
        S.perm[i] = orig;
        S.sid[i] = (uint16_t)subset_of(t, SID, orig, p);
        ordA[i] = (uint16_t)i;
        S.cellid[i] = 0;
      }
      if (tid == 0) {
        cc[0] = LCell{0u, (uint32_t)N, c.heap, c.stall, 0u, 0u, 0u, 0u};
        s_ncur = 1;
      }
    }
    __syncthreads();

    int level = c.level;
    for (;;) {
      const uint32_t ncur = s_ncur;
      if (ncur == 0) break;

      // ---- 1. key coordinate of every live cell
      if (t.key_rule == KEY_CYCLIC) {
        for (uint32_t k = tid; k < ncur; k += T) cc[k].dim = (uint32_t)(level % d);
      } else if (ncur >= (uint32_t)NW) {
        for (uint32_t k = warp; k < ncur; k += NW) {
          const uint32_t b = cc[k].begin, e = b + cc[k].count;
          int best = 0;
          double best_range = -1.0;
          for (int l = 0; l < d; ++l) {
            const uint32_t* kd = S.keys + (size_t)l * N;
            uint32_t lo = 0xffffffffu, hi = 0u;
            for (uint32_t i = b + lane; i < e; i += 32) {
              const uint32_t kk = kd[ordA[i]];
              lo = min(lo, kk);
              hi = max(hi, kk);
            }
            lo = warp_min(lo);
            hi = warp_max(hi);
            const double range = (lo == hi) ? 0.0 : (double)key_float(hi) - (double)key_float(lo);
            if (range > best_range) {
              best_range = range;
              best = l;
            }
          }
          if (lane == 0) cc[k].dim = (uint32_t)best;
        }
      } else {
        // few cells: several warps per cell, partial min/max merged in shared memory
        uint32_t* tab = S.bins;  // [ncur][d][2]
        for (uint32_t j = tid; j < ncur * (uint32_t)d; j += T) {
          tab[2 * j] = 0xffffffffu;
          tab[2 * j + 1] = 0u;
        }
        __syncthreads();
        const uint32_t G = NW / ncur;
        const uint32_t k = warp / G, part = warp % G;
        if (k < ncur) {
          const uint32_t b = cc[k].begin, cnt = cc[k].count;
          const uint32_t lo_i = b + (uint32_t)(((uint64_t)cnt * part) / G);
          const uint32_t hi_i = b + (uint32_t)(((uint64_t)cnt * (part + 1)) / G);
          for (int l = 0; l < d; ++l) {
            const uint32_t* kd = S.keys + (size_t)l * N;
            uint32_t lo = 0xffffffffu, hi = 0u;
            for (uint32_t i = lo_i + lane; i < hi_i; i += 32) {
              const uint32_t kk = kd[ordA[i]];
              lo = min(lo, kk);
              hi = max(hi, kk);
            }
            lo = warp_min(lo);
            hi = warp_max(hi);
            if (lane == 0) {
              atomicMin(&tab[(k * d + l) * 2], lo);
              atomicMax(&tab[(k * d + l) * 2 + 1], hi);
            }
          }
        }
        __syncthreads();
        for (uint32_t kk = tid; kk < ncur; kk += T) {
          int best = 0;
          double best_range = -1.0;
          for (int l = 0; l < d; ++l) {
            const uint32_t lo = tab[(kk * d + l) * 2], hi = tab[(kk * d + l) * 2 + 1];
            const double range = (lo == hi) ? 0.0 : (double)key_float(hi) - (double)key_float(lo);
            if (range > best_range) {
              best_range = range;
              best = l;
            }
          }
          cc[kk].dim = (uint32_t)best;
        }
      }
      __syncthreads();

      // ---- 2/3. per-(cell, subset) medians and their weighted median, in batches
      const uint32_t CB = max(1u, (uint32_t)kSubtreeBins / (uint32_t)r);
      for (uint32_t kb = 0; kb < ncur; kb += CB) {
        const uint32_t ke = min(ncur, kb + CB);
        const uint32_t nb = (ke - kb) * (uint32_t)r;
        const uint32_t pb = cc[kb].begin;
        const uint32_t pe = cc[ke - 1].begin + cc[ke - 1].count;
        for (uint32_t b = tid; b <= nb; b += T) S.bins[b] = 0;
        if (tid == 0) s_nbig = 0;
        __syncthreads();
        for (uint32_t i = pb + tid; i < pe; i += T) {
          const uint16_t k = S.cellid[i];
          if (k == kNoCell) continue;
          const uint32_t b = (k - kb) * (uint32_t)r + S.sid[ordA[i]];
          S.pre[i] = (uint16_t)atomicAdd(&S.bins[b], 1u);
        }
        __syncthreads();
        {  // exclusive scan of bins[0..nb), total in bins[nb]
          const uint32_t per = (nb + T - 1) / T;
          const uint32_t b0 = min(nb, tid * per), b1 = min(nb, b0 + per);
          uint32_t sum = 0;
          for (uint32_t b = b0; b < b1; ++b) sum += S.bins[b];
          uint32_t tot;
          uint32_t run = block_excl_scan(sum, tmp, &tot);
          for (uint32_t b = b0; b < b1; ++b) {
            const uint32_t v = S.bins[b];
            S.bins[b] = run;
            run += v;
          }
          if (tid == 0) S.bins[nb] = tot;
        }
        __syncthreads();
        for (uint32_t i = pb + tid; i < pe; i += T) {
          const uint16_t k = S.cellid[i];
          if (k == kNoCell) continue;
          const uint32_t b = (k - kb) * (uint32_t)r + S.sid[ordA[i]];
          ordB[pb + S.bins[b] + S.pre[i]] = ordA[i];
        }
        __syncthreads();
        for (uint32_t b = tid; b < nb; b += T) {
          const uint32_t beg = S.bins[b], w = S.bins[b + 1] - beg;
          if (w == 0) continue;
          if (w > 16) {
            const uint32_t slot = atomicAdd(&s_nbig, 1u);
            S.biglist[slot] = (uint16_t)b;
            continue;
          }
          const uint32_t k = kb + b / (uint32_t)r;
          const uint32_t* kd = S.keys + (size_t)cc[k].dim * N;
          const uint16_t* g = ordB + pb + beg;
          const uint32_t want = (w - 1) / 2;
          uint32_t m = 0;
          for (uint32_t j = 0; j < w; ++j) {
            const uint32_t kj = kd[g[j]];
            uint32_t rk = 0;
            for (uint32_t q = 0; q < w; ++q) {
              const uint32_t kq = kd[g[q]];
              rk += (kq < kj) || (kq == kj && q < j);
            }
            if (rk == want) {
              m = kj;
              break;
            }
          }
          S.med[b] = m;
        }
        __syncthreads();
        const uint32_t nbig = s_nbig;
        for (uint32_t j = warp; j < nbig; j += NW) {
          const uint32_t b = S.biglist[j];
          const uint32_t beg = S.bins[b], w = S.bins[b + 1] - beg;
          const uint32_t k = kb + b / (uint32_t)r;
          const uint32_t m = warp_select_indirect(S.keys + (size_t)cc[k].dim * N, ordB + pb + beg, w,
                                                  (w - 1) / 2, S.whist + warp * 256);
          if (lane == 0) S.med[b] = m;
        }
        __syncthreads();
        // weighted lower median per cell (one warp per cell)
        for (uint32_t k = kb + warp; k < ke; k += NW) {
          uint32_t* hist = S.whist + warp * 256;
          const uint32_t b0 = (k - kb) * (uint32_t)r;
          uint32_t rank = (cc[k].count - 1) / 2, prefix = 0, mask = 0;
          for (int shift = 24; shift >= 0; shift -= 8) {
            for (int i = lane; i < 256; i += 32) hist[i] = 0;
            __syncwarp();
            for (int j = lane; j < r; j += 32) {
              const uint32_t w = S.bins[b0 + j + 1] - S.bins[b0 + j];
              if (!w) continue;
              const uint32_t key = S.med[b0 + j];
              if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], w);
            }
            __syncwarp();
            uint32_t below;
            const uint32_t digit = warp_find_digit(hist, rank, &below);
            rank -= below;
            prefix |= digit << shift;
            mask |= 255u << shift;
            __syncwarp();
          }
          if (lane == 0) {
            cc[k].mkey = prefix;
            t.out_vals[cc[k].heap] = key_float(prefix);
            t.out_dims[cc[k].heap] = (int8_t)cc[k].dim;
          }
        }
        __syncthreads();
      }

      // ---- 4. stable partition of the local order (key <= split to the left)
      {
        const uint32_t per = ((uint32_t)N + T - 1) / T;
        const uint32_t i0 = min((uint32_t)N, tid * per), i1 = min((uint32_t)N, i0 + per);
        uint32_t sum = 0;
        for (uint32_t i = i0; i < i1; ++i) {
          const uint16_t k = S.cellid[i];
          if (k == kNoCell) continue;
          sum += S.keys[(size_t)cc[k].dim * N + ordA[i]] <= cc[k].mkey;
        }
        uint32_t tot;
        uint32_t run = block_excl_scan(sum, tmp, &tot);
        for (uint32_t i = i0; i < i1; ++i) {
          S.pre[i] = (uint16_t)run;
          const uint16_t k = S.cellid[i];
          if (k != kNoCell) run += S.keys[(size_t)cc[k].dim * N + ordA[i]] <= cc[k].mkey;
        }
        if (tid == 0) S.pre[N] = (uint16_t)tot;
      }
      __syncthreads();
      for (uint32_t k = tid; k < ncur; k += T)
        cc[k].lcount = (uint32_t)S.pre[cc[k].begin + cc[k].count] - S.pre[cc[k].begin];
      __syncthreads();
      for (uint32_t i = tid; i < (uint32_t)N; i += T) {
        const uint16_t k = S.cellid[i];
        if (k == kNoCell) {
          ordB[i] = ordA[i];
          continue;
        }
        const uint32_t b = cc[k].begin;
        const bool left = S.keys[(size_t)cc[k].dim * N + ordA[i]] <= cc[k].mkey;
        const uint32_t lb = (uint32_t)S.pre[i] - S.pre[b];
        const uint32_t dst = left ? b + lb : b + cc[k].lcount + (i - b - lb);
        ordB[dst] = ordA[i];
      }
      __syncthreads();
      {
        uint16_t* x = ordA;
        ordA = ordB;
        ordB = x;
      }

      // ---- 5. children
      const int nlevel = level + 1;
      uint32_t run_out = 0;
      for (uint32_t k0 = 0; k0 < ncur; k0 += T) {
        const uint32_t k = k0 + tid;
        LCell ch[2];
        int nlive = 0;
        if (k < ncur) {
          const LCell p = cc[k];
          const uint32_t L = p.lcount, R = p.count - L;
          const int stall = (R == 0) ? p.stall + 1 : 0;
          const uint32_t cb[2] = {p.begin, p.begin + L};
          const uint32_t cn[2] = {L, R};
          for (int side = 0; side < 2; ++side) {
            const uint32_t heap = 2u * p.heap + 1u + (uint32_t)side;
            if (is_terminal(t, cn[side], nlevel, stall)) {
              record_terminal(t, c.begin + cb[side], cn[side], heap, nlevel);
            } else if (t.depth == 0 && nlevel >= t.max_levels) {
              set_status(t, ST_LEVEL_CAP);
            } else {
              ch[nlive++] = LCell{cb[side], cn[side], heap, stall, 0u, 0u, 0u, 0u};
            }
          }
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan((uint32_t)nlive, tmp, &tot);
        for (int j = 0; j < nlive; ++j) nc[run_out + ex + j] = ch[j];
        run_out += tot;
      }
      for (uint32_t i = tid; i < (uint32_t)N; i += T) S.cellid[i] = kNoCell;
      if (tid == 0) s_ncur = run_out;
      __syncthreads();
      for (uint32_t j = warp; j < run_out; j += NW) {
        const uint32_t b = nc[j].begin, e = b + nc[j].count;
        for (uint32_t i = b + lane; i < e; i += 32) S.cellid[i] = (uint16_t)j;
      }
      __syncthreads();
      {
        LCell* x = cc;
        cc = nc;
        nc = x;
      }
      level = nlevel;
    }

    // ---- write the permutation in final order
    for (int i = tid; i < N; i += T) t.out_perm[(int64_t)c.begin + i] = S.perm[ordA[i]];
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

__global__ void k_iota(uint32_t* out, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = i;
}

}  // namespace

void launch_iota(uint32_t* out, uint32_t n, cudaStream_t st) {
  if (n == 0) return;
  k_iota<<<std::min<uint32_t>((n + 255) / 256, 4096u), 256, 0, st>>>(out, n);
}

cudaError_t prepare_subtree_kernel() {
  return cudaFuncSetAttribute(k_subtree, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSubtreeSmemBytes);
}

void launch_subtree(const TreeDev* trees, const Cell* list, uint32_t count, uint32_t* head, LCell* slices,
                    uint32_t slice_cells, uint32_t grid, cudaStream_t st) {
  if (count == 0) return;
  cudaMemsetAsync(head, 0, sizeof(uint32_t), st);
  k_subtree<<<grid, T, kSubtreeSmemBytes, st>>>(trees, list, count, head, slices, slice_cells);
}

void launch_finalize(const TreeDev* tree, const uint32_t* term_count, uint32_t max_terms, cudaStream_t st) {
  const uint32_t blocks = (max_terms + 7) / 8 + 1;
  k_finalize<<<blocks, 256, 0, st>>>(tree, term_count);
}

}  // namespace kdt
