// kdt_subtree.cu -- finish every remaining level of a small cell inside one
// CTA, and turn the terminal cells into the output offsets.
//
// A cell with at most subtree_capacity(d) points is staged once into shared
// memory with bulk asynchronous copies (cp.async.bulk, completion on an
// mbarrier): all d coordinate columns and the permutation. Then, level by
// level (paper, Sec. 2: each level splits every cell of the previous one
// along its key), for all live local cells at once:
//   1. key coordinate (cyclic, or widest range);
//   2. counting sort of the points by (cell, subset) into bins, in batches of
//      at most kSubtreeBins bins, gathering each bin's keys contiguously; the
//      lower median of every bin by per-point rank counting (bins of at most
//      kRankMax points) or a warp radix select (larger bins);
//   3. per cell, the count-weighted lower median of its bins' medians;
//   4. a stable partition of the local order around the split (ties left);
//   5. children: terminal cells are recorded, the others form the next level.
// The permutation is written once, at the end. The kernel is persistent: each
// CTA pulls cells from a queue.
#include <algorithm>

#include "kdt_internal.cuh"
#include "kdt_launch.h"
#include "kdt_ptx.cuh"
#include "kdt_trace.h"

namespace kdt {

namespace {

constexpr int T = kSubtreeThreads;
constexpr int NW = kSubtreeWarps;
constexpr uint16_t kNoCell = 0xffff;
constexpr uint32_t kRankMax = 24;

// -------------------------------------------------------- shared layout

struct Smem {
  uint32_t* bins;     // kSubtreeBins + 1 (also the widest min/max table)
  uint32_t* med;      // kSubtreeBins
  uint32_t* whist;    // NW * 256
  uint16_t* biglist;  // kSubtreeBigBinCap
  LCell* tab[2];      // kSubtreeSmemCells each
  uint32_t* keys;     // (d + 1) columns at stride `stride`; column d is the permutation
  uint32_t* gk;       // N: keys gathered in bin order
  uint16_t* sid;      // N
  uint16_t* ordA;     // N
  uint16_t* ordB;     // N
  uint16_t* cellid;   // N
  uint16_t* pre;      // N + 1
  uint16_t* aux;      // N: bin of a gathered position, then the left flag of a position
};

__device__ __forceinline__ uint8_t* al16(uint8_t* p) {
  return (uint8_t*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
}

__device__ Smem carve(uint8_t* base, uint32_t N, int d) {
  Smem s;
  uint8_t* p = base;
  s.bins = (uint32_t*)p;
  p += 16400;
  s.med = (uint32_t*)p;
  p += kSubtreeBins * 4;
  s.whist = (uint32_t*)p;
  p += NW * 256 * 4;
  s.biglist = (uint16_t*)p;
  p += kSubtreeBigBinCap * 2;
  s.tab[0] = (LCell*)p;
  p += kSubtreeSmemCells * sizeof(LCell);
  s.tab[1] = (LCell*)p;
  p += kSubtreeSmemCells * sizeof(LCell);
  const uint32_t stride = subtree_stride(N);
  s.keys = (uint32_t*)p;
  p += (size_t)(d + 1) * stride * 4;
  s.gk = (uint32_t*)p;
  p = al16(p + (size_t)N * 4);
  uint16_t** arr[6] = {&s.sid, &s.ordA, &s.ordB, &s.cellid, &s.pre, &s.aux};
  for (int i = 0; i < 6; ++i) {
    *arr[i] = (uint16_t*)p;
    p = al16(p + ((size_t)N + 1) * 2);
  }
  return s;
}

// Radix select over a contiguous run of keys in shared memory (one warp).
__device__ uint32_t warp_select_smem(const uint32_t* keys, uint32_t w, uint32_t rank, uint32_t* hist) {
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

__device__ __forceinline__ double key_range(uint32_t lo, uint32_t hi) {
  return (lo == hi) ? 0.0 : (double)key_float(hi) - (double)key_float(lo);
}

__global__ void __launch_bounds__(T, 1)
k_subtree(const TreeDev* trees, const Cell* list, uint32_t count, uint32_t* head, LCell* slices,
          uint32_t slice_cells) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t s_item, s_ncur, s_nbig, s_where, s_fail;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_colbase[kMaxDims + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  LCell* gslice[2] = {slices + (size_t)blockIdx.x * 2 * slice_cells,
                      slices + (size_t)blockIdx.x * 2 * slice_cells + slice_cells};
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
    const Cell c = list[item];
    const TreeDev& t = trees[c.tree];
    const uint32_t N = c.count;
    const int d = t.d, r = t.r;
    const int64_t n = t.n;
    const uint32_t stride = subtree_stride(N);
    Smem S = carve(smem_raw, N, d);
    // Column l of the cell sits at S.keys + s_colbase[l]; column d holds the
    // permutation. Each column's offset absorbs the 16-byte alignment phase
    // of its global source so that the bulk copies are aligned on both sides.

    // ---- 0. stage the cell: bulk copies of the aligned middle, plain loads at the edges
    {
      const float* X = src_cols(t, c.level);
      const uint32_t* P = src_perm(t, c.level);
      const uint32_t b0 = c.begin, e0 = c.begin + N;
      const int ncols = d + (P ? 1 : 0);
      auto src_of = [&](int l) -> const uint32_t* {
        return l < d ? (const uint32_t*)(X + (int64_t)l * n) : P;
      };
      // phase of element b0 of column l: elements past the previous 16-byte boundary
      auto phase_of = [&](int l) -> uint32_t {
        return (uint32_t)(((uintptr_t)(src_of(l) + b0) >> 2) & 3u);
      };
      if (tid <= d) s_colbase[tid] = (uint32_t)tid * stride + (tid < ncols ? phase_of(tid) : 0u);
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
            bulk_g2s(S.keys + (size_t)l * stride + ph + (a0 - b0), src_of(l) + a0, (a1 - a0) * 4u, &s_bar);
        }
      }
      for (int j = tid; j < ncols * 8; j += T) {
        const int l = j >> 3, e = j & 7;
        const uint32_t ph = phase_of(l);
        const uint32_t a0 = min(b0 + ((4u - ph) & 3u), e0);
        const uint32_t a1 = a0 + ((e0 - a0) & ~3u);
        const uint32_t idx = e < 4 ? b0 + e : a1 + (e - 4);
        const bool ok = e < 4 ? (idx < a0) : (idx < e0);
        if (ok) S.keys[(size_t)l * stride + ph + (idx - b0)] = src_of(l)[idx];
      }
      __syncthreads();
      uint32_t* pm0 = S.keys + s_colbase[d];
      if (!P)
        for (uint32_t i = tid; i < N; i += T) pm0[i] = b0 + i;
      if (!mbar_wait_bounded(&s_bar, phase)) {
        set_status(t, ST_TIMEOUT);
        atomicExch(&s_fail, 1u);
      }
      phase ^= 1u;
      __syncthreads();
      if (s_fail) {  // copies in flight: wait once more (bounded), then stop this CTA
        mbar_wait_bounded(&s_bar, phase ^ 1u);
        break;
      }
      bool nan = false;
      for (int l = 0; l < d; ++l) {
        uint32_t* col = S.keys + s_colbase[l];
        for (uint32_t i = tid; i < N; i += T) {
          const float x = __uint_as_float(col[i]);
          nan |= is_nan_bits(x);
          col[i] = ord_key(x);
        }
      }
      if (nan) set_status(t, ST_NAN_INPUT);
      const void* SID = src_sid(t, c.level);
      for (uint32_t i = tid; i < N; i += T) {
        S.sid[i] = (uint16_t)subset_of(t, SID, pm0[i], (int64_t)b0 + i);
        S.ordA[i] = (uint16_t)i;
        S.cellid[i] = 0;
      }
      if (tid == 0) {
        S.tab[0][0] = LCell{c.heap, 0u, 0, (uint16_t)N, 0, 0, (uint8_t)c.stall};
        s_ncur = 1;
        s_where = 0;
      }
    }
    __syncthreads();

    const uint32_t* pm = S.keys + s_colbase[d];
    uint16_t* ordA = S.ordA;
    uint16_t* ordB = S.ordB;
    int which = 0;
    int level = c.level;
    for (;;) {
      const uint32_t ncur = s_ncur;
      if (ncur == 0) break;
      LCell* cc = s_where ? gslice[which] : S.tab[which];

      // ---- 1. key coordinate of every live cell
      if (t.key_rule == KEY_CYCLIC) {
        for (uint32_t k = tid; k < ncur; k += T) cc[k].dim = (uint8_t)(level % d);
      } else if (ncur >= (uint32_t)NW) {
        for (uint32_t k = warp; k < ncur; k += NW) {
          const uint32_t b = cc[k].begin, e = b + cc[k].count;
          int best = 0;
          double best_range = -1.0;
          for (int l = 0; l < d; ++l) {
            const uint32_t* col = S.keys + s_colbase[l];
            uint32_t lo = 0xffffffffu, hi = 0u;
            for (uint32_t i = b + lane; i < e; i += 32) {
              const uint32_t kk = col[ordA[i]];
              lo = min(lo, kk);
              hi = max(hi, kk);
            }
            lo = warp_min(lo);
            hi = warp_max(hi);
            const double range = key_range(lo, hi);
            if (range > best_range) {
              best_range = range;
              best = l;
            }
          }
          if (lane == 0) cc[k].dim = (uint8_t)best;
        }
      } else {
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
          const uint32_t i0 = b + (cnt * part) / G, i1 = b + (cnt * (part + 1)) / G;
          for (int l = 0; l < d; ++l) {
            const uint32_t* col = S.keys + s_colbase[l];
            uint32_t lo = 0xffffffffu, hi = 0u;
            for (uint32_t i = i0 + lane; i < i1; i += 32) {
              const uint32_t kk = col[ordA[i]];
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
            const double range = key_range(tab[(kk * d + l) * 2], tab[(kk * d + l) * 2 + 1]);
            if (range > best_range) {
              best_range = range;
              best = l;
            }
          }
          cc[kk].dim = (uint8_t)best;
        }
      }
      __syncthreads();

      // ---- 2/3. per-(cell, subset) medians and their weighted median, in batches
      const uint32_t CB = max(1u, (uint32_t)kSubtreeBins / (uint32_t)r);
      for (uint32_t kb0 = 0; kb0 < ncur; kb0 += CB) {
        const uint32_t ke = min(ncur, kb0 + CB);
        const uint32_t nb = (ke - kb0) * (uint32_t)r;
        const uint32_t pb = cc[kb0].begin;
        const uint32_t pe = cc[ke - 1].begin + cc[ke - 1].count;
        for (uint32_t b = tid; b <= nb; b += T) S.bins[b] = 0;
        if (tid == 0) s_nbig = 0;
        __syncthreads();
        for (uint32_t i = pb + tid; i < pe; i += T) {
          const uint16_t k = S.cellid[i];
          if (k == kNoCell) continue;
          const uint32_t b = (k - kb0) * (uint32_t)r + S.sid[ordA[i]];
          S.pre[i] = (uint16_t)atomicAdd(&S.bins[b], 1u);
        }
        __syncthreads();
        {  // exclusive scan of bins[0..nb), total in bins[nb]
          const uint32_t per = (nb + T - 1) / T;
          const uint32_t q0 = min(nb, tid * per), q1 = min(nb, q0 + per);
          uint32_t sum = 0;
          for (uint32_t b = q0; b < q1; ++b) sum += S.bins[b];
          uint32_t tot;
          uint32_t run = block_excl_scan(sum, tmp, &tot);
          for (uint32_t b = q0; b < q1; ++b) {
            const uint32_t v = S.bins[b];
            S.bins[b] = run;
            run += v;
          }
          if (tid == 0) S.bins[nb] = tot;
        }
        __syncthreads();
        const uint32_t nact = S.bins[nb];
        for (uint32_t i = pb + tid; i < pe; i += T) {
          const uint16_t k = S.cellid[i];
          if (k == kNoCell) continue;
          const uint32_t b = (k - kb0) * (uint32_t)r + S.sid[ordA[i]];
          const uint32_t pos = pb + S.bins[b] + S.pre[i];
          ordB[pos] = ordA[i];
          S.aux[pos] = (uint16_t)b;
          S.gk[pos] = S.keys[s_colbase[cc[k].dim] + ordA[i]];
        }
        __syncthreads();
        for (uint32_t q = pb + tid; q < pb + nact; q += T) {
          const uint32_t b = S.aux[q];
          const uint32_t bs = pb + S.bins[b], be = pb + S.bins[b + 1];
          const uint32_t w = be - bs;
          if (w > kRankMax) {
            if (q == bs) S.biglist[atomicAdd(&s_nbig, 1u)] = (uint16_t)b;
            continue;
          }
          const uint32_t k = S.gk[q];
          uint32_t rk = 0;
          for (uint32_t j = bs; j < be; ++j) {
            const uint32_t kj = S.gk[j];
            rk += (kj < k) | ((kj == k) & (j < q));
          }
          if (rk == (w - 1) / 2) S.med[b] = k;
        }
        __syncthreads();
        const uint32_t nbig = s_nbig;
        for (uint32_t j = warp; j < nbig; j += NW) {
          const uint32_t b = S.biglist[j];
          const uint32_t bs = pb + S.bins[b], w = S.bins[b + 1] - S.bins[b];
          const uint32_t m = warp_select_smem(S.gk + bs, w, (w - 1) / 2, S.whist + warp * 256);
          if (lane == 0) S.med[b] = m;
        }
        __syncthreads();
        // weighted lower median per cell: smallest bin median m whose bins with
        // median <= m hold >= ceil(W/2) points (weighted 8-bit radix select)
        const uint32_t ncb = ke - kb0;
        if (ncb >= (uint32_t)NW) {
          for (uint32_t k = kb0 + warp; k < ke; k += NW) {
            uint32_t* hist = S.whist + warp * 256;
            const uint32_t q0 = (k - kb0) * (uint32_t)r;
            uint32_t rank = (cc[k].count - 1u) / 2u, prefix = 0, mask = 0;
            for (int shift = 24; shift >= 0; shift -= 8) {
              for (int i = lane; i < 256; i += 32) hist[i] = 0;
              __syncwarp();
              for (int j = lane; j < r; j += 32) {
                const uint32_t w = S.bins[q0 + j + 1] - S.bins[q0 + j];
                const uint32_t key = S.med[q0 + j];
                if (w && (key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], w);
              }
              __syncwarp();
              uint32_t below;
              const uint32_t digit = warp_find_digit(hist, rank, &below);
              rank -= below;
              prefix |= digit << shift;
              mask |= 255u << shift;
              __syncwarp();
            }
            if (lane == 0) cc[k].mkey = prefix;
          }
        } else {
          // few cells: G warps per cell share one histogram per cell
          const uint32_t G = NW / ncb;
          const uint32_t kk = warp / G, part = warp % G;
          uint32_t* hist = S.whist + (kk < ncb ? kk : 0) * 256;
          uint32_t rank = kk < ncb ? (cc[kb0 + kk].count - 1u) / 2u : 0u, prefix = 0, mask = 0;
          const uint32_t q0 = kk * (uint32_t)r;
          for (int shift = 24; shift >= 0; shift -= 8) {
            for (uint32_t i = tid; i < ncb * 256u; i += T) S.whist[i] = 0;
            __syncthreads();
            if (kk < ncb) {
              for (uint32_t j = part * 32 + lane; j < (uint32_t)r; j += G * 32) {
                const uint32_t w = S.bins[q0 + j + 1] - S.bins[q0 + j];
                const uint32_t key = S.med[q0 + j];
                if (w && (key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], w);
              }
            }
            __syncthreads();
            if (kk < ncb) {
              uint32_t below;
              const uint32_t digit = warp_find_digit(hist, rank, &below);
              rank -= below;
              prefix |= digit << shift;
              mask |= 255u << shift;
            }
            __syncthreads();
          }
          if (kk < ncb && part == 0 && lane == 0) cc[kb0 + kk].mkey = prefix;
        }
        __syncthreads();
        for (uint32_t k = kb0 + tid; k < ke; k += T) {
          t.out_vals[cc[k].heap] = key_float(cc[k].mkey);
          t.out_dims[cc[k].heap] = (int8_t)cc[k].dim;
        }
      }
      __syncthreads();

      // ---- 4. stable partition of the local order (key <= split to the left)
      {
        const uint32_t per = (N + T - 1) / T;
        const uint32_t i0 = min(N, tid * per), i1 = min(N, i0 + per);
        uint32_t sum = 0;
        for (uint32_t i = i0; i < i1; ++i) {
          const uint16_t k = S.cellid[i];
          uint16_t f = 0;
          if (k != kNoCell) f = S.keys[s_colbase[cc[k].dim] + ordA[i]] <= cc[k].mkey;
          S.aux[i] = f;
          sum += f;
        }
        uint32_t tot;
        uint32_t run = block_excl_scan(sum, tmp, &tot);
        for (uint32_t i = i0; i < i1; ++i) {
          S.pre[i] = (uint16_t)run;
          run += S.aux[i];
        }
        if (tid == 0) S.pre[N] = (uint16_t)tot;
      }
      __syncthreads();
      for (uint32_t k = tid; k < ncur; k += T)
        cc[k].lcount = (uint16_t)(S.pre[cc[k].begin + cc[k].count] - S.pre[cc[k].begin]);
      __syncthreads();
      for (uint32_t i = tid; i < N; i += T) {
        const uint16_t k = S.cellid[i];
        if (k == kNoCell) {
          ordB[i] = ordA[i];
          continue;
        }
        const uint32_t b = cc[k].begin;
        const uint32_t lb = (uint32_t)S.pre[i] - S.pre[b];
        const uint32_t dst = S.aux[i] ? b + lb : b + cc[k].lcount + (i - b - lb);
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
      const int nwhere = total_live <= (uint32_t)kSubtreeSmemCells ? 0 : 1;
      LCell* nc = nwhere ? gslice[which ^ 1] : S.tab[which ^ 1];
      uint32_t run_out = 0;
      for (uint32_t k0 = 0; k0 < ncur; k0 += T) {
        const uint32_t k = k0 + tid;
        LCell ch0{}, ch1{};
        uint32_t nlive = 0;
        if (k < ncur) {
          const LCell p = cc[k];
          const uint32_t L = p.lcount, R = p.count - L;
          const int stall = (R == 0) ? p.stall + 1 : 0;
          const uint32_t cbeg[2] = {p.begin, p.begin + L};
          const uint32_t cn[2] = {L, R};
          for (int side = 0; side < 2; ++side) {
            const uint32_t heap = 2u * p.heap + 1u + (uint32_t)side;
            if (is_terminal(t, cn[side], nlevel, stall)) {
              record_terminal(t, c.begin + cbeg[side], cn[side], heap, nlevel);
            } else if (t.depth == 0 && nlevel >= t.max_levels) {
              set_status(t, ST_LEVEL_CAP);
            } else {
              const LCell ch{heap, 0u, (uint16_t)cbeg[side], (uint16_t)cn[side], 0, 0, (uint8_t)stall};
              if (nlive == 0) ch0 = ch; else ch1 = ch;
              ++nlive;
            }
          }
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan(nlive, tmp, &tot);
        if (nlive > 0) nc[run_out + ex] = ch0;
        if (nlive > 1) nc[run_out + ex + 1] = ch1;
        run_out += tot;
      }
      for (uint32_t i = tid; i < N; i += T) S.cellid[i] = kNoCell;
      if (tid == 0) {
        s_ncur = run_out;
        s_where = (uint32_t)nwhere;
      }
      __syncthreads();
      for (uint32_t j = warp; j < run_out; j += NW) {
        const uint32_t b = nc[j].begin, e = b + nc[j].count;
        for (uint32_t i = b + lane; i < e; i += 32) S.cellid[i] = (uint16_t)j;
      }
      __syncthreads();
      which ^= 1;
      level = nlevel;
    }

    // ---- write the permutation in final order
    for (uint32_t i = tid; i < N; i += T) t.out_perm[(int64_t)c.begin + i] = pm[ordA[i]];
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

cudaError_t prepare_subtree_kernel() {
  return cudaFuncSetAttribute(k_subtree, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSubtreeSmemBytes);
}

void launch_subtree(const TreeDev* trees, const Cell* list, uint32_t count, uint32_t* head, LCell* slices,
                    uint32_t slice_cells, uint32_t grid, uint64_t points, cudaStream_t st) {
  if (count == 0) return;
  cudaMemsetAsync(head, 0, sizeof(uint32_t), st);
  TraceScope ts(K_SUBTREE, st, points);
  k_subtree<<<grid, T, kSubtreeSmemBytes, st>>>(trees, list, count, head, slices, slice_cells);
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
