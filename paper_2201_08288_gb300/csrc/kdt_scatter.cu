// kdt_scatter.cu -- the stable partition of one level, with its loads staged
// through shared memory by the bulk-copy (TMA) engine and a producer warp.
//
// For every tile of a big cell (paper, Sec. 2: after a cell's split, its
// points go to the two children; ties go left), in sub-tiles of T points:
//   producer warp (warp 8): waits until one of two shared-memory buffers is
//     free ("empty" mbarrier), copies the sub-tile's metadata and its tree's
//     descriptor into shared memory, raises the buffer's expected byte count,
//     starts bulk copies (cp.async.bulk) of the aligned middle of every
//     coordinate column and of the permutation, copies the ragged 16-byte
//     edges with 4-byte cp.async (tracked by the same mbarrier), and arrives
//     on the buffer's "full" mbarrier; the next tile's record is loaded one
//     tile ahead;
//   consumer warps (0-7): wait for "full" (bounded), compute each point's
//     left/right flag from its key and its rank by warp ballots in position
//     order (so the partition is stable), store every value straight from
//     shared memory to its destination, and release the buffer.
// A child that is terminal receives only its permutation, in out_perm. For
// widest spread the consumers also reduce each child's min and max key per
// coordinate. Points of a cell arrive in subset order (contiguous segments),
// and a stable partition keeps that order in both children; where the subset
// changes, the consumers write where each big child's segments start (its
// left or right rank there), which is the children's subset offset table.
#include <algorithm>

#include "kdt_internal.cuh"
#include "kdt_launch.h"
#include "kdt_ptx.cuh"
#include "kdt_trace.h"

namespace kdt {

namespace {

constexpr int kCW = 8;                // consumer warps
constexpr int kCT = kCW * 32;         // consumer threads
constexpr int kST = kCT + 32;         // + one producer warp
constexpr int kMaxItems = 4;          // points per consumer thread in a sub-tile (T <= 1024)
constexpr uint32_t kBufBytes = kScatterSmemBytes / 2;
constexpr uint32_t kConsumerBar = 1;  // named barrier of the consumer warps

// Largest power-of-two sub-tile whose ncols columns (stride T + 4 words)
// fit one buffer.
__device__ __forceinline__ uint32_t sub_tile(int ncols) {
  uint32_t T = 1024;
  while (T > 32 && (uint32_t)ncols * (T + 4) * 4u > kBufBytes) T >>= 1;
  return T;
}

// What the consumers need about the sub-tile in a buffer.
struct SubMeta {
  TreeDev t;
  Cell cell;
  uint32_t tile, sub, mcnt, T, dim, mkey, L, loff, tile_start;
  uint32_t row[2];            // rows of the children's subset offsets (kNoRow: not a big child)
  uint32_t prev_sub;          // subset of the point before the sub-tile (~0u at the cell's start)
  uint32_t ph[kMaxDims + 1];  // alignment phase of each staged column
};

__global__ void __launch_bounds__(kST, 2) k_scatter_tma(const TreeDev* trees, StepDev s) {
  extern __shared__ __align__(128) uint32_t sm[];
  __shared__ __align__(8) uint64_t full[2], empty[2];
  __shared__ SubMeta meta[2];
  __shared__ uint32_t wcnt[kMaxItems][kCW];
  __shared__ uint32_t sedge[kMaxItems][kCW];  // subset of each warp's last point per round
  __shared__ uint32_t wmm[kCW][2][kMaxDims][2];
  __shared__ uint32_t s_fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t ntiles = *s.ntiles_total;
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], kCW);
    mbar_init(&empty[1], kCW);
    mbar_init_fence();
    s_fail = 0;
  }
  __syncthreads();

  if (warp == kCW) {
    // ================================================================ producer
    uint32_t ephase[2] = {0u, 0u};
    uint32_t k = 0;
    // the next tile's record and cell are loaded one tile ahead
    uint2 tl_next = blockIdx.x < ntiles ? s.tiles[blockIdx.x] : make_uint2(0, 0);
    Cell c_next = s.cells[tl_next.x];
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const uint2 tl = tl_next;
      const Cell c = c_next;
      if (tile + gridDim.x < ntiles) {
        tl_next = s.tiles[tile + gridDim.x];
        c_next = s.cells[tl_next.x];
      }
      const TreeDev& tg = trees[c.tree];
      const int d = tg.d, ncols = d + 1;
      const uint32_t T = sub_tile(ncols), stride = T + 4;
      const uint32_t tend = min(tl.y + (uint32_t)kTile, c.count);
      const float* X = src_cols(tg, c.level);
      const uint32_t* P = src_perm(tg, c.level);
      const uint32_t dim = s.kdim[tl.x], mkey = s.mkey[tl.x], L = s.lcount[tl.x], loff = s.tile_loff[tile];
      const uint2 cr0 = s.crow[2 * tl.x], cr1 = s.crow[2 * tl.x + 1];
      for (uint32_t sub = tl.y; sub < tend; sub += T, ++k) {
        const int b = k & 1;
        if (k >= 2) {
          if (!mbar_wait_bounded(&empty[b], ephase[b])) {
            if (lane == 0) atomicExch(&s_fail, 1u);
            return;
          }
          ephase[b] ^= 1u;
        }
        if (s_fail) return;
        const uint32_t mcnt = min(T, tend - sub);
        const uint32_t g0 = c.begin + sub;
        SubMeta& m = meta[b];
        // tree descriptor and sub-tile metadata
        for (uint32_t w = lane; w < sizeof(TreeDev) / 4; w += 32)
          ((uint32_t*)&m.t)[w] = ((const uint32_t*)&tg)[w];
        if (lane == 0) {
          m.cell = c;
          m.tile = tile;
          m.sub = sub;
          m.mcnt = mcnt;
          m.T = T;
          m.dim = dim;
          m.mkey = mkey;
          m.L = L;
          m.loff = loff;
          m.tile_start = tl.y;
          m.row[0] = cr0.x == kNoRow ? kNoRow : cr0.y;
          m.row[1] = cr1.x == kNoRow ? kNoRow : cr1.y;
          m.prev_sub = (sub > 0u && (cr0.x != kNoRow || cr1.x != kNoRow))
                           ? subset_at(tg, c.level, (int64_t)g0 - 1)
                           : 0xffffffffu;
        }
        uint32_t* A = sm + (size_t)b * (kBufBytes / 4);
        uint32_t total = 0;
        for (int c0 = 0; c0 < ncols; c0 += 32) {
          const int col = c0 + lane;
          uint32_t bytes = 0;
          if (col < ncols) {
            const uint32_t* src = col < d ? (const uint32_t*)(X + (int64_t)col * tg.n) : P;
            uint32_t ph = 0;
            if (src) {
              ph = (uint32_t)(((uintptr_t)(src + g0) >> 2) & 3u);
              const uint32_t a0 = min(g0 + ((4u - ph) & 3u), g0 + mcnt);
              bytes = ((g0 + mcnt - a0) & ~3u) * 4u;
            }
            m.ph[col] = ph;
          }
          total += __reduce_add_sync(0xffffffffu, bytes);
        }
        if (lane == 0) mbar_expect_tx(&full[b], total);
        __syncwarp();
        for (int c0 = 0; c0 < ncols; c0 += 32) {
          const int col = c0 + lane;
          if (col >= ncols) continue;
          const uint32_t* src = col < d ? (const uint32_t*)(X + (int64_t)col * tg.n) : P;
          if (!src) continue;  // level 0: the identity permutation, filled below
          uint32_t* dst = A + (size_t)col * stride;
          const uint32_t ph = (uint32_t)(((uintptr_t)(src + g0) >> 2) & 3u);
          const uint32_t a0 = min(g0 + ((4u - ph) & 3u), g0 + mcnt);
          const uint32_t a1 = a0 + ((g0 + mcnt - a0) & ~3u);
          if (a1 > a0) bulk_g2s(dst + ph + (a0 - g0), src + a0, (a1 - a0) * 4u, &full[b]);
          for (uint32_t idx = g0; idx < a0; ++idx) cp_async4(dst + ph + (idx - g0), src + idx);
          for (uint32_t idx = a1; idx < g0 + mcnt; ++idx) cp_async4(dst + ph + (idx - g0), src + idx);
        }
        if (!P)
          for (uint32_t i = lane; i < mcnt; i += 32) A[(size_t)d * stride + i] = g0 + i;
        cp_async_mbar_arrive(&full[b]);  // this lane's edge copies count toward the phase
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[b]);
      }
    }
    return;
  }

  // ================================================================== consumers
  const unsigned lt_mask = (1u << lane) - 1u;
  uint32_t fphase[2] = {0u, 0u};
  uint32_t lnext = 0, rnext = 0;
  bool saw_nan = false;
  uint32_t k = 0;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (bool more = true; more; ++k) {
      const int b = k & 1;
      if (!mbar_wait_bounded(&full[b], fphase[b])) atomicExch(&s_fail, 1u);
      fphase[b] ^= 1u;
      named_sync(kConsumerBar, kCT);
      if (s_fail) return;
      const SubMeta& m = meta[b];
      const TreeDev& t = m.t;
      const Cell& cell = m.cell;
      const int level = cell.level;
      const int d = t.d;
      const int64_t n = t.n;
      const uint32_t T = m.T, stride = T + 4, mcnt = m.mcnt, L = m.L;
      const uint32_t tend = min(m.tile_start + (uint32_t)kTile, cell.count);
      const int child_stall = (cell.count == L) ? cell.stall + 1 : 0;
      const bool term_left = is_terminal(t, L, level + 1, child_stall);
      const bool term_right = is_terminal(t, cell.count - L, level + 1, child_stall);
      const bool want_mm = t.key_rule == KEY_WIDEST && !(term_left && term_right);
      const bool explicit_sid = t.subset_mode == SUB_EXPLICIT;
      const uint32_t g0 = cell.begin + m.sub;
      if (m.sub == m.tile_start) {
        lnext = cell.begin + m.loff;
        rnext = cell.begin + L + (m.tile_start - m.loff);
        if (want_mm)
          for (int j = lane; j < 2 * d * 2; j += 32) {
            const int side = j / (2 * d), l = (j / 2) % d, which = j & 1;
            wmm[warp][side][l][which] = which ? 0u : 0xffffffffu;
          }
      }
      uint32_t sidv[kMaxItems];
      if (explicit_sid) {
        const void* S = src_sid(t, level);
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
          const uint32_t i = tid + q * kCT;
          sidv[q] = 0;
          if (i < mcnt)
            sidv[q] = t.sid_bytes == 1 ? (uint32_t)((const uint8_t*)S)[g0 + i]
                                       : (uint32_t)((const uint16_t*)S)[g0 + i];
        }
      }
      const uint32_t* A = sm + (size_t)b * (kBufBytes / 4);

      // ---- flags and ranks (position order); subsets where offsets are kept
      bool left[kMaxItems];
      unsigned bal[kMaxItems];
      uint32_t sv[kMaxItems];
      const bool want_off = m.row[0] != kNoRow || m.row[1] != kNoRow;
      const uint32_t* keycol = A + (size_t)m.dim * stride + m.ph[m.dim];
      const uint32_t* pa = A + (size_t)d * stride + m.ph[d];
#pragma unroll
      for (int q = 0; q < kMaxItems; ++q) {
        const uint32_t i = tid + q * kCT;
        left[q] = i < mcnt && ord_key(__uint_as_float(keycol[i])) <= m.mkey;
        bal[q] = __ballot_sync(0xffffffffu, left[q]);
        if (lane == 0) wcnt[q][warp] = __popc(bal[q]);
        sv[q] = 0;
        if (want_off) {
          if (i < mcnt) sv[q] = explicit_sid ? min(sidv[q], (uint32_t)t.r - 1u) : subset_from_orig(t, pa[i]);
          if (lane == 31) sedge[q][warp] = sv[q];
        }
      }
      named_sync(kConsumerBar, kCT);
      uint32_t dst[kMaxItems], lrk[kMaxItems];
      uint32_t nL = 0;
#pragma unroll
      for (int q = 0; q < kMaxItems; ++q) {
        uint32_t below = 0, round = 0;
#pragma unroll
        for (int w = 0; w < kCW; ++w) {
          const uint32_t v = wcnt[q][w];
          below += (w < warp) ? v : 0u;
          round += v;
        }
        const uint32_t i = tid + q * kCT;
        const uint32_t lr = nL + below + __popc(bal[q] & lt_mask);
        dst[q] = left[q] ? lnext + lr : rnext + (i - lr);
        lrk[q] = lnext - cell.begin + lr;  // points of the cell before this one that go left
        nL += round;
      }

      // ---- stores, straight from shared memory
      {
        const uint32_t* a = A + (size_t)d * stride + m.ph[d];
        uint32_t* Po = t.pbuf[level & 1];
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
          const uint32_t i = tid + q * kCT;
          if (i >= mcnt) continue;
          if (left[q] ? term_left : term_right)
            t.out_perm[dst[q]] = a[i];
          else
            Po[dst[q]] = a[i];
        }
      }
      for (int c = 0; c < d; ++c) {
        const uint32_t* a = A + (size_t)c * stride + m.ph[c];
        float* out = t.xbuf[level & 1] + (int64_t)c * n;
        uint32_t lmin = 0xffffffffu, lmax = 0u, rmin = 0xffffffffu, rmax = 0u;
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
          const uint32_t i = tid + q * kCT;
          if (i >= mcnt) continue;
          const uint32_t v = a[i];
          if (level == 0) saw_nan |= is_nan_bits(__uint_as_float(v));
          if (left[q] ? term_left : term_right) continue;
          out[dst[q]] = __uint_as_float(v);
          if (want_mm) {
            const uint32_t key = ord_key(__uint_as_float(v));
            if (left[q]) {
              lmin = min(lmin, key);
              lmax = max(lmax, key);
            } else {
              rmin = min(rmin, key);
              rmax = max(rmax, key);
            }
          }
        }
        if (want_mm) {
          lmin = __reduce_min_sync(0xffffffffu, lmin);
          lmax = __reduce_max_sync(0xffffffffu, lmax);
          rmin = __reduce_min_sync(0xffffffffu, rmin);
          rmax = __reduce_max_sync(0xffffffffu, rmax);
          if (lane == 0) {
            wmm[warp][0][c][0] = min(wmm[warp][0][c][0], lmin);
            wmm[warp][0][c][1] = max(wmm[warp][0][c][1], lmax);
            wmm[warp][1][c][0] = min(wmm[warp][1][c][0], rmin);
            wmm[warp][1][c][1] = max(wmm[warp][1][c][1], rmax);
          }
        }
      }
      if (explicit_sid) {
        void* So = t.sbuf[level & 1];
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
          const uint32_t i = tid + q * kCT;
          if (i >= mcnt || (left[q] ? term_left : term_right)) continue;
          if (t.sid_bytes == 1)
            ((uint8_t*)So)[dst[q]] = (uint8_t)sidv[q];
          else
            ((uint16_t*)So)[dst[q]] = (uint16_t)sidv[q];
        }
      }
      // ---- subset offsets of the big children, at the segment starts
      // (each row holds r + 1 words below off_cap, checked when it was handed out)
      if (want_off) {
        const uint32_t r = (uint32_t)t.r;
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
          const uint32_t i = tid + q * kCT;
          const uint32_t p = m.sub + i;  // position in the cell
          int32_t sp = __shfl_up_sync(0xffffffffu, (int32_t)sv[q], 1);
          if (lane == 0)
            sp = (int32_t)(warp > 0 ? sedge[q][warp - 1] : (q > 0 ? sedge[q - 1][kCW - 1] : m.prev_sub));
          if (i >= mcnt) continue;
          if ((int32_t)sv[q] != sp)
            for (uint32_t u = (uint32_t)(sp + 1); u <= sv[q]; ++u) {
              if (m.row[0] != kNoRow) s.off_next[m.row[0] + u] = lrk[q];
              if (m.row[1] != kNoRow) s.off_next[m.row[1] + u] = p - lrk[q];
            }
          if (p + 1 == cell.count)
            for (uint32_t u = sv[q] + 1; u <= r; ++u) {
              if (m.row[0] != kNoRow) s.off_next[m.row[0] + u] = L;
              if (m.row[1] != kNoRow) s.off_next[m.row[1] + u] = cell.count - L;
            }
        }
      }
      lnext += nL;
      rnext += mcnt - nL;
      more = m.sub + T < tend;
      if (!more) {  // last sub-tile of the tile
        if (saw_nan) set_status(t, ST_NAN_INPUT);
        saw_nan = false;
        if (want_mm) {
          named_sync(kConsumerBar, kCT);
          for (int j = tid; j < 2 * d * 2; j += kCT) {
            const int side = j / (2 * d), l = (j / 2) % d, which = j & 1;
            uint32_t v = wmm[0][side][l][which];
            for (int w = 1; w < kCW; ++w) {
              const uint32_t u = wmm[w][side][l][which];
              v = which ? max(v, u) : min(v, u);
            }
            s.tile_mm[(((size_t)m.tile * 2 + side) * kMaxDims + l) * 2 + which] = v;
          }
        }
      }
      // ---- release the buffer (reads of it precede the next bulk writes)
      fence_proxy_async_smem();
      named_sync(kConsumerBar, kCT);
      if (lane == 0) mbar_arrive(&empty[b]);
    }
  }
}

}  // namespace

cudaError_t prepare_scatter_kernel() {
  return cudaFuncSetAttribute(k_scatter_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kScatterSmemBytes);
}

void launch_scatter(const TreeDev* trees, const StepDev& s, uint32_t max_tiles, uint32_t grid_cap,
                    uint64_t points, cudaStream_t st) {
  TraceScope ts(K_PART_SCATTER, st, points);
  const uint32_t grid = std::max<uint32_t>(1, std::min(max_tiles, grid_cap));
  k_scatter_tma<<<grid, kST, kScatterSmemBytes, st>>>(trees, s);
}

}  // namespace kdt
