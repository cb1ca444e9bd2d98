// kdt_scatter.cu -- the stable partition of one level, with its loads staged
// through shared memory by the bulk-copy (TMA) engine and a producer warp.
//
// For every tile of a big cell (paper, Sec. 2: after a cell's split, its
// points go to the two children; ties go left), in sub-tiles of T points:
//   producer warp (warp 8): waits until one of two shared-memory buffers is
//     free ("empty" mbarrier), writes the sub-tile's metadata (output
//     pointers, which children are terminal, what to compute), raises the
//     buffer's expected byte count, starts bulk copies (cp.async.bulk) of
//     the aligned middle of every coordinate column, of the permutation and
//     of the subset ids, copies the ragged 16-byte edges (4-byte cp.async for
//     word columns, plain loads for the ids) and arrives on the buffer's
//     "full" mbarrier; the next tile's record is loaded one tile ahead;
//   consumer warps (0-7): wait for "full" (bounded), compute each point's
//     left/right flag from its key and its rank by warp ballots in position
//     order (so the partition is stable), store every value straight from
//     shared memory to its destination, two columns at a time, and release
//     the buffer.
// A child that is terminal receives only its permutation, in out_perm. For
// widest spread the consumers also reduce each child's min and max key per
// coordinate (per warp, then one shared-memory reduction per warp and
// column, fire-and-forget). Points of a cell arrive in subset order
// (contiguous segments), and a stable partition keeps that order in both
// children; where the subset changes, the consumers write where each big
// child's segments start (its left or right rank there), which is the
// children's subset offset table.
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

// Largest power-of-two sub-tile whose ncols word columns (stride T + 4) and
// an id column of sid_bytes per point (T + 32 entries) fit one buffer.
__device__ __forceinline__ uint32_t sub_tile(int ncols, int sid_bytes) {
  uint32_t T = 1024;
  while (T > 32 && (uint32_t)ncols * (T + 4) * 4u + (T + 32) * (uint32_t)sid_bytes > kBufBytes) T >>= 1;
  return T;
}

// What the consumers need about the sub-tile in a buffer.
struct SubMeta {
  float* xout;         // coordinate columns of the next level
  uint32_t* pout;      // permutation of the next level
  void* sout;          // subset ids of the next level (explicit ids)
  uint32_t* out_perm;  // final permutation (terminal children)
  int32_t* status;
  int64_t n;
  uint32_t cell_begin, cell_count, cell_idx, tile, sub, mcnt, T, dim, mkey, L, loff, tile_start;
  uint32_t row[2];     // rows of the children's subset offsets (kNoRow: not a big child)
  uint32_t prev_sub;   // subset of the point before the CTA's first sub-tile (~0u at a cell's start)
  uint32_t r, subset_mode, sid_bytes, sid_ph, tn;
  int32_t d;
  uint8_t term_left, term_right, want_mm, want_off, nan_check;
  uint8_t run_more;  // this CTA's next tile is of the same cell (its min / max run goes on)
  uint8_t pad1, pad2;
  uint32_t ph[kMaxDims + 1];  // alignment phase of each staged word column
};

__device__ __forceinline__ uint32_t meta_subset(const SubMeta& m, uint32_t orig) {
  if (m.subset_mode == SUB_MOD) return orig % m.r;
  return (uint32_t)(((uint64_t)orig * (uint64_t)m.r) / (uint64_t)m.tn);
}

// kD > 0: compiled for trees of kD coordinates (the column loops unroll);
// kD = 0: any d.
template <int kD>
__global__ void __launch_bounds__(kST, 2) k_scatter_tma(const TreeDev* trees, StepDev s) {
  extern __shared__ __align__(128) uint32_t sm[];
  __shared__ __align__(8) uint64_t full[2], empty[2];
  __shared__ SubMeta meta[2];
  __shared__ uint32_t wcnt[kMaxItems][kCW];
  __shared__ uint32_t sedge[kMaxItems][kCW];  // subset of each warp's last point per round
  __shared__ unsigned wbal[kMaxItems][kCW];   // each (round, warp) block's left flags (explicit ids)
  __shared__ uint32_t tmm[2][kMaxDims][2];    // this CTA's run of tiles of one cell: per child,
                                              // min / max key per coordinate
  __shared__ uint32_t s_fail;
  __shared__ uint32_t s_carry;  // subset of the last point of the sub-tile the consumers finished last
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t ntiles = *s.ntiles_total;
  // this CTA's contiguous range of tiles: consecutive tiles mostly share a
  // cell, so the per-cell min / max stay in the CTA for long runs
  const uint32_t t_begin = (uint32_t)(((uint64_t)blockIdx.x * ntiles) / gridDim.x);
  const uint32_t t_end = (uint32_t)(((uint64_t)(blockIdx.x + 1) * ntiles) / gridDim.x);
  for (int j = tid; j < 2 * kMaxDims * 2; j += kST) (&tmm[0][0][0])[j] = (j & 1) ? 0u : 0xffffffffu;
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
    uint32_t ephase = 0u;  // bit b: parity of buffer b's next "empty" phase
    uint32_t k = 0;
    // the next tile's record and cell are loaded one tile ahead
    uint2 tl_next = t_begin < t_end ? s.tiles[t_begin] : make_uint2(0, 0);
    Cell c_next = s.cells[tl_next.x];
    for (uint32_t tile = t_begin; tile < t_end; ++tile) {
      const uint2 tl = tl_next;
      const Cell c = c_next;
      if (tile + 1 < t_end) {
        tl_next = s.tiles[tile + 1];
        c_next = s.cells[tl_next.x];
      }
      const bool run_more = tile + 1 < t_end && tl_next.x == tl.x;
      const TreeDev& tg = trees[c.tree];
      const int d = kD > 0 ? kD : tg.d, ncols = d + 1;
      const bool expl = tg.subset_mode == SUB_EXPLICIT;
      const int es = expl ? tg.sid_bytes : 0;
      const uint32_t T = sub_tile(ncols, es), stride = T + 4;
      const uint32_t tend = min(tl.y + (uint32_t)kTile, c.count);
      const float* X = src_cols(tg, c.level);
      const uint32_t* P = src_perm(tg, c.level);
      const uint8_t* SID = (const uint8_t*)src_sid(tg, c.level);
      const uint32_t dim = s.kdim[tl.x], mkey = s.mkey[tl.x], L = s.lcount[tl.x], loff = s.tile_loff[tile];
      const uint2 cr0 = s.crow[2 * tl.x], cr1 = s.crow[2 * tl.x + 1];
      const int child_stall = (c.count == L) ? c.stall + 1 : 0;
      const bool term_left = is_terminal(tg, L, c.level + 1, child_stall);
      const bool term_right = is_terminal(tg, c.count - L, c.level + 1, child_stall);
      for (uint32_t sub = tl.y; sub < tend; sub += T, ++k) {
        const int b = k & 1;
        if (k >= 2) {
          if (!mbar_wait_bounded(&empty[b], (ephase >> b) & 1u)) {
            if (lane == 0) atomicExch(&s_fail, 1u);
            return;
          }
          ephase ^= 1u << b;
        }
        if (s_fail) return;
        const uint32_t mcnt = min(T, tend - sub);
        const uint32_t g0 = c.begin + sub;
        SubMeta& m = meta[b];
        uint32_t* A = sm + (size_t)b * (kBufBytes / 4);
        uint8_t* SA = (uint8_t*)(A + (size_t)ncols * stride);  // 16-byte aligned (stride * 4 is)
        // id column: 16-byte phase in elements, aligned middle [sa0, sa1)
        uint32_t sph = 0, sa0 = g0, sa1 = g0;
        if (expl) {
          const uint32_t per16 = 16u / (uint32_t)es;
          sph = (uint32_t)(((uintptr_t)(SID + (size_t)g0 * es) / (uintptr_t)es) & (per16 - 1u));
          sa0 = min(g0 + ((per16 - sph) & (per16 - 1u)), g0 + mcnt);
          sa1 = sa0 + ((g0 + mcnt - sa0) & ~(per16 - 1u));
        }
        if (lane == 0) {
          m.xout = tg.xbuf[c.level & 1];
          m.pout = tg.pbuf[c.level & 1];
          m.sout = tg.sbuf[c.level & 1];
          m.out_perm = tg.out_perm;
          m.status = tg.status;
          m.n = tg.n;
          m.cell_begin = c.begin;
          m.cell_count = c.count;
          m.cell_idx = tl.x;
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
          m.r = (uint32_t)tg.r;
          m.subset_mode = (uint32_t)tg.subset_mode;
          m.sid_bytes = (uint32_t)es;
          m.sid_ph = sph;
          m.tn = (uint32_t)tg.n;
          m.d = d;
          m.term_left = term_left;
          m.term_right = term_right;
          m.want_mm = tg.key_rule == KEY_WIDEST && !(term_left && term_right);
          m.want_off = cr0.x != kNoRow || cr1.x != kNoRow;
          // the input's NaN check: the root's first pass over its columns (a
          // presorted root's presort checks them)
          m.nan_check = c.level == 0 && !tg.presorted;
          m.run_more = run_more;
        }
        uint32_t total = expl ? (sa1 - sa0) * (uint32_t)es : 0u;
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
          if (!src) continue;  // level 0 without a presort: the identity permutation, filled below
          uint32_t* dst = A + (size_t)col * stride;
          const uint32_t ph = (uint32_t)(((uintptr_t)(src + g0) >> 2) & 3u);
          const uint32_t a0 = min(g0 + ((4u - ph) & 3u), g0 + mcnt);
          const uint32_t a1 = a0 + ((g0 + mcnt - a0) & ~3u);
          if (a1 > a0) bulk_g2s(dst + ph + (a0 - g0), src + a0, (a1 - a0) * 4u, &full[b]);
          for (uint32_t idx = g0; idx < a0; ++idx) cp_async4(dst + ph + (idx - g0), src + idx);
          for (uint32_t idx = a1; idx < g0 + mcnt; ++idx) cp_async4(dst + ph + (idx - g0), src + idx);
        }
        if (expl) {
          if (lane == 0 && sa1 > sa0)
            bulk_g2s(SA + (size_t)(sph + sa0 - g0) * es, SID + (size_t)sa0 * es, (sa1 - sa0) * (uint32_t)es,
                     &full[b]);
          // ragged ends of the id column: fewer than 16 bytes each, plain loads
          const uint32_t nlo = sa0 - g0, nhi = g0 + mcnt - sa1;
          if ((uint32_t)lane < nlo + nhi) {
            const uint32_t idx = (uint32_t)lane < nlo ? g0 + lane : sa1 + (lane - nlo);
            if (es == 1)
              SA[sph + idx - g0] = SID[idx];
            else
              ((uint16_t*)SA)[sph + idx - g0] = ((const uint16_t*)SID)[idx];
          }
        }
        if (!P)
          for (uint32_t i = lane; i < mcnt; i += 32) A[(size_t)d * stride + i] = g0 + i;
        // the subset of the point before the CTA's first sub-tile, if that is
        // not a cell's start: one global load per CTA (each later sub-tile
        // follows the one before it in the same cell, whose last subset the
        // consumers keep)
        if (lane == 0)
          m.prev_sub = (k == 0 && sub > 0u && (cr0.x != kNoRow || cr1.x != kNoRow))
                           ? subset_at(tg, c.level, (int64_t)g0 - 1)
                           : 0xffffffffu;
        cp_async_mbar_arrive(&full[b]);  // this lane's edge copies count toward the phase
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[b]);
      }
    }
    return;
  }

  // ================================================================== consumers
  const unsigned lt_mask = (1u << lane) - 1u;
  uint32_t fphase = 0u;  // bit b: parity of buffer b's next "full" phase
  uint32_t lnext = 0, rnext = 0;
  bool saw_nan = false;
  // For a compile-time d of at most 8 every lane keeps the min / max of its
  // points per coordinate and child over the whole run of the cell's tiles
  // (registers), reduced over the warp once at the run's end; otherwise the
  // warps reduce after every sub-tile.
  constexpr bool kAcc = kD > 0 && kD <= 8;
  constexpr int kAD = kAcc ? kD : 1;
  const float inf = __int_as_float(0x7f800000);
  float acc[kAD][2][2];  // [coordinate][child][min, max]
#pragma unroll
  for (int l = 0; l < kAD; ++l)
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      acc[l][side][0] = inf;
      acc[l][side][1] = -inf;
    }
  uint32_t k = 0;
  for (uint32_t tile = t_begin; tile < t_end; ++tile) {
    for (bool more = true; more; ++k) {
      const int b = k & 1;
      // one consumer thread waits for the sub-tile (a waiting thread keeps
      // issuing try_wait); the named barrier parks the others and makes what
      // the copies wrote visible to them
      if (tid == 0 && !mbar_wait_bounded(&full[b], (fphase >> b) & 1u)) atomicExch(&s_fail, 1u);
      fphase ^= 1u << b;
      named_sync(kConsumerBar, kCT);
      if (s_fail) return;
      const SubMeta& m = meta[b];
      const int d = kD > 0 ? kD : m.d;
      const int64_t n = m.n;
      const uint32_t T = m.T, stride = T + 4, mcnt = m.mcnt, L = m.L;
      const uint32_t cbeg = m.cell_begin, ccount = m.cell_count;
      const uint32_t tend = min(m.tile_start + (uint32_t)kTile, ccount);
      const bool term_left = m.term_left, term_right = m.term_right;
      const bool want_mm = m.want_mm, want_off = m.want_off, nan_check = m.nan_check;
      const bool explicit_sid = m.sid_bytes != 0;
      // subset of the point before this sub-tile (~0u at the cell's start):
      // the CTA's sub-tiles run in position order, so after its first one it
      // is the last subset of the previous sub-tile (read here, before this
      // sub-tile's second consumer barrier; rewritten after it)
      const uint32_t prev_sub = m.sub == 0u ? 0xffffffffu : (k == 0 ? m.prev_sub : s_carry);
      if (m.sub == m.tile_start) {
        lnext = cbeg + m.loff;
        rnext = cbeg + L + (m.tile_start - m.loff);
      }
      const uint32_t* A = sm + (size_t)b * (kBufBytes / 4);
      const uint8_t* SA = (const uint8_t*)(A + (size_t)(d + 1) * stride) + (size_t)m.sid_ph * m.sid_bytes;
      auto sid_of = [&](uint32_t i) -> uint32_t {
        const uint32_t v = m.sid_bytes == 1 ? (uint32_t)SA[i] : (uint32_t)((const uint16_t*)SA)[i];
        return min(v, m.r - 1u);
      };

      // ---- flags and ranks (position order); subsets where offsets are kept
      bool left[kMaxItems];
      unsigned bal[kMaxItems];
      uint32_t sv[kMaxItems];
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
          if (explicit_sid) {
            if (lane == 0) wbal[q][warp] = bal[q];
          } else {
            if (i < mcnt) sv[q] = meta_subset(m, pa[i]);
            if (lane == 31) sedge[q][warp] = sv[q];
          }
        }
      }
      named_sync(kConsumerBar, kCT);
      // left points before each (round, warp) block: one scan over the
      // kMaxItems * kCW = 32 block counts in position order
      static_assert(kMaxItems * kCW == 32, "one lane per (round, warp) block");
      const uint32_t wv = (&wcnt[0][0])[lane];
      const uint32_t winc = warp_incl_scan(wv);
      const uint32_t wexc = winc - wv;
      const uint32_t nL = __shfl_sync(0xffffffffu, winc, 31);
      uint32_t dst[kMaxItems], lrk[kMaxItems];
      bool keep[kMaxItems];  // the point's child is not terminal: its columns move
#pragma unroll
      for (int q = 0; q < kMaxItems; ++q) {
        const uint32_t i = tid + q * kCT;
        const uint32_t lr = __shfl_sync(0xffffffffu, wexc, q * kCW + warp) + __popc(bal[q] & lt_mask);
        dst[q] = left[q] ? lnext + lr : rnext + (i - lr);
        lrk[q] = lnext - cbeg + lr;  // points of the cell before this one that go left
        keep[q] = i < mcnt && !(left[q] ? term_left : term_right);
      }

      // ---- permutation
#pragma unroll
      for (int q = 0; q < kMaxItems; ++q) {
        const uint32_t i = tid + q * kCT;
        if (i >= mcnt) continue;
        if (keep[q])
          m.pout[dst[q]] = pa[i];
        else
          m.out_perm[dst[q]] = pa[i];
      }

      // ---- coordinate columns, two at a time, straight from shared memory
#pragma unroll
      for (int c = 0; c < d; c += 2) {
        const bool two = c + 1 < d;
        const uint32_t* a0 = A + (size_t)c * stride + m.ph[c];
        const uint32_t* a1 = two ? A + (size_t)(c + 1) * stride + m.ph[c + 1] : a0;
        float* o0 = m.xout + (int64_t)c * n;
        float* o1 = m.xout + (int64_t)(c + 1) * n;
        uint32_t v0[kMaxItems], v1[kMaxItems];
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
          const uint32_t i = tid + q * kCT;
          v0[q] = i < mcnt ? a0[i] : 0u;
          v1[q] = i < mcnt ? a1[i] : 0u;
        }
        if (nan_check)
#pragma unroll
          for (int q = 0; q < kMaxItems; ++q)
            saw_nan |= (tid + q * kCT < mcnt) &&
                       (is_nan_bits(__uint_as_float(v0[q])) || is_nan_bits(__uint_as_float(v1[q])));
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q)
          if (keep[q]) {
            o0[dst[q]] = __uint_as_float(v0[q]);
            if (two) o1[dst[q]] = __uint_as_float(v1[q]);
          }
        if (want_mm && kAcc) {
          // min / max as floats (the widest rule only uses max - min, which -0
          // and +0 do not change); keys are formed at the run's end
          const int c1 = two ? c + 1 : c;
#pragma unroll
          for (int q = 0; q < kMaxItems; ++q)
            if (keep[q]) {
              const float x0 = __uint_as_float(v0[q]), x1 = __uint_as_float(v1[q]);
              const int side = left[q] ? 0 : 1;
              if (side == 0) {
                acc[c % kAD][0][0] = fminf(acc[c % kAD][0][0], x0);
                acc[c % kAD][0][1] = fmaxf(acc[c % kAD][0][1], x0);
                if (two) {
                  acc[c1 % kAD][0][0] = fminf(acc[c1 % kAD][0][0], x1);
                  acc[c1 % kAD][0][1] = fmaxf(acc[c1 % kAD][0][1], x1);
                }
              } else {
                acc[c % kAD][1][0] = fminf(acc[c % kAD][1][0], x0);
                acc[c % kAD][1][1] = fmaxf(acc[c % kAD][1][1], x0);
                if (two) {
                  acc[c1 % kAD][1][0] = fminf(acc[c1 % kAD][1][0], x1);
                  acc[c1 % kAD][1][1] = fmaxf(acc[c1 % kAD][1][1], x1);
                }
              }
            }
        } else if (want_mm) {
          // min / max as floats, then keys once per warp and sub-tile
          float mm[2][2][2] = {{{inf, -inf}, {inf, -inf}}, {{inf, -inf}, {inf, -inf}}};  // [col][side][min,max]
#pragma unroll
          for (int q = 0; q < kMaxItems; ++q)
            if (keep[q]) {
              const float x0 = __uint_as_float(v0[q]), x1 = __uint_as_float(v1[q]);
              if (left[q]) {
                mm[0][0][0] = fminf(mm[0][0][0], x0);
                mm[0][0][1] = fmaxf(mm[0][0][1], x0);
                mm[1][0][0] = fminf(mm[1][0][0], x1);
                mm[1][0][1] = fmaxf(mm[1][0][1], x1);
              } else {
                mm[0][1][0] = fminf(mm[0][1][0], x0);
                mm[0][1][1] = fmaxf(mm[0][1][1], x0);
                mm[1][1][0] = fminf(mm[1][1][0], x1);
                mm[1][1][1] = fmaxf(mm[1][1][1], x1);
              }
            }
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            if (cc == 1 && !two) break;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
              const uint32_t lo = __reduce_min_sync(0xffffffffu, ord_key(mm[cc][side][0]));
              const uint32_t hi = __reduce_max_sync(0xffffffffu, ord_key(mm[cc][side][1]));
              if (lane == 0) {
                atomic_min_shared(&tmm[side][c + cc][0], lo);
                atomic_max_shared(&tmm[side][c + cc][1], hi);
              }
            }
          }
        }
      }
      if (explicit_sid) {
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
          const uint32_t i = tid + q * kCT;
          if (!keep[q]) continue;
          if (m.sid_bytes == 1)
            ((uint8_t*)m.sout)[dst[q]] = SA[i];
          else
            ((uint16_t*)m.sout)[dst[q]] = ((const uint16_t*)SA)[i];
        }
      }
      // ---- subset offsets of the big children, at the segment starts
      // (each row holds r + 1 words below off_cap, checked when it was handed out)
      if (want_off && explicit_sid) {
        // thread tid checks positions 4 tid .. 4 tid + 3 against the one before
        // each, reading the staged ids; only a warp holding a subset change or
        // the cell's last point goes on, taking the left rank of a position
        // from its block's count scan and left-flag ballot
        const uint32_t r = m.r, i0 = 4u * (uint32_t)tid;
        uint32_t v[5];
        v[0] = i0 == 0u ? prev_sub : sid_of(i0 - 1u);
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j + 1] = i0 + j < mcnt ? sid_of(i0 + j) : v[j];
        if (i0 < mcnt && i0 + 4u >= mcnt) s_carry = v[4];  // the sub-tile's last subset
        bool any = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) any |= i0 + j < mcnt && (v[j] != v[j + 1] || m.sub + i0 + j + 1u == ccount);
        if (__any_sync(0xffffffffu, any)) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint32_t i = i0 + j;
            const uint32_t blk = ((i / kCT) * kCW + ((i % kCT) >> 5)) & 31u;  // i < kMaxItems kCT
            const uint32_t lr = __shfl_sync(0xffffffffu, wexc, blk) +
                                __popc((&wbal[0][0])[blk] & ((1u << (i & 31u)) - 1u));
            if (i >= mcnt) continue;
            const uint32_t p = m.sub + i, lk = lnext - cbeg + lr;  // left points of the cell before i
            for (int32_t u = (int32_t)v[j] + 1; u <= (int32_t)v[j + 1]; ++u) {
              if (m.row[0] != kNoRow) s.off_next[m.row[0] + u] = lk;
              if (m.row[1] != kNoRow) s.off_next[m.row[1] + u] = p - lk;
            }
            if (p + 1 == ccount)
              for (uint32_t u = v[j + 1] + 1; u <= r; ++u) {
                if (m.row[0] != kNoRow) s.off_next[m.row[0] + u] = L;
                if (m.row[1] != kNoRow) s.off_next[m.row[1] + u] = ccount - L;
              }
          }
        }
      } else if (want_off) {
        const uint32_t r = m.r;
#pragma unroll
        for (int q = 0; q < kMaxItems; ++q) {
          const uint32_t i = tid + q * kCT;
          const uint32_t p = m.sub + i;  // position in the cell
          int32_t sp = __shfl_up_sync(0xffffffffu, (int32_t)sv[q], 1);
          if (lane == 0)
            sp = (int32_t)(warp > 0 ? sedge[q][warp - 1] : (q > 0 ? sedge[q - 1][kCW - 1] : prev_sub));
          if (i >= mcnt) continue;
          if (i + 1 == mcnt) s_carry = sv[q];
          if ((int32_t)sv[q] != sp)
            for (uint32_t u = (uint32_t)(sp + 1); u <= sv[q]; ++u) {
              if (m.row[0] != kNoRow) s.off_next[m.row[0] + u] = lrk[q];
              if (m.row[1] != kNoRow) s.off_next[m.row[1] + u] = p - lrk[q];
            }
          if (p + 1 == ccount)
            for (uint32_t u = sv[q] + 1; u <= r; ++u) {
              if (m.row[0] != kNoRow) s.off_next[m.row[0] + u] = L;
              if (m.row[1] != kNoRow) s.off_next[m.row[1] + u] = ccount - L;
            }
        }
      }
      lnext += nL;
      rnext += mcnt - nL;
      more = m.sub + T < tend;
      if (!more) {  // last sub-tile of the tile
        if (saw_nan) atomicCAS(m.status, ST_OK, ST_NAN_INPUT);
        saw_nan = false;
        if (want_mm) {
          // keep reducing while this CTA's next tile is of the same cell (the
          // producer, which reads the tile list ahead, says so); else add the
          // run's min / max to the cell's with atomics
          if (!m.run_more) {
            if (kAcc) {
              // transpose-reduce over the warp: value u = (l * 2 + side) * 2 +
              // which, maxima negated so that every step is a minimum; after
              // the steps lane u holds value u reduced over all 32 lanes
              constexpr int kV = 4 * kAD;
              constexpr int kVP = kV <= 8 ? 8 : (kV <= 16 ? 16 : 32);
              float v[kVP];
#pragma unroll
              for (int u = 0; u < kVP; ++u) {
                const int l = u / 4, side = (u / 2) & 1, which = u & 1;
                v[u] = u >= kV ? inf : (which ? -acc[l % kAD][side][1] : acc[l % kAD][side][0]);
              }
#pragma unroll
              for (int h = kVP / 2; h >= 1; h >>= 1) {
                const bool upper = (lane & h) != 0;
#pragma unroll
                for (int i = 0; i < h; ++i) {
                  const float keep = upper ? v[i + h] : v[i];
                  const float send = upper ? v[i] : v[i + h];
                  v[i] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, h));
                }
              }
#pragma unroll
              for (int o = kVP; o < 32; o <<= 1) v[0] = fminf(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
              if (lane < kV) {
                const int l = lane / 4, side = (lane / 2) & 1;
                if (lane & 1)
                  atomic_max_shared(&tmm[side][l][1], ord_key(-v[0]));
                else
                  atomic_min_shared(&tmm[side][l][0], ord_key(v[0]));
              }
#pragma unroll
              for (int l = 0; l < kAD; ++l)
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                  acc[l][side][0] = inf;
                  acc[l][side][1] = -inf;
                }
            }
            named_sync(kConsumerBar, kCT);
            // add the run's min / max to the cell's; reset the table
            for (int j = tid; j < 4 * d; j += kCT) {
              const int side = j / (2 * d), l = (j / 2) % d, which = j & 1;
              uint32_t* dst = &s.child_mm[(((size_t)m.cell_idx * 2 + side) * kMaxDims + l) * 2 + which];
              if (which) atomicMax(dst, tmm[side][l][which]); else atomicMin(dst, tmm[side][l][which]);
              tmm[side][l][which] = which ? 0u : 0xffffffffu;
            }
          }
        }
      }
      // ---- release the buffer: each warp's reads of it precede the next bulk
      // writes; the "empty" barrier counts the consumer warps (the next
      // sub-tile's first barrier orders the reuse of wcnt and sedge)
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[b]);
    }
  }
}

}  // namespace

template <int kD>
cudaError_t prepare_one() {
  return cudaFuncSetAttribute(k_scatter_tma<kD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmemBytes);
}

cudaError_t prepare_scatter_kernel() {
  for (cudaError_t e : {prepare_one<0>(), prepare_one<2>(), prepare_one<3>(), prepare_one<8>(), prepare_one<16>()})
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

void launch_scatter(const TreeDev* trees, const StepDev& s, uint32_t max_tiles, uint32_t grid_cap,
                    uint64_t points, int uniform_d, cudaStream_t st) {
  TraceScope ts(K_PART_SCATTER, st, points);
  const uint32_t grid = std::max<uint32_t>(1, std::min(max_tiles, grid_cap));
  switch (uniform_d) {
    case 2: k_scatter_tma<2><<<grid, kST, kScatterSmemBytes, st>>>(trees, s); break;
    case 3: k_scatter_tma<3><<<grid, kST, kScatterSmemBytes, st>>>(trees, s); break;
    case 8: k_scatter_tma<8><<<grid, kST, kScatterSmemBytes, st>>>(trees, s); break;
    case 16: k_scatter_tma<16><<<grid, kST, kScatterSmemBytes, st>>>(trees, s); break;
    default: k_scatter_tma<0><<<grid, kST, kScatterSmemBytes, st>>>(trees, s); break;
  }
}

}  // namespace kdt
