// kdt_leafsort.cu -- restore the order of the permutation inside every leaf.
//
// In the sequential definition of the build (paper, Sec. 2: each level
// partitions its cells around their splits) the partition is stable and
// starts from the identity, so inside every terminal cell the permutation is
// ascending original index. The multi-CTA pipeline keeps cells in subset
// order instead (every (cell, subset) segment contiguous), which leaves the
// same set of indices in every leaf in another order. This pass sorts each
// terminal cell's slice of the permutation ascending:
//   - up to kLeafWarpMax points: one warp, bitonic network in registers;
//   - up to kLeafBlockMax points: one CTA, LSD radix sort (8-bit digits) in
//     shared memory, stable ranks from warp match masks;
//   - larger: the same LSD passes over global memory, tiles of kLeafBlockMax
//     points, per-(tile, digit) counts scanned per leaf (host-driven; only
//     shallow trees or cells that stop splitting produce such leaves).
// Original indices are distinct, so the result does not depend on stability
// across equal keys; stability is what makes the LSD passes correct.
#include <algorithm>
#include <vector>

#include "kdt_internal.cuh"
#include "kdt_launch.h"
#include "kdt_trace.h"

namespace kdt {

namespace {

constexpr int kLsThreads = 256;
constexpr int kLsWarps = kLsThreads / 32;
constexpr int kLsItems = kLeafBlockMax / kLsThreads;  // 16 keys per thread
constexpr uint32_t kInvalidDigit = 256u;

// Number of 8-bit digits that cover original indices below n.
__host__ __device__ inline int index_digits(uint64_t n) {
  int bits = 0;
  while (bits < 32 && (n - 1) >> bits) ++bits;
  const int digits = (bits + 7) / 8;
  return digits > 1 ? digits : 1;
}

// -------------------------------------------------------- one warp, <= 32K

template <int K>
__device__ void warp_sort_slice(uint32_t* a, uint32_t m) {
  const int lane = threadIdx.x & 31;
  uint32_t v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t e = (uint32_t)(k * 32 + lane);
    v[k] = e < m ? a[e] : 0xffffffffu;
  }
  constexpr int N = 32 * K;
#pragma unroll
  for (int size = 2; size <= N; size <<= 1) {
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
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t e = (uint32_t)(k * 32 + lane);
    if (e < m) a[e] = v[k];
  }
}

__device__ void warp_sort_any(uint32_t* a, uint32_t m) {
  if (m <= 32) warp_sort_slice<1>(a, m);
  else if (m <= 64) warp_sort_slice<2>(a, m);
  else if (m <= 128) warp_sort_slice<4>(a, m);
  else warp_sort_slice<8>(a, m);
}

// ------------------------------------------------------ block ranking

// Stable ranks by digit (key >> shift) & 255 of the m <= kLeafBlockMax keys
// src[0..m) (shared memory). Warp w owns positions [w*512, w*512+512) in 16
// rounds of 32 in order; within a round, lanes sharing a digit are ranked by
// their match mask. On return whist[w][b] holds the number of keys with digit
// b in warps before w, dtot[b] the keys with digit b, rank[j] the rank of the
// thread's j-th key among equal digits of its warp, dig[j] its digit.
__device__ void block_rank(const uint32_t* src, uint32_t m, int shift, uint32_t (*whist)[256], uint32_t* dtot,
                           uint32_t (&rank)[kLsItems], uint32_t (&dig)[kLsItems]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int i = threadIdx.x; i < kLsWarps * 256; i += kLsThreads) (&whist[0][0])[i] = 0;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kLsItems; ++j) {
    const uint32_t idx = (uint32_t)(warp * (32 * kLsItems) + j * 32 + lane);
    const uint32_t dgt = idx < m ? (src[idx] >> shift) & 255u : kInvalidDigit;
    const unsigned peers = __match_any_sync(0xffffffffu, dgt);
    const uint32_t base = dgt != kInvalidDigit ? whist[warp][dgt] : 0u;
    __syncwarp();
    if (dgt != kInvalidDigit && (peers & lt) == 0u) whist[warp][dgt] = base + (uint32_t)__popc(peers);
    __syncwarp();
    rank[j] = base + (uint32_t)__popc(peers & lt);
    dig[j] = dgt;
  }
  __syncthreads();
  {
    const int b = threadIdx.x;  // kLsThreads == 256 digits
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kLsWarps; ++w) {
      const uint32_t v = whist[w][b];
      whist[w][b] = run;
      run += v;
    }
    dtot[b] = run;
  }
  __syncthreads();
}

struct LsShared {
  uint32_t buf[2][kLeafBlockMax];
  uint32_t whist[kLsWarps][256];
  uint32_t dtot[256];
  uint32_t dbase[256];
  uint32_t tmp[33];
};

// One CTA: sort a[0..m) (global) with the keys staged in shared memory.
__device__ void block_sort_slice(uint32_t* a, uint32_t m, int digits, LsShared& S) {
  for (uint32_t i = threadIdx.x; i < m; i += kLsThreads) S.buf[0][i] = a[i];
  __syncthreads();
  int cur = 0;
  for (int p = 0; p < digits; ++p) {
    uint32_t rank[kLsItems], dig[kLsItems];
    block_rank(S.buf[cur], m, 8 * p, S.whist, S.dtot, rank, dig);
    uint32_t tot;
    const uint32_t ex = block_excl_scan(S.dtot[threadIdx.x], S.tmp, &tot);
    S.dbase[threadIdx.x] = ex;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < kLsItems; ++j) {
      if (dig[j] == kInvalidDigit) continue;
      const uint32_t idx = (uint32_t)(warp * (32 * kLsItems) + j * 32 + lane);
      S.buf[cur ^ 1][S.dbase[dig[j]] + S.whist[warp][dig[j]] + rank[j]] = S.buf[cur][idx];
    }
    __syncthreads();
    cur ^= 1;
  }
  for (uint32_t i = threadIdx.x; i < m; i += kLsThreads) a[i] = S.buf[cur][i];
  __syncthreads();
}

// Grid (chunks, trees). Warps sort the small terminal cells, CTAs the middle
// ones; the largest are listed for the global passes. Four CTAs per SM by a
// register bound: the warps' networks, which sort nearly every leaf of a deep
// tree, want the warps; the CTA path spills a few words.
__global__ void __launch_bounds__(kLsThreads, 4) k_leaf_sort(const TreeDev* trees, const uint32_t* slots,
                                                          uint32_t nslots) {
  __shared__ LsShared S;
  const uint32_t si = blockIdx.y;
  if (si >= nslots) return;
  const TreeDev& t = trees[slots[si]];
  const uint32_t nrec = min(*t.term_count, t.term_cap);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wstride = gridDim.x * kLsWarps;
  uint32_t rec = blockIdx.x * kLsWarps + warp;
  TermRec trn = rec < nrec ? t.terms[rec] : TermRec{};
  for (; rec < nrec; rec += wstride) {
    const TermRec tr = trn;  // the next record is read before this cell is sorted
    if (rec + wstride < nrec) trn = t.terms[rec + wstride];
    if (tr.count <= 1u) continue;
    if (tr.count <= (uint32_t)kLeafWarpMax) {
      warp_sort_any(t.out_perm + tr.begin, tr.count);
    } else if (tr.count > (uint32_t)kLeafBlockMax && lane == 0) {
      const uint32_t k = atomicAdd(t.huge_count, 1u);
      if (k < t.huge_cap) t.huge[k] = rec; else set_status(t, ST_CAPACITY);
    }
  }
  // the middle cells: the CTA reads kLsThreads records at once and sorts the
  // ones of its chunk that need a CTA, one after another
  __shared__ uint32_t mids[kLsThreads];
  __shared__ uint32_t nmid;
  const int digits = index_digits((uint64_t)t.n);
  for (uint32_t base = blockIdx.x * kLsThreads; base < nrec; base += gridDim.x * kLsThreads) {
    if (threadIdx.x == 0) nmid = 0;
    __syncthreads();
    const uint32_t rec = base + threadIdx.x;
    const uint32_t cnt = rec < nrec ? t.terms[rec].count : 0u;
    if (cnt > (uint32_t)kLeafWarpMax && cnt <= (uint32_t)kLeafBlockMax) mids[atomicAdd(&nmid, 1u)] = rec;
    __syncthreads();
    const uint32_t nm = nmid;
    for (uint32_t j = 0; j < nm; ++j) {
      const TermRec tr = t.terms[mids[j]];
      block_sort_slice(t.out_perm + tr.begin, tr.count, digits, S);
    }
    __syncthreads();  // mids and nmid are reused by the next chunk
  }
}

// --------------------------------------------- global passes (large leaves)

// Tile of a large leaf: absolute begin of the leaf, its size, the tile's
// offset inside it.
struct LeafTile {
  uint32_t begin, count, off, pad;
};

__global__ void __launch_bounds__(kLsThreads) k_leaf_hist(const uint32_t* src, const LeafTile* tiles, int shift,
                                                          uint32_t* hist) {
  __shared__ uint32_t h[256];
  const LeafTile tl = tiles[blockIdx.x];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t m = min((uint32_t)kLeafBlockMax, tl.count - tl.off);
  const uint32_t* a = src + tl.begin + tl.off;
  for (uint32_t i = threadIdx.x; i < m; i += kLsThreads) atomicAdd(&h[(a[i] >> shift) & 255u], 1u);
  __syncthreads();
  hist[(size_t)blockIdx.x * 256 + threadIdx.x] = h[threadIdx.x];
}

// One CTA per large leaf (its tiles are [first, first + ntiles)): turn the
// per-tile digit counts into destinations relative to the leaf (digit-major
// order, tiles in order inside a digit).
__global__ void __launch_bounds__(kLsThreads) k_leaf_scan(const uint32_t* first_tile, const uint32_t* ntiles,
                                                          uint32_t* hist) {
  __shared__ uint32_t tmp[33];
  const uint32_t f = first_tile[blockIdx.x], nt = ntiles[blockIdx.x];
  const uint32_t b = threadIdx.x;
  uint32_t run = 0;
#pragma unroll 8
  for (uint32_t k = 0; k < nt; ++k) {
    uint32_t* h = hist + (size_t)(f + k) * 256 + b;
    const uint32_t v = *h;
    *h = run;
    run += v;
  }
  uint32_t tot;
  const uint32_t base = block_excl_scan(run, tmp, &tot);
#pragma unroll 8
  for (uint32_t k = 0; k < nt; ++k) hist[(size_t)(f + k) * 256 + b] += base;
}

__global__ void __launch_bounds__(kLsThreads) k_leaf_scatter(const uint32_t* src, uint32_t* dst,
                                                             const LeafTile* tiles, int shift,
                                                             const uint32_t* hist) {
  __shared__ uint32_t keys[kLeafBlockMax];
  __shared__ uint32_t whist[kLsWarps][256];
  __shared__ uint32_t dtot[256];
  const LeafTile tl = tiles[blockIdx.x];
  const uint32_t m = min((uint32_t)kLeafBlockMax, tl.count - tl.off);
  const uint32_t* a = src + tl.begin + tl.off;
  for (uint32_t i = threadIdx.x; i < m; i += kLsThreads) keys[i] = a[i];
  __syncthreads();
  uint32_t rank[kLsItems], dig[kLsItems];
  block_rank(keys, m, shift, whist, dtot, rank, dig);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t* hb = hist + (size_t)blockIdx.x * 256;
  uint32_t* out = dst + tl.begin;
#pragma unroll
  for (int j = 0; j < kLsItems; ++j) {
    if (dig[j] == kInvalidDigit) continue;
    const uint32_t idx = (uint32_t)(warp * (32 * kLsItems) + j * 32 + lane);
    const uint32_t pos = hb[dig[j]] + whist[warp][dig[j]] + rank[j];
    if (pos < tl.count) out[pos] = keys[idx];
  }
}

__global__ void k_leaf_copy(const uint32_t* src, uint32_t* dst, const LeafTile* tiles) {
  const LeafTile tl = tiles[blockIdx.x];
  const uint32_t m = min((uint32_t)kLeafBlockMax, tl.count - tl.off);
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) dst[tl.begin + tl.off + i] = src[tl.begin + tl.off + i];
}

}  // namespace

void launch_leaf_sort(const TreeDev* trees, const uint32_t* slots, uint32_t nslots, uint32_t max_records,
                      cudaStream_t st) {
  if (nslots == 0 || max_records == 0) return;
  TraceScope ts(K_LEAF_SORT, st, max_records);
  const uint32_t chunks = std::max<uint32_t>(1, std::min<uint32_t>((max_records + 63) / 64, 2048));
  k_leaf_sort<<<dim3(chunks, nslots), kLsThreads, 0, st>>>(trees, slots, nslots);
}

size_t leaf_huge_tiles_cap(uint64_t n) { return (size_t)(2 * (n / kLeafBlockMax) + 2); }

cudaError_t leaf_sort_huge(const TreeHost& th, const std::vector<TermRec>& recs, cudaStream_t st) {
  if (recs.empty()) return cudaSuccess;
  std::vector<LeafTile> tiles;
  std::vector<uint32_t> first, ntiles;
  for (const TermRec& r : recs) {
    first.push_back((uint32_t)tiles.size());
    uint32_t k = 0;
    for (uint32_t off = 0; off < r.count; off += kLeafBlockMax, ++k) tiles.push_back(LeafTile{r.begin, r.count, off, 0});
    ntiles.push_back(k);
  }
  const size_t nt = tiles.size(), nr = recs.size();
  const size_t need = nt * sizeof(LeafTile) + nt * 256 * 4 + 2 * nr * 4 + 4 * 256;
  if (need > th.scratch_bytes) return cudaErrorMemoryAllocation;
  uint8_t* p = (uint8_t*)th.scratch;
  LeafTile* d_tiles = (LeafTile*)p;
  p += ((nt * sizeof(LeafTile) + 255) & ~(size_t)255);
  uint32_t* d_hist = (uint32_t*)p;
  p += ((nt * 256 * 4 + 255) & ~(size_t)255);
  uint32_t* d_first = (uint32_t*)p;
  uint32_t* d_nt = d_first + nr;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_tiles, tiles.data(), nt * sizeof(LeafTile), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(d_first, first.data(), nr * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(d_nt, ntiles.data(), nr * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  const int digits = index_digits(th.n);
  uint32_t* a = th.out_perm;
  uint32_t* b = th.keys;
  for (int d = 0; d < digits; ++d) {
    { TraceScope ts(K_LEAF_HIST, st); k_leaf_hist<<<(unsigned)nt, kLsThreads, 0, st>>>(a, d_tiles, 8 * d, d_hist); }
    { TraceScope ts(K_LEAF_SCAN, st); k_leaf_scan<<<(unsigned)nr, kLsThreads, 0, st>>>(d_first, d_nt, d_hist); }
    {
      TraceScope ts(K_LEAF_SCATTER, st);
      k_leaf_scatter<<<(unsigned)nt, kLsThreads, 0, st>>>(a, b, d_tiles, 8 * d, d_hist);
    }
    std::swap(a, b);
  }
  if (a != th.out_perm) {
    TraceScope ts(K_LEAF_COPY, st);
    k_leaf_copy<<<(unsigned)nt, kLsThreads, 0, st>>>(a, th.out_perm, d_tiles);
  }
  return cudaGetLastError();
}

}  // namespace kdt
