// kdt_shard.cu -- the sharded build: G logical shards on one GPU, each owning
// whole subsets, exchange what the paper's reduce step exchanges.
//
// The paper's setting is data that stays in its R subsets on R workers
// (App. C.2: the user's partition I_1..I_R, a map step on each, a reduce
// across them; Sec. 3.2: the statistics of any partition into subsets
// combine exactly). Here subset s belongs to shard s % G. Every shard is a
// tree of one forest holding only its own points (with their subset ids);
// the forest's trees advance level by level together. In each level step:
//   - every shard takes the lower median and the size of each of its
//     (cell, subset) segments (the per-subset statistic);
//   - an all-gather hands every shard the (median, size) pairs of the other
//     shards' subsets of the same cell, and the cell's total size, so that
//     every shard runs the identical combine and gets the identical split;
//   - for the widest-spread rule, the per-coordinate min / max of the root
//     and of every child are reduced over the shards the same way;
//   - the partition is local: no point changes shard.
// At the end the leaves are merged: the offsets are sums over the shards,
// and each leaf lists its points from all shards in increasing original
// index (the order of the sequential definition), restored by the leaf sort.
// The result is bit-identical to the build on one shard.
//
// On one GPU the all-gather is a kernel that reads the other shards' tables
// in device memory; on several GPUs it would be one collective per level of
// the same tables (8 bytes per (cell, subset), 16 d bytes per child).
#include <algorithm>
#include <vector>

#include "kdt.h"
#include "kdt_engine.h"
#include "kdt_launch.h"
#include "kdt_trace.h"

namespace kdt {

namespace {

// ------------------------------------------------------- exchange kernels

// Step cell of every (shard, heap) of this step's level.
__global__ void k_shard_index(StepDev s) {
  const uint32_t nc = ncells_of(s);
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const Cell cell = s.cells[c];
    const uint32_t k = cell.heap - ((1u << cell.level) - 1u);
    if ((uint32_t)cell.tree < s.shards && k < s.shard_span) s.shard_idx[(size_t)cell.tree * s.shard_span + k] = c;
  }
}

// One warp per cell: the (median, size) pairs of the subsets that other
// shards own come from the same cell of their owner; the cell's size over
// all shards is the combine's weight.
__global__ void k_shard_medians(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  const int lane = threadIdx.x & 31;
  for (uint32_t c = blockIdx.x * 8u + (threadIdx.x >> 5); c < nc; c += gridDim.x * 8u) {
    const Cell cell = s.cells[c];
    const TreeDev& t = trees[cell.tree];
    const uint32_t g = (uint32_t)cell.tree, G = s.shards, r = (uint32_t)t.r;
    const uint32_t k = cell.heap - ((1u << cell.level) - 1u);
    const uint32_t* row = s.shard_idx + k;  // row[o * span]: the cell in shard o
    uint32_t w = 0;
    for (uint32_t o = lane; o < G; o += 32) {
      const uint32_t co = row[(size_t)o * s.shard_span];
      w += co == kNoRow ? 0u : s.cells[co].count;
    }
    w = warp_sum(w);
    if (lane == 0) s.wcount[c] = w;
    const uint32_t g0 = s.seg_base[c];
    for (uint32_t j = lane; j < r; j += 32) {
      const uint32_t o = j % G;
      if (o == g) continue;  // this shard's own subset
      const uint32_t co = row[(size_t)o * s.shard_span];
      uint32_t med = 0, wj = 0;
      if (co != kNoRow) {
        med = s.seg_med[s.seg_base[co] + j];
        wj = s.seg_w[s.seg_base[co] + j];
      }
      s.seg_med[g0 + j] = med;
      s.seg_w[g0 + j] = wj;
    }
  }
}

// Children's min / max keys per coordinate over all shards (widest spread):
// first every cell gathers them into mm_tmp, then writes them back, so that
// no cell reads a table another is writing.
__global__ void k_shard_mm_gather(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  const int lane = threadIdx.x & 31;
  for (uint32_t c = blockIdx.x * 8u + (threadIdx.x >> 5); c < nc; c += gridDim.x * 8u) {
    const Cell cell = s.cells[c];
    const TreeDev& t = trees[cell.tree];
    if (t.key_rule != KEY_WIDEST) continue;
    const int d = t.d;
    const uint32_t k = cell.heap - ((1u << cell.level) - 1u);
    const uint32_t* row = s.shard_idx + k;
    for (int j = lane; j < 2 * d; j += 32) {
      const int side = j / d, l = j % d;
      uint32_t lo = 0xffffffffu, hi = 0u;
      for (uint32_t o = 0; o < s.shards; ++o) {
        const uint32_t co = row[(size_t)o * s.shard_span];
        if (co == kNoRow) continue;
        const uint32_t* mm = s.child_mm + (((size_t)co * 2 + side) * kMaxDims + l) * 2;
        lo = min(lo, mm[0]);
        hi = max(hi, mm[1]);
      }
      s.mm_tmp[((size_t)c * 2 * d + j) * 2] = lo;
      s.mm_tmp[((size_t)c * 2 * d + j) * 2 + 1] = hi;
    }
  }
}

__global__ void k_shard_mm_put(const TreeDev* trees, StepDev s) {
  const uint32_t nc = ncells_of(s);
  const int lane = threadIdx.x & 31;
  for (uint32_t c = blockIdx.x * 8u + (threadIdx.x >> 5); c < nc; c += gridDim.x * 8u) {
    const Cell cell = s.cells[c];
    const TreeDev& t = trees[cell.tree];
    if (t.key_rule != KEY_WIDEST) continue;
    const int d = t.d;
    for (int j = lane; j < 2 * d; j += 32) {
      const int side = j / d, l = j % d;
      uint32_t* mm = s.child_mm + (((size_t)c * 2 + side) * kMaxDims + l) * 2;
      mm[0] = s.mm_tmp[((size_t)c * 2 * d + j) * 2];
      mm[1] = s.mm_tmp[((size_t)c * 2 * d + j) * 2 + 1];
    }
  }
}

}  // namespace

void launch_shard_index(const StepDev& s, uint32_t ncells_cap, cudaStream_t st) {
  cudaMemsetAsync(s.shard_idx, 0xff, (size_t)s.shards * s.shard_span * 4, st);
  TraceScope ts(K_SHARD_EXCHANGE, st);
  k_shard_index<<<std::max<uint32_t>(1, std::min<uint32_t>((ncells_cap + 255) / 256, 4096u)), 256, 0, st>>>(s);
}

void launch_shard_medians(const TreeDev* trees, const StepDev& s, uint32_t ncells_cap, cudaStream_t st) {
  TraceScope ts(K_SHARD_EXCHANGE, st);
  k_shard_medians<<<std::max<uint32_t>(1, std::min<uint32_t>((ncells_cap + 7) / 8, 8192u)), 256, 0, st>>>(trees, s);
}

void launch_shard_minmax(const TreeDev* trees, const StepDev& s, uint32_t ncells_cap, cudaStream_t st) {
  TraceScope ts(K_SHARD_EXCHANGE, st);
  const uint32_t grid = std::max<uint32_t>(1, std::min<uint32_t>((ncells_cap + 7) / 8, 8192u));
  k_shard_mm_gather<<<grid, 256, 0, st>>>(trees, s);
  k_shard_mm_put<<<grid, 256, 0, st>>>(trees, s);
}


namespace {

constexpr int kShTile = 2048;     // points per tile of the split
constexpr int kShThreads = 256;
constexpr int kShRounds = kShTile / kShThreads;
constexpr int kMaxShards = 16;

struct SplitArgs {
  const float* x;         // [d][n]
  const void* sid_in;     // explicit ids (in_bytes wide) or null
  int64_t n;
  int32_t d, r, subset_mode, in_bytes, out_bytes, shards;  // id widths: input (explicit), shards' ids
  uint32_t ntiles;
  uint32_t* counts;       // [ntiles][shards]
  uint32_t* toff;         // [ntiles][shards] exclusive offset of the tile inside its shard
  uint32_t* ntot;         // [shards]
  const uint32_t* base;   // [shards] first point of each shard (host-computed)
  float* xs;              // shard g's columns [d][n_g] at d * base[g]
  void* sids;             // shard ids (out_bytes wide)
  uint32_t* gidx;         // original index of every shard point
  int32_t* status;
};

__device__ __forceinline__ uint32_t sh_subset(const SplitArgs& a, int64_t i) {
  if (a.subset_mode == SUB_MOD) return (uint32_t)(i % a.r);
  if (a.subset_mode == SUB_CONTIG) return (uint32_t)(((uint64_t)i * (uint64_t)a.r) / (uint64_t)a.n);
  const uint32_t v = a.in_bytes == 1 ? (uint32_t)((const uint8_t*)a.sid_in)[i] : (uint32_t)((const uint16_t*)a.sid_in)[i];
  if (v >= (uint32_t)a.r) {
    atomicCAS(a.status, ST_OK, ST_INVALID_ARG);
    return 0;
  }
  return v;
}

// Points of every shard in every tile.
__global__ void __launch_bounds__(kShThreads) k_sh_count(SplitArgs a) {
  __shared__ uint32_t cnt[kMaxShards];
  const uint32_t tile = blockIdx.x;
  if (threadIdx.x < (uint32_t)a.shards) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)tile * kShTile;
  for (int q = 0; q < kShRounds; ++q) {
    const int64_t i = t0 + q * kShThreads + threadIdx.x;
    const uint32_t o = i < a.n ? sh_subset(a, i) % (uint32_t)a.shards : 0xffffffffu;
    const unsigned same = __match_any_sync(0xffffffffu, o);
    if (o != 0xffffffffu && (threadIdx.x & 31) == (uint32_t)(__ffs(same) - 1))
      atomicAdd(&cnt[o], (uint32_t)__popc(same));
  }
  __syncthreads();
  if (threadIdx.x < (uint32_t)a.shards) a.counts[(size_t)tile * a.shards + threadIdx.x] = cnt[threadIdx.x];
}

// One CTA per shard: exclusive scan of its per-tile counts.
__global__ void k_sh_scan(SplitArgs a) {
  __shared__ uint32_t tmp[33];
  const uint32_t g = blockIdx.x;
  uint32_t run = 0;
  for (uint32_t j0 = 0; j0 < a.ntiles; j0 += blockDim.x) {
    const uint32_t j = j0 + threadIdx.x;
    const uint32_t v = j < a.ntiles ? a.counts[(size_t)j * a.shards + g] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, tmp, &tot);
    if (j < a.ntiles) a.toff[(size_t)j * a.shards + g] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) a.ntot[g] = run;
}

// Stable move of every point into its shard (original order inside a
// shard): a point's place is its tile's offset in the shard, plus the points
// of its shard in earlier blocks of 32 of the tile, plus its rank among the
// lanes of its block with the same shard.
__global__ void __launch_bounds__(kShThreads) k_sh_scatter(SplitArgs a) {
  __shared__ uint32_t bc[kMaxShards][kShRounds * kShThreads / 32];
  const uint32_t tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kBlocks = kShRounds * kShThreads / 32;  // 64 blocks of 32 points, in position order
  for (int j = threadIdx.x; j < kMaxShards * kBlocks; j += kShThreads) (&bc[0][0])[j] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)tile * kShTile;
  uint32_t oq[kShRounds], sq[kShRounds], rq[kShRounds];
#pragma unroll
  for (int q = 0; q < kShRounds; ++q) {
    const int64_t i = t0 + q * kShThreads + threadIdx.x;
    sq[q] = i < a.n ? sh_subset(a, i) : 0u;
    oq[q] = i < a.n ? sq[q] % (uint32_t)a.shards : 0xffffffffu;
    const unsigned same = __match_any_sync(0xffffffffu, oq[q]);
    rq[q] = (uint32_t)__popc(same & ((1u << lane) - 1u));
    if (oq[q] != 0xffffffffu && lane == __ffs(same) - 1) bc[oq[q]][q * (kShThreads / 32) + warp] = __popc(same);
  }
  __syncthreads();
  // exclusive scan of every shard's 64 block counts (a warp per shard)
  for (int g = warp; g < a.shards; g += kShThreads / 32) {
    const uint32_t c0 = bc[g][lane], c1 = bc[g][lane + 32];
    const uint32_t i0 = warp_incl_scan(c0);
    const uint32_t i1 = warp_incl_scan(c1) + __shfl_sync(0xffffffffu, i0, 31);
    __syncwarp();
    bc[g][lane] = i0 - c0;
    bc[g][lane + 32] = i1 - c1;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kShRounds; ++q) {
    const uint32_t o = oq[q];
    if (o == 0xffffffffu) continue;
    const int64_t i = t0 + q * kShThreads + threadIdx.x;
    const uint32_t loc = a.toff[(size_t)tile * a.shards + o] + bc[o][q * (kShThreads / 32) + warp] + rq[q];
    const uint32_t ng = a.ntot[o], b = a.base[o];
    float* xs = a.xs + (size_t)a.d * b;
    for (int l = 0; l < a.d; ++l) xs[(size_t)l * ng + loc] = a.x[(int64_t)l * a.n + i];
    if (a.out_bytes == 1)
      ((uint8_t*)a.sids)[b + loc] = (uint8_t)sq[q];
    else
      ((uint16_t*)a.sids)[b + loc] = (uint16_t)sq[q];
    a.gidx[b + loc] = (uint32_t)i;
  }
}

struct MergeArgs {
  int32_t shards, L;
  uint32_t nl;               // 2^L leaves
  const int64_t* offs_sh;    // [shards][nl + 1]
  const float* vals_sh;      // [shards][nl - 1]
  const int8_t* dims_sh;     // [shards][nl - 1]
  const uint32_t* perm_sh;   // shard g's permutation (local indices) at base[g]
  const uint32_t* base;      // [shards]
  const uint32_t* ntot;      // [shards]
  const uint32_t* gidx;
  uint32_t* pre;             // [shards][nl]: points of leaf k in shards before g
  int64_t* offs;             // [nl + 1]
  float* vals;
  int8_t* dims;
  uint32_t* perm;
  TermRec* terms;            // [nl]
  uint32_t* term_count;
  int32_t* status;
};

__global__ void k_sh_merge_offsets(MergeArgs a) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= a.nl; k += gridDim.x * blockDim.x) {
    int64_t tot = 0;
    uint32_t run = 0;
    for (int g = 0; g < a.shards; ++g) {
      const int64_t* o = a.offs_sh + (size_t)g * (a.nl + 1);
      tot += o[k];
      if (k < a.nl) {
        a.pre[(size_t)g * a.nl + k] = run;
        run += (uint32_t)(o[k + 1] - o[k]);
      }
    }
    a.offs[k] = tot;
  }
}

// Every node's split from a shard that holds points of it (all such shards
// computed the same one); the sentinel where none does.
__global__ void k_sh_merge_splits(MergeArgs a) {
  for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h + 1 < a.nl; h += gridDim.x * blockDim.x) {
    int8_t dm = -1;
    float v = __int_as_float(0x7f800000);
    for (int g = 0; g < a.shards; ++g) {
      const int8_t dg = a.dims_sh[(size_t)g * (a.nl - 1) + h];
      const float vg = a.vals_sh[(size_t)g * (a.nl - 1) + h];
      if (dg < 0) continue;
      if (dm >= 0 && (dg != dm || __float_as_uint(vg) != __float_as_uint(v))) atomicCAS(a.status, ST_OK, ST_INTERNAL);
      dm = dg;
      v = vg;
    }
    a.dims[h] = dm;
    a.vals[h] = v;
  }
}

// Every shard point to its leaf's range of the merged order (shards in turn);
// the leaf sort then puts each leaf in increasing original index.
__global__ void k_sh_merge_perm(MergeArgs a, uint32_t total) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
    int g = 0;
    while (g + 1 < a.shards && a.base[g + 1] <= p) ++g;
    const uint32_t lp = p - a.base[g];
    const int64_t* o = a.offs_sh + (size_t)g * (a.nl + 1);
    uint32_t lo = 0, hi = a.nl;  // the leaf k with o[k] <= lp < o[k + 1]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) / 2;
      if (o[mid] <= (int64_t)lp) lo = mid; else hi = mid;
    }
    const int64_t dst = a.offs[lo] + a.pre[(size_t)g * a.nl + lo] + ((int64_t)lp - o[lo]);
    a.perm[dst] = a.gidx[a.base[g] + a.perm_sh[a.base[g] + lp]];
  }
}

__global__ void k_sh_terms(MergeArgs a) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < a.nl; k += gridDim.x * blockDim.x)
    a.terms[k] = TermRec{(uint32_t)a.offs[k], (uint32_t)(a.offs[k + 1] - a.offs[k]), a.nl - 1u + k, a.L};
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.term_count = a.nl;
}

}  // namespace

namespace {

inline size_t sh_align(size_t x) { return (x + 255) & ~(size_t)255; }

struct DevMem {
  void* p = nullptr;
  ~DevMem() {
    if (p) cudaFree(p);
  }
};

#define SH_TRY(expr)             \
  do {                           \
    if ((expr) != cudaSuccess) { \
      (void)cudaGetLastError();  \
      return KDT_ERR_CUDA;       \
    }                            \
  } while (0)

kdt_status sharded_build(const float* points, const kdt_params& p, int32_t G, uint32_t* out_perm, float* out_vals,
                         int8_t* out_dims, int64_t* out_offs, int32_t* out_levels, cudaStream_t st) {
  const int64_t n = p.n;
  const int d = p.d, L = p.depth;
  const uint32_t nl = 1u << L;
  const uint32_t ntiles = (uint32_t)((n + kShTile - 1) / kShTile);
  const int out_bytes = p.r <= 256 ? 1 : 2;
  const int in_bytes = p.subset_mode == KDT_SUBSET_EXPLICIT ? (p.subset_id16 ? 2 : 1) : 0;

  // ---- split: points per shard per tile, then each shard's size
  size_t off = 0;
  const size_t o_counts = off;
  off += sh_align((size_t)ntiles * G * 4 + 4);
  const size_t o_toff = off;
  off += sh_align((size_t)ntiles * G * 4 + 4);
  const size_t o_ntot = off;
  off += sh_align((size_t)G * 4);
  const size_t o_base = off;
  off += sh_align((size_t)G * 4);
  const size_t o_words = off;  // split status, merge status, term count, huge count
  off += sh_align(16);
  DevMem small;
  if (dev_malloc(&small.p, off) != cudaSuccess) {
    (void)cudaGetLastError();
    return KDT_ERR_OOM;
  }
  uint8_t* sm = (uint8_t*)small.p;
  int32_t* words = (int32_t*)(sm + o_words);
  SplitArgs a{};
  a.x = points;
  a.sid_in = p.subset_id16 ? (const void*)p.subset_id16 : (const void*)p.subset_id8;
  a.n = n;
  a.d = d;
  a.r = p.r;
  a.subset_mode = p.subset_mode;
  a.in_bytes = in_bytes;
  a.out_bytes = out_bytes;
  a.shards = G;
  a.ntiles = ntiles;
  a.counts = (uint32_t*)(sm + o_counts);
  a.toff = (uint32_t*)(sm + o_toff);
  a.ntot = (uint32_t*)(sm + o_ntot);
  a.base = (const uint32_t*)(sm + o_base);
  a.status = words;
  SH_TRY(cudaMemsetAsync(words, 0, 16, st));
  SH_TRY(cudaMemsetAsync(a.ntot, 0, (size_t)G * 4, st));
  if (ntiles) {
    TraceScope ts(K_SHARD_SPLIT, st, (uint64_t)n);
    k_sh_count<<<ntiles, kShThreads, 0, st>>>(a);
    k_sh_scan<<<G, 1024, 0, st>>>(a);
  }
  std::vector<uint32_t> ntot(G), base(G);
  SH_TRY(cudaMemcpyAsync(ntot.data(), a.ntot, (size_t)G * 4, cudaMemcpyDeviceToHost, st));
  SH_TRY(cudaStreamSynchronize(st));
  uint64_t run = 0;
  for (int g = 0; g < G; ++g) {
    base[g] = (uint32_t)run;
    run += ntot[g];
  }
  if (run != (uint64_t)n) return KDT_ERR_CUDA;
  SH_TRY(cudaMemcpyAsync((void*)a.base, base.data(), (size_t)G * 4, cudaMemcpyHostToDevice, st));

  // ---- the forest: shard g is tree g, with its points' subset ids
  std::vector<kdt_params> pg(G);
  std::vector<TreePlan> tp(G);
  StepNeeds needs;
  static const uint8_t kPlanId = 0;  // a non-null id pointer while planning
  for (int g = 0; g < G; ++g) {
    pg[g] = p;
    pg[g].n = ntot[g];
    pg[g].subset_mode = KDT_SUBSET_EXPLICIT;
    pg[g].subset_id8 = out_bytes == 1 ? &kPlanId : nullptr;
    pg[g].subset_id16 = out_bytes == 2 ? (const uint16_t*)&kPlanId : nullptr;
    tp[g] = plan_tree(pg[g], /*no_subtree=*/true);
    tp[g].leafsort = false;  // the merged leaves are sorted once, at the end (the subset-order presort stays)
    needs.add(pg[g], tp[g]);
  }
  const StepPlan sp = plan_step(needs);
  const uint32_t span = std::max<uint32_t>(1u, nl / 2u);
  off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off += sh_align(b);
    return o;
  };
  const size_t o_step = take(sp.bytes);
  std::vector<size_t> o_tree(G);
  for (int g = 0; g < G; ++g) o_tree[g] = take(tp[g].bytes);
  const size_t o_xs = take((size_t)d * n * 4);
  const size_t o_sids = take((size_t)n * out_bytes);
  const size_t o_gidx = take((size_t)n * 4);
  const size_t o_perm = take((size_t)n * 4);
  const size_t o_vals = take((size_t)G * (nl - 1) * 4);
  const size_t o_dims = take((size_t)G * (nl - 1));
  const size_t o_offs = take((size_t)G * (nl + 1) * 8);
  const size_t o_idx = take((size_t)G * span * 4);
  const size_t o_wc = take((size_t)sp.maxB * 4);
  const size_t o_mm = take((size_t)sp.maxB * 4 * d * 4);
  const size_t o_pre = take((size_t)G * nl * 4);
  const size_t o_terms = take((size_t)nl * sizeof(TermRec));
  const size_t o_huge = take((size_t)nl * 4);
  const size_t o_td = take(sizeof(TreeDev));
  const size_t o_slot = take(4);
  DevMem big;
  if (dev_malloc(&big.p, off) != cudaSuccess) {
    (void)cudaGetLastError();
    return KDT_ERR_OOM;
  }
  uint8_t* ws = (uint8_t*)big.p;
  a.xs = (float*)(ws + o_xs);
  a.sids = ws + o_sids;
  a.gidx = (uint32_t*)(ws + o_gidx);
  if (ntiles) {
    TraceScope ts(K_SHARD_SPLIT, st, (uint64_t)n);
    k_sh_scatter<<<ntiles, kShThreads, 0, st>>>(a);
  }
  SH_TRY(cudaGetLastError());

  Engine e(sp, ws + o_step, st);
  kdt_status s = e.reset();
  if (s != KDT_OK) return s;
  e.set_sharding((uint32_t)G, span, (uint32_t*)(ws + o_idx), (uint32_t*)(ws + o_wc), (uint32_t*)(ws + o_mm));
  uint32_t* perm_sh = (uint32_t*)(ws + o_perm);
  float* vals_sh = (float*)(ws + o_vals);
  int8_t* dims_sh = (int8_t*)(ws + o_dims);
  int64_t* offs_sh = (int64_t*)(ws + o_offs);
  std::vector<uint32_t> slots(G);
  for (int g = 0; g < G; ++g) {
    slots[g] = (uint32_t)g;
    if (out_bytes == 1)
      pg[g].subset_id8 = (const uint8_t*)(ws + o_sids) + base[g];
    else
      pg[g].subset_id16 = (const uint16_t*)(ws + o_sids) + base[g];
    s = e.admit((uint32_t)g, a.xs + (size_t)d * base[g], pg[g], tp[g], ws + o_tree[g], perm_sh + base[g],
                vals_sh + (size_t)g * (nl - 1), dims_sh + (size_t)g * (nl - 1), offs_sh + (size_t)g * (nl + 1));
    if (s != KDT_OK) return s;
  }
  s = e.run_to_completion();
  if (s != KDT_OK) return s;
  std::vector<kdt_status> status;
  std::vector<int32_t> levels;
  s = e.finalize(slots, &status, &levels);
  if (s != KDT_OK) return s;
  int32_t split_status = 0;
  SH_TRY(cudaMemcpyAsync(&split_status, words, 4, cudaMemcpyDeviceToHost, st));
  SH_TRY(cudaStreamSynchronize(st));
  if (split_status == ST_INVALID_ARG) return KDT_ERR_INVALID_ARG;
  for (kdt_status x : status)
    if (x != KDT_OK) return x;

  // ---- merge the shards' leaves
  MergeArgs m{};
  m.shards = G;
  m.L = L;
  m.nl = nl;
  m.offs_sh = offs_sh;
  m.vals_sh = vals_sh;
  m.dims_sh = dims_sh;
  m.perm_sh = perm_sh;
  m.base = a.base;
  m.ntot = a.ntot;
  m.gidx = a.gidx;
  m.pre = (uint32_t*)(ws + o_pre);
  m.offs = out_offs;
  m.vals = out_vals;
  m.dims = out_dims;
  m.perm = out_perm;
  m.terms = (TermRec*)(ws + o_terms);
  m.term_count = (uint32_t*)(words + 2);
  m.status = words + 1;
  {
    TraceScope ts(K_SHARD_MERGE, st, (uint64_t)n);
    k_sh_merge_offsets<<<std::min<uint32_t>((nl + 256) / 256, 4096u), 256, 0, st>>>(m);
    if (nl > 1) k_sh_merge_splits<<<std::min<uint32_t>((nl + 255) / 256, 4096u), 256, 0, st>>>(m);
    if (n) k_sh_merge_perm<<<(uint32_t)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, st>>>(m, (uint32_t)n);
    k_sh_terms<<<std::min<uint32_t>((nl + 255) / 256, 4096u), 256, 0, st>>>(m);
  }
  SH_TRY(cudaGetLastError());
  // each leaf in increasing original index: the library's leaf sort over a
  // view of the merged output
  TreeDev td{};
  td.n = n;
  td.d = d;
  td.r = p.r;
  td.out_perm = out_perm;
  td.terms = m.terms;
  td.term_cap = nl;
  td.term_count = m.term_count;
  td.huge = (uint32_t*)(ws + o_huge);
  td.huge_count = (uint32_t*)(words + 3);
  td.huge_cap = nl;
  td.status = words + 1;
  TreeDev* td_dev = (TreeDev*)(ws + o_td);
  uint32_t* slot_dev = (uint32_t*)(ws + o_slot);
  const uint32_t zero = 0;
  SH_TRY(cudaMemcpyAsync(td_dev, &td, sizeof td, cudaMemcpyHostToDevice, st));
  SH_TRY(cudaMemcpyAsync(slot_dev, &zero, 4, cudaMemcpyHostToDevice, st));
  launch_leaf_sort(td_dev, slot_dev, 1, nl, st);
  SH_TRY(cudaGetLastError());
  uint32_t nh = 0;
  int32_t merge_status = 0;
  SH_TRY(cudaMemcpyAsync(&nh, words + 3, 4, cudaMemcpyDeviceToHost, st));
  SH_TRY(cudaMemcpyAsync(&merge_status, words + 1, 4, cudaMemcpyDeviceToHost, st));
  SH_TRY(cudaStreamSynchronize(st));
  if (merge_status != ST_OK) return KDT_ERR_CUDA;  // the shards disagreed on a split (an internal error)
  nh = std::min(nh, nl);
  if (nh) {
    std::vector<uint32_t> idx(nh);
    std::vector<TermRec> all(nl), recs;
    SH_TRY(cudaMemcpyAsync(idx.data(), td.huge, (size_t)nh * 4, cudaMemcpyDeviceToHost, st));
    SH_TRY(cudaMemcpyAsync(all.data(), m.terms, (size_t)nl * sizeof(TermRec), cudaMemcpyDeviceToHost, st));
    SH_TRY(cudaStreamSynchronize(st));
    for (uint32_t k : idx)
      if (k < nl) recs.push_back(all[k]);
    // the shards' permutations and points are free now: key and tile scratch
    SH_TRY(leaf_sort_huge(TreeHost{(uint64_t)n, out_perm, perm_sh, (void*)a.xs, (size_t)d * n * 4}, recs, st));
  }
  SH_TRY(cudaStreamSynchronize(st));
  if (out_levels) *out_levels = L;
  return KDT_OK;
}

}  // namespace

}  // namespace kdt

extern "C" kdt_status kdt_build_sharded(const float* points, const kdt_params* p, int32_t shards, uint32_t* out_perm,
                                        float* out_split_vals, int8_t* out_split_dims, int64_t* out_node_offsets,
                                        int32_t* out_levels, void* stream) {
  const kdt_status v = kdt::validate_params(p);
  if (v != KDT_OK) return v;
  if (p->depth < 1 || p->fourier_j != 0 || shards < 1 || shards > kdt::kMaxShards) return KDT_ERR_INVALID_ARG;
  if ((p->n > 0 && (!points || !out_perm)) || !out_node_offsets || !out_split_vals || !out_split_dims)
    return KDT_ERR_INVALID_ARG;
  if (kdt::capturing((cudaStream_t)stream)) return KDT_ERR_INVALID_ARG;  // the build waits on its stream
  return kdt::sharded_build(points, *p, shards, out_perm, out_split_vals, out_split_dims, out_node_offsets,
                            out_levels, (cudaStream_t)stream);
}
