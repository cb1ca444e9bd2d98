// kdt_launch.h -- host-side declarations shared by the CUDA translation units.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "kdt_internal.cuh"

namespace kdt {

// Per-level local cell of the subtree kernel (shared memory while a level's
// live cells fit the shape's table, else a per-CTA slice of global memory).
struct LCell {
  uint32_t heap;
  uint32_t mkey;    // split key
  uint16_t begin;   // local position
  uint16_t count;
  uint16_t lcount;  // left child size
  uint8_t dim;      // key coordinate
  uint8_t stall;    // consecutive splits that left the right child empty
};
static_assert(sizeof(LCell) == 16, "LCell is 16 bytes");

// The subtree kernel comes in two shapes (kSubtreeThreads threads per CTA in
// both); each tree uses one, by its coordinate count:
//   narrow (d <= kSubtreeNarrowMaxD): at most 5 positions per thread (1280
//     points), three CTAs per SM in 74 KB of dynamic shared memory each, cell
//     tables of 128 cells;
//   wide (larger d): at most 8 positions per thread (2048 points), two CTAs
//     per SM in 112 KB each, cell tables of 256 cells.
// Several CTAs share an SM, each finishing its own cell, so that one CTA's
// barriers and copies overlap the others' work.
struct SubtreeShape {
  int q;        // positions per thread
  int ctas;     // CTAs per SM
  size_t smem;  // dynamic shared memory per CTA
  int cells;    // cells of one level's table in shared memory
};
constexpr SubtreeShape kSubNarrow{5, 3, 74 * 1024, 128};
constexpr SubtreeShape kSubWide{8, 2, 112 * 1024, 256};
constexpr int kSubtreeNarrowMaxD = 8;
constexpr int kSubtreeBigCap = 64;           // segments above the rank-counting size (32): N / 33 < 64
constexpr int kSubtreeHistWords = kSubtreeWarps * 256;  // warp histograms; also the root's subset counts
__host__ __device__ constexpr size_t subtree_fixed_bytes(int cells) {
  return (size_t)kSubtreeHistWords * 4 + (size_t)kSubtreeBigCap * 2 + 2 * (size_t)cells * sizeof(LCell);
}
inline const SubtreeShape& subtree_shape(int d) { return d <= kSubtreeNarrowMaxD ? kSubNarrow : kSubWide; }

// Column stride (elements) of a cell of N points in shared memory: room for
// the 16-byte alignment phase of the bulk copies.
__host__ __device__ inline uint32_t subtree_stride(uint32_t N) { return (N + 8 + 3) & ~3u; }

// Bytes of shared memory a cell of N points with d coordinates needs beyond
// the fixed part: d key columns at the padded stride, the keys in local order
// and the segment medians (4 bytes each), the subset ids, two orders, cell
// ids, a scan and the segment starts (2 bytes each).
__host__ __device__ inline size_t subtree_point_bytes(uint32_t N, int d) {
  const size_t stride = subtree_stride(N);
  return (size_t)d * stride * 4 + 2 * (((size_t)N * 4 + 15) & ~(size_t)15) +
         6 * ((((size_t)N + 1) * 2 + 15) & ~(size_t)15);
}

// Largest cell (points) the subtree kernel holds for d coordinates in the
// shape that trees of d coordinates use.
inline int subtree_capacity(int d) {
  if (d < 1) return 0;
  const SubtreeShape& sh = subtree_shape(d);
  const size_t fixed = subtree_fixed_bytes(sh.cells);
  int lo = 32, hi = 8192;
  if (fixed + subtree_point_bytes(lo, d) > sh.smem) return 0;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (fixed + subtree_point_bytes(mid, d) <= sh.smem) lo = mid; else hi = mid - 1;
  }
  return std::min(lo & ~31, sh.q * kSubtreeThreads);
}

// Subset counts of a small root (put in subset order by the subtree kernel)
// live in the warp histograms: trees with more subsets presort their root in
// the multi-CTA pipeline instead.
inline bool subtree_sorts_root(int r) { return r <= kSubtreeHistWords; }

// The tuning of the select paths (kdt_tuning, validated) in force when a level
// step starts.
struct SelectTuning {
  uint32_t tiny_max, bitonic_max, warp_max;
  int cta_threads, digit_bits;
};
SelectTuning current_tuning();

cudaError_t prepare_step_kernels();
// One thread: the loop condition of a graph whose body is a pair of level
// steps (keep going while ncells_next > 0, at most `limit` iterations; the
// count of iterations is kept in *iters).
void launch_loop_cond(cudaGraphConditionalHandle h, const uint32_t* ncells_next, uint32_t* iters, uint32_t limit,
                      cudaStream_t st);
void launch_big_step(const TreeDev* trees, const StepDev& s, uint32_t max_tiles, uint32_t nseg,
                     uint32_t max_bigseg, bool has_roots, bool need_root_dims, bool any_widest, int max_d, int uniform_d,
                     const SelectTuning& tune, uint64_t points, uint32_t sms, cudaStream_t st, bool fourier = false);

// Dynamic shared memory of the staged scatter (two CTAs per SM).
constexpr uint32_t kScatterSmemBytes = 100 * 1024;
cudaError_t prepare_scatter_kernel();
// uniform_d: the coordinate count of every tree of the step, 0 if they differ
// (a kernel compiled for that d is used where there is one)
void launch_scatter(const TreeDev* trees, const StepDev& s, uint32_t max_tiles, uint32_t grid_cap,
                    uint64_t points, int uniform_d, cudaStream_t st);

// Sharded build (kdt_shard.cu): the per-level exchanges among the shards of
// a step whose StepDev has shards > 0 (ncells_cap bounds the step's cells).
void launch_shard_index(const StepDev& s, uint32_t ncells_cap, cudaStream_t st);
void launch_shard_medians(const TreeDev* trees, const StepDev& s, uint32_t ncells_cap, cudaStream_t st);
void launch_shard_minmax(const TreeDev* trees, const StepDev& s, uint32_t ncells_cap, cudaStream_t st);

cudaError_t prepare_subtree_kernel();
// One launch of the subtree kernel in the given shape over a queue of small
// cells. count_dev: if set, the device word holding the queue's length
// (count is then its cap). reversed: the queue is filled from the end of the
// list (item j at list[count_cap - 1 - j], count_cap = count).
void launch_subtree(const SubtreeShape& sh, const TreeDev* trees, const Cell* list, uint32_t count,
                    const uint32_t* count_dev, bool reversed, uint32_t* head, LCell* slices, uint32_t slice_cells,
                    uint32_t grid, uint64_t points, cudaStream_t st);

void launch_iota(uint32_t* out, uint32_t n, cudaStream_t st);

// Leaf sort (kdt_leafsort.cu): terminal cells up to kLeafWarpMax points are
// sorted by one warp, up to kLeafBlockMax by one CTA; larger ones are listed
// in the tree's `huge` table and sorted by leaf_sort_huge.
constexpr int kLeafWarpMax = 256;
constexpr int kLeafBlockMax = 4096;
void launch_leaf_sort(const TreeDev* trees, const uint32_t* slots, uint32_t nslots, uint32_t max_records,
                      cudaStream_t st);
// Host view of a finished tree for the global leaf-sort passes: the
// permutation, a ping-pong buffer of n words and scratch for tile tables
// (the tree's working buffers, free once its build is done).
struct TreeHost {
  uint64_t n;
  uint32_t* out_perm;
  uint32_t* keys;
  void* scratch;
  size_t scratch_bytes;
};
size_t leaf_huge_tiles_cap(uint64_t n);
cudaError_t leaf_sort_huge(const TreeHost& th, const std::vector<TermRec>& recs, cudaStream_t st);

}  // namespace kdt

#include "kdt.h"

namespace kdt {

// Fault injection (kdt_fault.cu): true if an injected failure of this kind
// (a kdt_fault value) is due now; it is then consumed.
bool fault_take(int kind);
// The library's device allocations go through here (an injected
// KDT_FAULT_ALLOC fails it without calling cudaMalloc).
cudaError_t dev_malloc(void** p, size_t bytes);

kdt_status build_in_workspace(const float* points, const kdt_params* p, void* workspace, size_t workspace_bytes,
                              uint32_t* out_perm, float* out_split_vals, int8_t* out_split_dims,
                              int64_t* out_node_offsets, int32_t* out_levels, cudaStream_t st);

void launch_finalize_many(const TreeDev* trees, const uint32_t* slots, uint32_t nslots, uint32_t max_records,
                          cudaStream_t st);
void launch_finalize(const TreeDev* tree, const uint32_t* term_count, uint32_t max_terms, cudaStream_t st);

}  // namespace kdt
