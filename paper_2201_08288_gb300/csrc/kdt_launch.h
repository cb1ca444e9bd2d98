// kdt_launch.h -- host-side declarations shared by the CUDA translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "kdt_internal.cuh"

namespace kdt {

// Per-level local cell of the subtree kernel (kept in a per-CTA slice of
// global memory).
struct LCell {
  uint32_t begin;   // local position
  uint32_t count;
  uint32_t heap;
  int32_t stall;
  uint32_t dim;
  uint32_t mkey;
  uint32_t lcount;
  uint32_t pad;
};

// Shared-memory budget of the subtree kernel.
constexpr size_t kSubtreeSmemBytes = 231424;        // dynamic part
constexpr int kSubtreeBigBinCap = 1024;
constexpr size_t kSubtreeFixedBytes =
    (size_t)(kSubtreeBins + 1) * 4 + (size_t)kSubtreeBins * 4 + (size_t)kSubtreeWarps * 256 * 4 +
    (size_t)kSubtreeBigBinCap * 2;

// Largest cell (points) the subtree kernel holds for d coordinates: keys
// (4d bytes), permutation (4), subset id (2), two orders, cell ids and the
// scan (2 each, +2 once).
inline int subtree_capacity(int d) {
  const size_t per_point = 4 * (size_t)d + 14;
  size_t cap = (kSubtreeSmemBytes - kSubtreeFixedBytes - 2) / per_point;
  if (cap > 8192) cap = 8192;
  cap &= ~(size_t)31;
  return (int)cap;
}

void launch_big_step(const TreeDev* trees, const StepDev& s, uint32_t max_tiles, uint32_t nseg,
                     uint32_t max_bigseg, bool any_widest, cudaStream_t st);

cudaError_t prepare_subtree_kernel();
void launch_subtree(const TreeDev* trees, const Cell* list, uint32_t count, uint32_t* head, LCell* slices,
                    uint32_t slice_cells, uint32_t grid, cudaStream_t st);

void launch_iota(uint32_t* out, uint32_t n, cudaStream_t st);

void launch_finalize(const TreeDev* tree, const uint32_t* term_count, uint32_t max_terms, cudaStream_t st);

}  // namespace kdt
