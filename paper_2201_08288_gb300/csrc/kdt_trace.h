// kdt_trace.h -- launch counting and optional per-kernel CUDA-event timing.
//
// Every kernel launch of the library goes through a TraceScope. Launches are
// always counted; when tracing is enabled (kdt_trace_enable), the scope also
// records a CUDA event before and after the launch on the launching stream,
// and kdt_trace_read turns the pairs into per-kernel totals.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kdt {

enum KernelId {
  K_PREP, K_TILES, K_PS_COUNT, K_PS_OFFSETS, K_PS_MOVE, K_SEGS, K_MINMAX, K_PICK_DIM,
  K_SELECT_TINY, K_SELECT_SMALL, K_SELECT_BIG, K_COMBINE, K_PART_COUNT, K_PART_SCAN, K_CLASSIFY, K_PART_SCATTER,
  K_CHILD_DIMS, K_SUBTREE, K_FINALIZE, K_IOTA, K_LEAF_SORT, K_LEAF_HIST, K_LEAF_SCAN,
  K_LEAF_SCATTER, K_LEAF_COPY, K_FOURIER_MOMENTS, K_FOURIER_SPLIT, K_SHARD_EXCHANGE, K_SHARD_SPLIT,
  K_SHARD_MERGE, K_QUERY, K_NUM
};

// Launches replayed by a graph beyond the ones counted while it was captured.
void trace_add_launches(uint64_t n);
// True while `st` is being captured into a graph.
bool capturing(cudaStream_t st);

class TraceScope {
 public:
  // units: work items the launch processes (points), for bandwidth figures
  TraceScope(KernelId id, cudaStream_t st, uint64_t units = 0);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;

 private:
  KernelId id_;
  cudaStream_t st_;
  uint64_t units_;
  cudaEvent_t start_ = nullptr;
};

}  // namespace kdt
