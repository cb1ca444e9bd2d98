// kdt_trace.cu -- launch counter and per-kernel event timing (see kdt_trace.h).
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "kdt.h"
#include "kdt_trace.h"

namespace kdt {
namespace {

const char* const kNames[K_NUM] = {
    "k_prep",       "k_tiles",      "k_ps_count",   "k_ps_offsets",  "k_ps_move",     "k_segs",
    "k_minmax",     "k_pick_dim",   "k_select_tiny", "k_select_small", "k_select_big", "k_combine",    "k_part_count",
    "k_part_scan",  "k_classify",   "k_part_scatter", "k_child_dims",  "k_subtree",
    "k_finalize",   "k_iota",       "k_leaf_sort",  "k_leaf_hist",   "k_leaf_scan",   "k_leaf_scatter",
    "k_leaf_copy",  "k_fourier_moments", "k_fourier_split", "k_shard_exchange", "k_shard_split",
    "k_shard_merge", "k_query"};

struct Pending {
  KernelId id;
  uint64_t units;
  cudaEvent_t a, b;
};

struct Tracer {
  std::atomic<uint64_t> launches{0};
  std::atomic<bool> on{false};
  std::mutex mu;
  std::vector<Pending> pending;
  uint64_t count[K_NUM] = {};
  uint64_t units[K_NUM] = {};
  double ms[K_NUM] = {};
};

Tracer& tracer() {
  static Tracer t;
  return t;
}

}  // namespace

// A launch recorded into a graph (stream capture) is counted but not timed:
// its events would be replayed by every launch of the graph.
bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

void trace_add_launches(uint64_t n) { tracer().launches.fetch_add(n, std::memory_order_relaxed); }

TraceScope::TraceScope(KernelId id, cudaStream_t st, uint64_t units) : id_(id), st_(st), units_(units) {
  Tracer& t = tracer();
  t.launches.fetch_add(1, std::memory_order_relaxed);
  if (t.on.load(std::memory_order_relaxed) && !capturing(st_)) {
    if (cudaEventCreate(&start_) == cudaSuccess) {
      cudaEventRecord(start_, st_);
    } else {
      (void)cudaGetLastError();
      start_ = nullptr;
    }
  }
}

TraceScope::~TraceScope() {
  // KDT_SYNC_CHECK=1: synchronise after every launch and name the kernel of
  // the first error (a debugging aid; off by default)
  static const bool sync_check = [] {
    const char* v = std::getenv("KDT_SYNC_CHECK");
    return v && *v && *v != '0';
  }();
  if (sync_check && !capturing(st_)) {
    const cudaError_t e = cudaStreamSynchronize(st_);
    if (e != cudaSuccess) std::fprintf(stderr, "kdt: %s: %s\n", kNames[id_], cudaGetErrorString(e));
  }
  if (!start_) return;
  cudaEvent_t stop = nullptr;
  if (cudaEventCreate(&stop) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaEventDestroy(start_);
    return;
  }
  cudaEventRecord(stop, st_);
  Tracer& t = tracer();
  std::lock_guard<std::mutex> g(t.mu);
  t.pending.push_back(Pending{id_, units_, start_, stop});
}

}  // namespace kdt

using namespace kdt;

extern "C" {

void kdt_trace_enable(int32_t on) { tracer().on.store(on != 0); }

uint64_t kdt_launch_count(void) { return tracer().launches.load(); }

int32_t kdt_trace_read(kdt_kernel_stat* out, int32_t max, int32_t reset) {
  Tracer& t = tracer();
  std::lock_guard<std::mutex> g(t.mu);
  for (const Pending& p : t.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      t.ms[p.id] += ms;
      t.count[p.id] += 1;
      t.units[p.id] += p.units;
    } else {
      (void)cudaGetLastError();
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  t.pending.clear();
  int32_t n = 0;
  for (int k = 0; k < K_NUM; ++k) {
    if (!t.count[k]) continue;
    if (out && n < max) {
      out[n].name = kNames[k];
      out[n].launches = t.count[k];
      out[n].total_ms = t.ms[k];
      out[n].units = t.units[k];
    }
    ++n;
  }
  if (reset) {
    for (int k = 0; k < K_NUM; ++k) {
      t.count[k] = 0;
      t.units[k] = 0;
      t.ms[k] = 0.0;
    }
  }
  return n;
}

}  // extern "C"
