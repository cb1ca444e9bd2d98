// kdt_tune.cu -- the tuning of the select paths (which kernel takes a
// (cell, subset) segment of a given size, and the shape of the CTA radix
// select) and the autotuner that times candidate tunings on the caller's
// trees. The tuning changes only speed: every path computes the exact lower
// median (paper, Sec. 2), so outputs are identical under every choice.
#include <cuda_runtime.h>

#include <mutex>

#include "kdt.h"
#include "kdt_launch.h"

namespace kdt {
namespace {

std::mutex g_mu;
kdt_tuning g_tuning = {64, 256, 4096, 256, 11, {0, 0, 0}};

template <size_t N>
bool one_of(int32_t v, const int32_t (&choices)[N]) {
  for (int32_t c : choices)
    if (v == c) return true;
  return false;
}

const int32_t kTiny[] = {8, 16, 32, 64};
const int32_t kBitonic[] = {64, 128, 256};
const int32_t kWarp[] = {1024, 2048, 4096};
const int32_t kThreads[] = {256, 512};
const int32_t kBits[] = {8, 11};

bool valid(const kdt_tuning& t) {
  return one_of(t.tiny_max, kTiny) && one_of(t.bitonic_max, kBitonic) && one_of(t.warp_max, kWarp) &&
         one_of(t.cta_threads, kThreads) && one_of(t.digit_bits, kBits) && t.reserved[0] == 0 &&
         t.reserved[1] == 0 && t.reserved[2] == 0;
}

}  // namespace

SelectTuning current_tuning() {
  std::lock_guard<std::mutex> lk(g_mu);
  return SelectTuning{(uint32_t)g_tuning.tiny_max, (uint32_t)g_tuning.bitonic_max, (uint32_t)g_tuning.warp_max,
                      g_tuning.cta_threads, g_tuning.digit_bits};
}

}  // namespace kdt

extern "C" {

void kdt_tuning_default(kdt_tuning* t) {
  if (t) *t = kdt_tuning{64, 256, 4096, 256, 11, {0, 0, 0}};
}

kdt_status kdt_set_tuning(const kdt_tuning* t) {
  kdt_tuning v;
  if (t) {
    v = *t;
    if (!kdt::valid(v)) return KDT_ERR_INVALID_ARG;
  } else {
    kdt_tuning_default(&v);
  }
  std::lock_guard<std::mutex> lk(kdt::g_mu);
  kdt::g_tuning = v;
  return KDT_OK;
}

kdt_status kdt_get_tuning(kdt_tuning* t) {
  if (!t) return KDT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(kdt::g_mu);
  *t = kdt::g_tuning;
  return KDT_OK;
}

kdt_status kdt_autotune(const kdt_tree_desc* trees, int32_t num_trees, void* workspace, size_t workspace_bytes,
                        int32_t repeats, kdt_tuning* best, float* best_ms, void* stream) {
  if (!best || repeats < 1 || repeats > 100) return KDT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  kdt_tuning saved;
  kdt_get_tuning(&saved);
  size_t need = 0;
  kdt_status s = kdt_workspace_size_batched(trees, num_trees, &need);
  if (s != KDT_OK) return s;
  void* owned = nullptr;
  if (!workspace) {
    if (kdt::dev_malloc(&owned, need) != cudaSuccess) {
      (void)cudaGetLastError();
      return KDT_ERR_OOM;
    }
    workspace = owned;
    workspace_bytes = need;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto finish = [&](kdt_status r) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (owned) {
      cudaStreamSynchronize(st);
      cudaFree(owned);
    }
    if (r != KDT_OK) kdt_set_tuning(&saved);
    return r;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return finish(KDT_ERR_CUDA);
  // one batched build per repeat under tuning c; ms per build
  auto time_one = [&](const kdt_tuning& c, float* ms) -> kdt_status {
    kdt_status r = kdt_set_tuning(&c);
    if (r != KDT_OK) return r;
    if (cudaEventRecord(e0, st) != cudaSuccess) return KDT_ERR_CUDA;
    for (int32_t i = 0; i < repeats; ++i) {
      r = kdt_build_batched(trees, num_trees, workspace, workspace_bytes, nullptr, nullptr, stream);
      if (r != KDT_OK) return r;
    }
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return KDT_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return KDT_ERR_CUDA;
    *ms = t / (float)repeats;
    return KDT_OK;
  };
  s = kdt_build_batched(trees, num_trees, workspace, workspace_bytes, nullptr, nullptr, stream);  // warm-up
  if (s != KDT_OK) return finish(s);
  kdt_tuning b = saved;
  float b_ms = 0.f;
  if ((s = time_one(b, &b_ms)) != KDT_OK) return finish(s);
  // coordinate sweep: each field over its choices, the others at the best so far
  struct Field {
    int32_t kdt_tuning::*f;
    const int32_t* choices;
    int n;
  };
  const Field fields[] = {{&kdt_tuning::tiny_max, kdt::kTiny, 4},
                          {&kdt_tuning::bitonic_max, kdt::kBitonic, 3},
                          {&kdt_tuning::warp_max, kdt::kWarp, 3},
                          {&kdt_tuning::cta_threads, kdt::kThreads, 2},
                          {&kdt_tuning::digit_bits, kdt::kBits, 2}};
  for (const Field& fd : fields)
    for (int k = 0; k < fd.n; ++k) {
      if (fd.choices[k] == b.*(fd.f)) continue;
      kdt_tuning c = b;
      c.*(fd.f) = fd.choices[k];
      float ms = 0.f;
      if ((s = time_one(c, &ms)) != KDT_OK) return finish(s);
      if (ms < b_ms) {
        b = c;
        b_ms = ms;
      }
    }
  kdt_set_tuning(&b);
  *best = b;
  if (best_ms) *best_ms = b_ms;
  return finish(KDT_OK);
}

}  // extern "C"
