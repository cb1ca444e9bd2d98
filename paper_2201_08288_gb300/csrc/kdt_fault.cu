// kdt_fault.cu -- host-side fault injection (kdt_fault_inject) and the
// library's one device-allocation call.
//
// Each fault kind holds a count of the events it still fails. Nothing here
// touches the GPU: an injected allocation failure returns before cudaMalloc
// is called, an injected server-step failure before anything is launched,
// and the subtree wait probe is a bounded wait on a barrier with no copy in
// flight (the kernel reads the probe's bound as a launch argument).
#include <atomic>

#include "kdt.h"
#include "kdt_launch.h"

namespace kdt {

namespace {
constexpr int kKinds = 5;
std::atomic<int32_t> g_fault[kKinds];
}  // namespace

bool fault_take(int kind) {
  if (kind <= 0 || kind >= kKinds) return false;
  int32_t v = g_fault[kind].load(std::memory_order_relaxed);
  while (v > 0)
    if (g_fault[kind].compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return true;
  return false;
}

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (fault_take(KDT_FAULT_ALLOC)) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

}  // namespace kdt

extern "C" {

kdt_status kdt_fault_inject(kdt_fault kind, int32_t count) {
  if ((int)kind <= 0 || (int)kind >= kdt::kKinds || count < 0) return KDT_ERR_INVALID_ARG;
  kdt::g_fault[(int)kind].store(count);
  return KDT_OK;
}

void kdt_fault_clear(void) {
  for (int k = 0; k < kdt::kKinds; ++k) kdt::g_fault[k].store(0);
}

}  // extern "C"
