// kdt_noalloc.cu -- a build entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: a host application that hands the GPU
// to this library under a fixed device-memory budget already owned by its own
// allocator, or a latency-critical path where cudaMalloc's cost and its
// implicit device-wide synchronisation are not acceptable. For them,
// kdt_build_noalloc runs the same build with its workspace in a file-scope
// device array of fixed size (kdt_noalloc_scratch below), which the CUDA
// runtime creates when it loads this module on a device and keeps until the
// process exits. The caller still passes the points and the output buffers.
#include <mutex>

#include "kdt.h"
#include "kdt_launch.h"
#include "kdt_trace.h"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)64 << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

// The shared workspace. In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) uint8_t kdt_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" kdt_status kdt_build_noalloc(const float* points, const kdt_params* p, uint32_t* out_perm,
                                        float* out_split_vals, int8_t* out_split_dims,
                                        int64_t* out_node_offsets, int32_t* out_levels, void* stream) {
  size_t need = 0;
  const kdt_status v = kdt_workspace_size(p, &need);
  if (v != KDT_OK) return v;
  if (need > kNoallocScratchBytes) return KDT_ERR_CAPACITY;  // problem too large for the fixed scratch
  if (kdt::capturing((cudaStream_t)stream)) return KDT_ERR_INVALID_ARG;  // the build waits on its stream
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return KDT_ERR_CUDA;
  }
  void* scratch = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, kdt_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
        (void)cudaGetLastError();
        return KDT_ERR_CUDA;
      }
      g_scratch_addr[dev] = ptr;
    }
    scratch = g_scratch_addr[dev];
  }
  // The build clears every counter it relies on at its start, so the previous
  // call's leftovers in the scratch array do not matter.
  return kdt::build_in_workspace(points, p, scratch, kNoallocScratchBytes, out_perm, out_split_vals,
                                 out_split_dims, out_node_offsets, out_levels, (cudaStream_t)stream);
}
