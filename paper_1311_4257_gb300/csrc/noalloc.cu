// dfmm_apply_noalloc: the matvec without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: services that forbid
// allocation after start-up (the allocator is owned by someone else, or its
// latency and possible failure are not allowed on the request path), and
// hosts whose device memory is budgeted up front.  For them this entry point
// runs the same computation as dfmm_apply with every per-apply buffer taken
// from one file-scope device array of fixed size, which exists on every
// device that loads the library until the process exits.  The plan itself
// (built by dfmm_plan) is still allocated at plan time.
//
// Layout of the array: the device status word of the last apply at offset 0,
// then the rest of the workspace (the layout of dfmm_apply_workspace_bytes).
#include <mutex>

#include "common.h"
#include "dfmm.h"
#include "internal.h"

namespace {

// 64 MiB of scratch (dfmm_noalloc_capacity)
constexpr size_t kScratchBytes = (size_t)64 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
cudaStream_t g_last_stream[kMaxDevices] = {};   // stream of the last apply on each device

}  // namespace

namespace dfmm {

const unsigned* noalloc_status_word(cudaStream_t stream) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev] || g_last_stream[dev] != stream) return nullptr;
  return (const unsigned*)g_scratch_addr[dev];
}

}  // namespace dfmm

extern "C" int dfmm_apply_noalloc(dfmm_plan_t plan, const void* f, void* u, int nrhs, cudaStream_t stream) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dfmm::set_error(DFMM_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return dfmm::set_error(DFMM_ERR_UNSUPPORTED, "device index out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_addr[dev]) {
      // Host code cannot use the array's name as a device address: ask the
      // runtime for this device's copy (once per device, device current).
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return dfmm::set_error(DFMM_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
    g_last_stream[dev] = stream;
  }
  return dfmm::apply_with_scratch(plan, f, u, nrhs, stream, scratch, kScratchBytes);
}

extern "C" int64_t dfmm_noalloc_capacity(void) { return (int64_t)kScratchBytes; }
