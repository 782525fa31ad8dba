// Solve without any allocation: the workspace is a fixed device array.
//
// Some callers cannot call cudaMalloc when they solve: a model driver whose time
// loop must not allocate (cudaMalloc can synchronise the device and has
// unbounded latency), or a host program that owns the device memory pool and
// hands this library only field pointers.  For them, poisson_solve_static_workspace
// runs the ordinary solve with its scratch in the file-scope array below instead
// of a caller-provided workspace.  The array has a fixed maximum size and is held
// by every GPU that loads this library until the process exits.
#include <mutex>

#include "../../include/poisson.h"

namespace {

static __device__ __align__(256) unsigned char g_static_workspace[POISSON_STATIC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_device_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int poisson_solve_static_workspace(poisson_plan* plan, const void* S, void* p, void* stream,
                                              poisson_info* info) {
  if (!plan || !S || !p) return POISSON_ERR_INVALID_ARG;
  size_t need = 0;
  int rc = poisson_plan_workspace_bytes(plan, &need);
  if (rc != POISSON_OK) return rc;
  if (need > (size_t)POISSON_STATIC_WORKSPACE_BYTES) return POISSON_ERR_WORKSPACE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return POISSON_ERR_CUDA;
  void* ptr = nullptr;
  {
    // First call on a device: look up the device address of the array with that
    // device current.  In host code the array's name is only a stand-in, never a
    // device address.
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_device_ptr[dev]) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_static_workspace) != cudaSuccess || !addr) return POISSON_ERR_CUDA;
      g_device_ptr[dev] = addr;
    }
    ptr = g_device_ptr[dev];
  }
  // the solve clears the parts of its scratch that must start at zero
  return poisson_solve(plan, S, p, ptr, stream, info);
}
