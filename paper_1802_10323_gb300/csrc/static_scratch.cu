// static_scratch.cu — ps_solve_static: the solve of ps_solve with its workspace
// in a fixed device array compiled into the library, for callers that cannot
// allocate device memory when they solve.
//
// The array is a file-scope __device__ object of kStaticScratchBytes; every GPU
// on which the library's module is loaded holds it until the process exits. In
// host code its name is only a host-side stand-in, so the device address is
// obtained once per device with cudaGetSymbolAddress (with that device current)
// and cached. Nothing here calls cudaMalloc, cudaFree or an allocating library
// routine.
#include <mutex>
#include <stdio.h>

#include "internal.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)8 << 20;  // 8 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

}  // namespace

extern "C" {

ps_status ps_solve_static(ps_plan* plan, const double* f, double* p, void* stream, ps_info* info) {
  if (!plan) return PS_INVALID_ARG;
  size_t need = 0;
  ps_status st = ps_workspace_bytes(plan, &need);
  if (st != PS_OK) return st;
  char msg[256];
  if (need > kStaticScratchBytes) {
    snprintf(msg, sizeof(msg),
             "ps_solve_static: this plan needs %zu bytes of workspace, the static scratch holds %zu "
             "(use ps_solve with a caller-allocated workspace)",
             need, kStaticScratchBytes);
    ps::set_plan_error(plan, msg);
    return PS_UNSUPPORTED_SIZE;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    snprintf(msg, sizeof(msg), "ps_solve_static: cudaGetDevice: %s", cudaGetErrorString(e));
    ps::set_plan_error(plan, msg);
    return PS_CUDA_ERROR;
  }
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      // first call on this device: resolve the array's device address
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess || !ptr) {
        snprintf(msg, sizeof(msg), "ps_solve_static: cudaGetSymbolAddress: %s",
                 cudaGetErrorString(e));
        ps::set_plan_error(plan, msg);
        return PS_CUDA_ERROR;
      }
      g_scratch_addr[dev] = ptr;
    }
    ws = g_scratch_addr[dev];
  }
  return ps_solve(plan, f, p, ws, stream, info);
}

}  // extern "C"
