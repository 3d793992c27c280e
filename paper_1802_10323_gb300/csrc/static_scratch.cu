// static_scratch.cu — ps_solve_static: the solve of ps_solve with its workspace
// in a fixed device array compiled into the library, for callers that cannot
// allocate device memory when they solve.
//
// The array is a file-scope __device__ object of kStaticScratchBytes; every GPU
// on which the library's module is loaded holds it until the process exits. In
// host code its name is only a host-side stand-in, so the device address is
// obtained with cudaGetSymbolAddress (with that device current) and cached per
// device together with the id of the CUDA context it belongs to: a context
// created anew on that device (after cudaDeviceReset, which unloads the module)
// may hold the array elsewhere, so the address is looked up again then. Nothing
// here calls cudaMalloc, cudaFree or an allocating library routine.
#include <cuda.h>
#include <mutex>
#include <stdio.h>

#include "internal.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)8 << 20;  // 8 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
struct Slot {
  unsigned long long ctx_id;  // context the address was resolved in
  void* addr;
};
Slot g_slot[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Driver entry points for the current context's unique id (CUDA 12.0+), taken
// through the runtime so that the library needs no link-time libcuda.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return false;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

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
    // the context the solve's kernels will run in; if none is current yet the
    // runtime has not initialised dev, and cudaSetDevice makes its primary
    // context current (a device that is current already stays so)
    unsigned long long ctx_id = 0;
    bool have = current_context_id(&ctx_id);
    if (!have && cudaSetDevice(dev) == cudaSuccess) have = current_context_id(&ctx_id);
    if (!have) {
      snprintf(msg, sizeof(msg), "ps_solve_static: cannot identify the current CUDA context");
      ps::set_plan_error(plan, msg);
      return PS_CUDA_ERROR;
    }
    Slot& s = g_slot[dev];
    if (!s.addr || s.ctx_id != ctx_id) {
      // first call on this device (or in a new context on it): resolve the
      // array's device address
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess || !ptr) {
        snprintf(msg, sizeof(msg), "ps_solve_static: cudaGetSymbolAddress: %s",
                 cudaGetErrorString(e));
        ps::set_plan_error(plan, msg);
        return PS_CUDA_ERROR;
      }
      s.addr = ptr;
      s.ctx_id = ctx_id;
    }
    ws = s.addr;
  }
  return ps_solve(plan, f, p, ws, stream, info);
}

}  // extern "C"
