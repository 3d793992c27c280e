// probe.cu — ps_probe_fp64: the FP64 FMA throughput of the current device, the
// denominator of the plain FP64 solve's roofline (that solve is bound by the FP64
// pipe on this part, not by HBM).
//
// Every thread runs eight independent chains of fused multiply-adds in FP64
// (x ← x·a + b, with a just below 1 so nothing overflows), enough chains per SM to
// keep the pipe busy; the result is stored so that nothing is eliminated. Timed
// with CUDA events on the caller's stream; two FLOPs per FMA.
#include <stdio.h>

#include "internal.h"

namespace ps {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_kernel(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace ps

extern "C" ps_status ps_probe_fp64(int iters, double* tflops, double* ms, void* stream) {
  if (iters < 1 || !tflops || !ms) return PS_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PS_CUDA_ERROR;
  const int blocks = sms * 8, threads = 256;
  double* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return PS_OUT_OF_MEMORY;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ps::fp64_fma_kernel<<<blocks, threads, 0, st>>>(out, iters / 8 + 1, 0.999999, 1e-7);  // warm-up
  cudaEventRecord(e0, st);
  ps::fp64_fma_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return PS_CUDA_ERROR;
  *ms = t;
  *tflops = 2.0 * ps::kChains * (double)iters * blocks * threads / (t * 1e-3) / 1e12;
  return PS_OK;
}
