// xform.cu — launchers of the generic line transforms (device code in xform_dev.cuh).
#include "xform_dev.cuh"

namespace ps {

template <class T, class TI, class TO, bool FWD>
__global__ void __launch_bounds__(256) xform_kernel(XformArgs<T> a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  xform_group<T, TI, TO, FWD>(a, blockIdx.x, smem_raw);
}

// ---- host-side launcher ------------------------------------------------------------------

template <class T>
int pick_lines(int n, int axis, int nx, int nlines) {
  const size_t per_line = 2 * (size_t)(n / 2 + 1) * 2 * sizeof(T);
  int L = (int)(65536 / per_line);
  if (L < 1) L = 1;
  if (L > 64) L = 64;
  if (axis == 1) {
    while (L > 1 && nx % L) --L;
  } else if (L > nlines) {
    L = nlines;
  }
  return L;
}

template <class T, class TI, class TO, bool FWD>
cudaError_t launch_xform(XformArgs<T> a, cudaStream_t st) {
  // (pick_lines sizes the buffers for m = n/2; a face-centred line's FFT has m = n)
  a.L = pick_lines<T>(a.m == a.n ? 2 * a.n : a.n, a.axis, a.nx, a.nlines);
  const size_t smem = 2 * (size_t)a.L * (a.m + 1) * sizeof(cplx<T>);
  int grid = (a.axis == 0) ? (a.nlines + a.L - 1) / a.L : a.nz * (a.nx / a.L);
  auto k = xform_kernel<T, TI, TO, FWD>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_xform<double, double, double, true>(XformArgs<double>, cudaStream_t);
template cudaError_t launch_xform<double, double, double, false>(XformArgs<double>, cudaStream_t);
template cudaError_t launch_xform<float, float, float, true>(XformArgs<float>, cudaStream_t);
template cudaError_t launch_xform<float, float, float, false>(XformArgs<float>, cudaStream_t);
template cudaError_t launch_xform<float, double, float, true>(XformArgs<float>, cudaStream_t);
template cudaError_t launch_xform<float, float, double, false>(XformArgs<float>, cudaStream_t);
template int pick_lines<float>(int, int, int, int);
template int pick_lines<double>(int, int, int, int);

}  // namespace ps
