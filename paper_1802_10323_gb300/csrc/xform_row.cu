// xform_row.cu — x-axis line transforms read and written by the warp that owns the line.
//
// Same mathematics as the other line transforms (one M-point complex FFT per
// line of n = 2M contiguous reals, with the Table 2 pre/post processing per BC).
// TPL = M/E lanes own a line (a warp, or half of one for M = 64), E complex
// points each, and nothing but the FFT exchanges goes through shared memory:
//   * Lane t's first-stage operands are the points t + TPL·j, so for each j the
//     lanes of a line touch consecutive memory. The forward gather loads its
//     operands straight from the line: P reads pairs (x_{2p}, x_{2p+1}); the
//     cosine/sine orderings read one 4-vector (x_{4p} … x_{4p+3}) that holds two
//     values of point p and two of point M−1−p, and point M−1−p is the mirrored
//     slot E−1−s of the mirrored lane t ^ (TPL−1): one shuffle hands them over.
//     The backward outputs are assembled into the same vectors the same way.
//   * The other side of each transform (forward outputs, backward inputs) pairs
//     wavenumbers k and M−k; those go through the line's exchange buffer and
//     touch memory with scalar accesses at consecutive or every-other address.
//   * A line never leaves its warp: exchanges synchronise with __syncwarp, and
//     warps stride over the lines independently (persistent grid).
#include <type_traits>

#include "xform_units.cuh"

namespace ps {
namespace row {

template <class T, class TI, class TO, int M, bool FWD, int OM>
__global__ void __launch_bounds__(32 * WARPS, sizeof(T) == 4 ? (M >= 512 ? 3 : 4) : 2)
    xform_row_kernel(FastArgs<T> a) {
  if (a.skip && *a.skip) return;
  constexpr int LPW = 32 / Shape<M>::TPL;
  constexpr int LB = M + M / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* stw = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* ptw = stw + M;
  cplx<T>* xtw = ptw + (M + 1);
  cplx<T>* bufs = reinterpret_cast<cplx<T>*>(smem_raw + fast_table_bytes<T, M>(a.bc));
  load_line_tables<T, M>(a.tw, a.bc, stw);
  __syncthreads();  // the only block-wide barrier: tables ready
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // max |transform output| of FP64 outputs, tracked on the values before widening
  // (exact) so that no 64-bit work per value reaches the FP64 pipe
  T tmax = (T)0;
  const int wstride = gridDim.x * WARPS * LPW;
  for (int l0 = (blockIdx.x * WARPS + warp) * LPW; l0 < a.nlines; l0 += wstride)
    row_line<T, TI, TO, M, FWD, OM>(a, stw, ptw, xtw, bufs + warp * LPW * LB, l0, tmax);
  if constexpr (sizeof(TO) == 8) {
    if (a.amax) {
      for (int o = 16; o > 0; o >>= 1) tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
      const unsigned long long amax =
          (unsigned long long)__double_as_longlong(st_cvt<double, T>::f(tmax));  // ≥ 0: the bits order as the values
      if (lane == 0 && amax) atomicMax(a.amax, amax);
    }
  }
}

}  // namespace row

namespace {
template <class T, class TI, class TO, int M, bool FWD, int OM>
cudaError_t launch_row_mode(FastArgs<T> a, cudaStream_t st) {
  using S = fast::Shape<M>;
  constexpr int LPW = 32 / S::TPL;
  constexpr size_t LB = M + M / 8;
  auto k = row::xform_row_kernel<T, TI, TO, M, FWD, OM>;
  const size_t smem = fast_table_bytes<T, M>(a.bc) + (size_t)row::WARPS * LPW * LB * sizeof(cplx<T>);
  static int smem_set = 0;
  static int blocks_per_sm[2] = {};
  if (!smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(fast_table_bytes<T, M>(1) + row::WARPS * LPW * LB * sizeof(cplx<T>)));
    if (e != cudaSuccess) return e;
    smem_set = 1;
  }
  int& bps = blocks_per_sm[a.bc != 0];
  if (bps == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, 32 * row::WARPS, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_cta = row::WARPS * LPW;
  const int ctas = (a.nlines + per_cta - 1) / per_cta;
  const int grid = ctas < sms * bps ? ctas : sms * bps;
  (void)cudaGetLastError();  // a stale error from elsewhere must not be blamed here
  k<<<grid, 32 * row::WARPS, smem, st>>>(a);
  return cudaGetLastError();
}
}  // namespace

template <class T, class TI, class TO, int M, bool FWD>
cudaError_t launch_xform_row(FastArgs<T> a, cudaStream_t st) {
  if (a.axis != 0 || a.nx != 2 * M) return cudaErrorInvalidValue;
  if constexpr (!FWD && sizeof(TO) == 8 && sizeof(T) == 4) {
    if (a.base32) return launch_row_mode<T, TI, TO, M, FWD, row::OM_BASE>(a, st);
    if (!a.out) return launch_row_mode<T, TI, TO, M, FWD, row::OM_NONE>(a, st);
  }
  if (a.accumulate) return launch_row_mode<T, TI, TO, M, FWD, row::OM_ACC>(a, st);
  return launch_row_mode<T, TI, TO, M, FWD, row::OM_STORE>(a, st);
}

#define PS_ROW_INST(M)                                                                                   \
  template cudaError_t launch_xform_row<double, double, double, M, true>(FastArgs<double>, cudaStream_t); \
  template cudaError_t launch_xform_row<double, double, double, M, false>(FastArgs<double>, cudaStream_t); \
  template cudaError_t launch_xform_row<float, float, float, M, true>(FastArgs<float>, cudaStream_t);     \
  template cudaError_t launch_xform_row<float, float, float, M, false>(FastArgs<float>, cudaStream_t);    \
  template cudaError_t launch_xform_row<float, double, float, M, true>(FastArgs<float>, cudaStream_t);    \
  template cudaError_t launch_xform_row<float, float, double, M, false>(FastArgs<float>, cudaStream_t);

PS_ROW_INST(64)
PS_ROW_INST(128)
PS_ROW_INST(256)
PS_ROW_INST(512)

}  // namespace ps
