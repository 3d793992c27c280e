// xform_col.cu — y-axis line transforms with the lines spread across lanes.
//
// Same mathematics as the other line transforms (one M-point complex FFT per
// line of n = 2M reals, with the Table 2 pre/post processing per BC), laid out
// for lines that are strided in memory. A CTA owns CW = 16 consecutive x columns
// of one z plane: lane c of each half-warp is column x0 + c, and the TPL threads
// that share a column split its line, E = M/TPL complex points each.
//   * Every global access is a row segment of CW consecutive x values (64 bytes
//     in FP32), and the BC pre/post processing happens at that interface: the
//     forward transform gathers its first-stage operands straight from the
//     permuted rows, and both directions write their outputs straight to rows.
//     No shared-memory transpose of the lines is needed.
//   * Stockham stages of radix R | E with the operands in registers; between
//     stages the line goes through a shared buffer laid out [index][column], so
//     each half-warp reads or writes 16 consecutive complex values: two
//     wavefronts per warp access, whatever the index pattern.
//   * A column's threads span several warps, so the exchanges synchronise the
//     CTA; twiddles come from shared tables loaded once per persistent CTA.
#include "xform_units.cuh"

namespace ps {
namespace col {

template <class T, int M, bool FWD, int CW>
__global__ void __launch_bounds__(CShape<M, CW>::NT, sizeof(T) == 4 ? 1024 / CShape<M, CW>::NT : 1)
    xform_col_kernel(FastArgs<T> a) {
  if (a.skip && *a.skip) return;
  static_assert(CShape<M, CW>::radix(0) == CShape<M, CW>::E, "the first stage takes all of a thread's points");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* stw = reinterpret_cast<cplx<T>*>(smem_raw);  // ω_M^t, t < M
  cplx<T>* ptw = stw + M;                               // e^{−2πik/n}, k ≤ M
  cplx<T>* xtw = ptw + (M + 1);                         // NN/DD: e^{−iπq/2n}, q < n; ND: pre, post
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw + fast_table_bytes<T, M>(a.bc));  // [M][CW]
  load_line_tables<T, M>(a.tw, a.bc, stw);
  const int ntiles = a.nz * (a.nx / CW);
  const int tpz = a.nx / CW;
  for (int g = blockIdx.x; g < ntiles; g += gridDim.x) {
    // forward: ask L2 for the rows of this CTA's next tile, so that its loads do not
    // wait on HBM (measured at 1024³: −5 % forward; the backward tiles gain nothing)
    const int gn = g + gridDim.x;
    if (FWD && gn < ntiles) {
      const int zb = gn / tpz, x0 = (gn - zb * tpz) * CW;
      const T* nb = static_cast<const T*>(a.in) + (size_t)zb * a.ny * a.nx + x0;
      for (int q = threadIdx.x; q < a.ny; q += blockDim.x)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(nb + (size_t)q * a.nx));
    }
    col_tile<T, M, FWD, CW>(a, stw, ptw, xtw, buf, g);
  }
}

}  // namespace col

namespace {
template <class T, int M, bool FWD, int CW>
cudaError_t launch_col_cw(FastArgs<T> a, cudaStream_t st) {
  using S = col::CShape<M, CW>;
  auto k = col::xform_col_kernel<T, M, FWD, CW>;
  const size_t smem = col::col_smem<T, M, CW>(a.bc);
  static int smem_set = 0;
  static int blocks_per_sm[2] = {};  // [bc != P]
  if (!smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)col::col_smem<T, M, CW>(1));
    if (e != cudaSuccess) return e;
    smem_set = 1;
  }
  int& bps = blocks_per_sm[a.bc != 0];
  if (bps == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, S::NT, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = a.nz * (a.nx / CW);
  const int grid = ntiles < sms * bps ? ntiles : sms * bps;
  (void)cudaGetLastError();  // a stale error from elsewhere must not be blamed here
  k<<<grid, S::NT, smem, st>>>(a);
  return cudaGetLastError();
}
}  // namespace

// Tiles of 16 columns: 64-byte rows in FP32, 128-byte rows in FP64.
template <class T, int M, bool FWD>
cudaError_t launch_xform_col(FastArgs<T> a, cudaStream_t st) {
  constexpr int CW = 16;  // (measured at 1024^3: 8 and 32 columns are slower)
  if (a.axis != 1 || a.ny != 2 * M || a.nx % CW != 0 || a.accumulate || a.amax)
    return cudaErrorInvalidValue;
  return launch_col_cw<T, M, FWD, CW>(a, st);
}

#define PS_COL_INST(M)                                                                              \
  template cudaError_t launch_xform_col<float, M, true>(FastArgs<float>, cudaStream_t);           \
  template cudaError_t launch_xform_col<float, M, false>(FastArgs<float>, cudaStream_t);          \
  template cudaError_t launch_xform_col<double, M, true>(FastArgs<double>, cudaStream_t);         \
  template cudaError_t launch_xform_col<double, M, false>(FastArgs<double>, cudaStream_t);

PS_COL_INST(64)
PS_COL_INST(128)
PS_COL_INST(256)
PS_COL_INST(512)

}  // namespace ps
