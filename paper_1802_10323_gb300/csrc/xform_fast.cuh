// xform_fast.cuh — register-resident line transforms for n = 2M with M ∈ {64, 128, 256, 512}.
//
// Same mathematics as xform.cu (one M-point complex FFT per line of n reals
// with the Table 2 pre/post processing per BC), organised for throughput:
//   * TPL = M/E threads own one line, E complex points each (E = 16, 8, 4),
//     so a line lives in one warp (or a fraction of one) and stages synchronise
//     with __syncwarp only;
//   * Stockham stages of radix R | E; each thread does E/R butterflies per
//     stage with its operands in registers, exchanging through the line's own
//     shared-memory buffer between stages;
//   * all index arithmetic is compile-time (M is a template parameter);
//   * twiddles come from shared-memory tables loaded once per CTA; the grid is
//     persistent (CTAs stride over line groups);
//   * lines are staged through shared memory with 16-byte global accesses
//     (x: contiguous rows; y: a tile of LPC consecutive x columns, so every row
//     segment is LPC·sizeof(T) ≥ 64 bytes).
#pragma once
#include "internal.h"

namespace ps {
namespace fast {

template <int M>
struct Shape {
  static constexpr int E = (M >= 512) ? 16 : (M >= 256 ? 8 : 4);   // points per thread
  static constexpr int TPL = M / E;                                  // threads per line
  // radix of stage s (all divide E); stages multiply to M
  static constexpr int NST = (M == 512) ? 3 : (M == 256 ? 3 : (M == 128 ? 4 : 3));
  __host__ __device__ static constexpr int radix(int s) {
    return (M == 512) ? 8 : (M == 256 ? (s < 2 ? 8 : 4) : (M == 128 ? (s < 3 ? 4 : 2) : 4));
  }
};

// Skewed index of the complex exchange buffer: one pad slot per 8 entries turns
// the stride-8 (64-byte) writes of a radix-8 stage into conflict-free ones.
__device__ __forceinline__ int cpad(int i) { return i + (i >> 3); }

template <class T, bool INV>
__device__ __forceinline__ void dft2(cplx<T>& a, cplx<T>& b) {
  cplx<T> t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <class T, bool INV>
__device__ __forceinline__ void dft4(cplx<T>* v) {
  cplx<T> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  cplx<T> t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
  t3 = INV ? mul_i(t3) : mul_mi(t3);
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

template <class T, bool INV>
__device__ __forceinline__ void dft8(cplx<T>* v) {
  // radix-2 over (r, r+4), twiddle by W8^r, then two radix-4 on evens/odds
  const T h = (T)0.70710678118654752440;
  cplx<T> a[4], b[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = cadd(v[r], v[r + 4]);
    b[r] = csub(v[r], v[r + 4]);
  }
  // b[r] *= W8^{±r}
  b[1] = INV ? cplx<T>{(b[1].x - b[1].y) * h, (b[1].x + b[1].y) * h}
             : cplx<T>{(b[1].x + b[1].y) * h, (b[1].y - b[1].x) * h};
  b[2] = INV ? mul_i(b[2]) : mul_mi(b[2]);
  b[3] = INV ? cplx<T>{-(b[3].x + b[3].y) * h, (b[3].x - b[3].y) * h}
             : cplx<T>{(b[3].y - b[3].x) * h, -(b[3].x + b[3].y) * h};
  dft4<T, INV>(a);
  dft4<T, INV>(b);
  // outputs: X[2k] = A[k], X[2k+1] = B[k]
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = a[k];
    v[2 * k + 1] = b[k];
  }
}

template <class T, int R, bool INV>
__device__ __forceinline__ void dftR(cplx<T>* v) {
  if constexpr (R == 2) dft2<T, INV>(v[0], v[1]);
  if constexpr (R == 4) dft4<T, INV>(v);
  if constexpr (R == 8) dft8<T, INV>(v);
}

// Stages STAGE… of the M-point FFT of one line. On entry v holds this stage's
// inputs in (butterfly q, element r) order: v[q*R + r] = x[b_q + r*M/R] with
// b_q = t + q*TPL. On return v holds the last stage's outputs, v[q*R + r] at
// position b_q + r*(M/R_last). buf is the line's M-complex shared buffer.
template <class T, int M, bool INV, int STAGE, int NS>
__device__ __forceinline__ void fft_stages(cplx<T> (&v)[Shape<M>::E], cplx<T>* buf,
                                           const cplx<T>* stw, int t) {
  using S = Shape<M>;
  constexpr int E = S::E, TPL = S::TPL;
  constexpr int R = S::radix(STAGE);
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
    const int b = t + q * TPL;
    if constexpr (STAGE > 0) {
      const int k = b & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = stw[(r * k * (M / (NS * R))) & (M - 1)];
        if (INV) w.y = -w.y;
        v[q * R + r] = cmul(v[q * R + r], w);
      }
    }
    dftR<T, R, INV>(&v[q * R]);
  }
  if constexpr (STAGE + 1 < S::NST) {
    constexpr int R2 = S::radix(STAGE + 1);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < E / R; ++q) {
      const int b = t + q * TPL;
      const int o = (b / NS) * NS * R + (b & (NS - 1));
#pragma unroll
      for (int r = 0; r < R; ++r) buf[cpad(o + r * NS)] = v[q * R + r];
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < E / R2; ++q) {
      const int b = t + q * TPL;
#pragma unroll
      for (int r = 0; r < R2; ++r) v[q * R2 + r] = buf[cpad(b + r * (M / R2))];
    }
    fft_stages<T, M, INV, STAGE + 1, NS * R>(v, buf, stw, t);
  }
}

}  // namespace fast

// Bytes of the twiddle tables for a given BC (16-byte aligned): ω_M^t (M), the
// real-FFT split factors (M + 1) and, except for P, the BC factors (≤ 2M).
template <class T, int M>
__host__ __device__ constexpr size_t fast_table_bytes(int bc) {
  return ((size_t)(2 * M + 1 + (bc == 0 ? 0 : 2 * M + 1)) * sizeof(cplx<T>) + 15) / 16 * 16;
}

template <class T>
struct FastArgs {
  const void* in;
  void* out;
  int axis, nx, ny, nz, bc;
  int nlines;           // x: ny*nz rows; y: nx*nz columns
  const cplx<T>* tw;    // 8n-entry table, e^{−2πi t/(8n)}
  const T* plane_scale;
  int accumulate;
  const int* skip;
  unsigned long long* amax;  // FP64 output: atomicMax of |transform output| bit patterns, or null
  int lpc;              // lines per CTA
  float* out2;          // FP64 output (x lines): also store the FP32 transform output here, or null
  const float* base32;  // FP64 output (x lines): out = widen(base32) + v instead of (out +) v, or null
};

template <class T, class TI, class TO, int M, bool FWD>
cudaError_t launch_xform_fast(FastArgs<T> a, cudaStream_t st);

// x-axis lines read and written by their own warp (xform_row.cu): nx = 2M.
template <class T, class TI, class TO, int M, bool FWD>
cudaError_t launch_xform_row(FastArgs<T> a, cudaStream_t st);

// y-axis lines with the columns on lanes (xform_col.cu): ny = 2M, nx a multiple
// of 16, TI = TO = T, no accumulation and no FP64 max tracking.
template <class T, int M, bool FWD>
cudaError_t launch_xform_col(FastArgs<T> a, cudaStream_t st);

// Lines of n = 2M contiguous reals with M ∈ {1024, 2048, 4096}, one CTA per line
// (xform_long.cu): a.nlines lines, line ln in plane ln / a.ny; x-row output modes.
template <class T, class TI, class TO, int M, bool FWD>
cudaError_t launch_xform_long(FastArgs<T> a, cudaStream_t st);

// dst[z][c][r] = src[z][r][c] for every plane z < nz (rows × cols per plane).
template <class T>
cudaError_t launch_plane_transpose(const T* src, T* dst, int rows, int cols, int nz, const int* skip,
                                   cudaStream_t st);

}  // namespace ps
