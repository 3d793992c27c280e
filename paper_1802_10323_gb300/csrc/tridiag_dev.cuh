// tridiag_dev.cuh — device code of the z tridiagonal solves of Eq. 5 (see tridiag.cu).
#pragma once
#include "internal.h"

namespace ps {

template <class T>
__device__ __forceinline__ T rcp_(T x) { return (T)1 / x; }

// One column of Eq. 5 (Thomas; Sherman–Morrison when z is periodic), in place,
// with the eliminated super-diagonal in the scratch array.
template <class T>
__device__ void zsolve_column(const ZArgs<T>& a, int col) {
  const int ncol = a.nx * a.ny;
  if (col >= ncol) return;
  if (a.singular && col == 0) return;
  const int i = col % a.nx, j = col / a.nx;
  const T lam = a.lamx[i] + a.lamy[j];
  const size_t st = (size_t)ncol;
  const int nz = a.nz;
  T* __restrict__ d = a.data + col;
  T* __restrict__ sc = a.scr_c + col;
  T* __restrict__ su = a.periodic ? a.scr_u + col : nullptr;
  const T* __restrict__ za = a.za;
  const T* __restrict__ zb = a.zb;
  const T* __restrict__ zc = a.zc;

  T gamma = (T)0, corner = (T)0;
  if (a.periodic) {
    gamma = -(zb[0] + lam);
    corner = za[0] * zc[nz - 1] / gamma;
  }
  // forward elimination
  T cp = (T)0, dp = (T)0, up = (T)0;
  for (int k = 0; k < nz; ++k) {
    T bk = zb[k] + lam;
    const T ak = (k > 0) ? za[k] : (T)0;
    const T ck = (k < nz - 1) ? zc[k] : (T)0;
    if (a.periodic) {
      if (k == 0) bk -= gamma;
      if (k == nz - 1) bk -= corner;
    }
    const T mk = rcp_(bk - ak * cp);
    cp = ck * mk;
    const T dk = d[k * st];
    dp = (dk - ak * dp) * mk;
    d[k * st] = dp;
    sc[k * st] = cp;
    if (a.periodic) {
      const T uk = (k == 0) ? gamma : ((k == nz - 1) ? zc[nz - 1] : (T)0);
      up = (uk - ak * up) * mk;
      su[k * st] = up;
    }
  }
  // back substitution
  T x = (T)0, zz = (T)0;
  for (int k = nz - 1; k >= 0; --k) {
    const T cpk = (k < nz - 1) ? sc[k * st] : (T)0;
    x = d[k * st] - cpk * x;
    d[k * st] = x;
    if (a.periodic) {
      zz = su[k * st] - cpk * zz;
      su[k * st] = zz;
    }
  }
  if (a.periodic) {
    const T y0 = d[0], yn = d[(nz - 1) * st];
    const T z0 = su[0], zn = su[(nz - 1) * st];
    const T r = za[0] / gamma;
    const T beta = (y0 + r * yn) / ((T)1 + z0 + r * zn);
    for (int k = 0; k < nz; ++k) d[k * st] -= beta * su[k * st];
  }
}

// Column (0,0) of a singular problem; one CTA (≤ 256 threads), the column staged
// in shared memory (2·nz values of T in smem_raw).
template <class T>
__device__ void zsingular_block(const ZArgs<T>& a, unsigned char* smem_raw) {
  const int nz = a.nz;
  T* s = reinterpret_cast<T*>(smem_raw);  // nz values
  T* cps = s + nz;                         // nz values
  __shared__ T red[2][256];
  const size_t st = (size_t)a.nx * a.ny;
  T num = 0, den = 0;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    T v = a.data[k * st];
    s[k] = v;
    num += a.dzf[k] * v;
    den += a.dzf[k];
  }
  red[0][threadIdx.x] = num;
  red[1][threadIdx.x] = den;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  const T mean = red[0][0] / red[1][0];
  const T wsum = red[1][0];
  __syncthreads();
  if (threadIdx.x == 0) {
    // rows 1 … nz−1 with Φ̂_0 = 0 (no wrap term survives)
    T cp = 0, dp = 0;
    for (int k = 1; k < nz; ++k) {
      const T ak = (k > 1) ? a.za[k] : (T)0;
      const T ck = (k < nz - 1) ? a.zc[k] : (T)0;
      const T mk = (T)1 / (a.zb[k] - ak * cp);
      cp = ck * mk;
      dp = ((s[k] - mean) - ak * dp) * mk;
      s[k] = dp;
      cps[k] = cp;
    }
    s[0] = 0;
    T x = 0;
    for (int k = nz - 1; k >= 1; --k) {
      x = s[k] - ((k < nz - 1) ? cps[k] : (T)0) * x;
      s[k] = x;
    }
  }
  __syncthreads();
  num = 0;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) num += a.dzf[k] * s[k];
  red[0][threadIdx.x] = num;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[0][threadIdx.x] += red[0][threadIdx.x + w];
    __syncthreads();
  }
  const T mx = red[0][0] / wsum;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) a.data[k * st] = s[k] - mx;
}

}  // namespace ps
