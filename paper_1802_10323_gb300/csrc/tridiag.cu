// tridiag.cu — the N_x·N_y tridiagonal systems of Eq. 5 along z.
//
// Column (q_x, q_y) solves a_k Φ̂_{k−1} + (b_k + λ_qx/Δx² + λ_qy/Δy²) Φ̂_k + c_k Φ̂_{k+1} = f̂_k.
// One thread per column; a warp covers 32 consecutive q_x, so every access to
// plane k is a coalesced row segment. Gauss elimination without pivoting
// (each column is weakly diagonally dominant with a strictly dominant row).
// The eliminated super-diagonal c'_k goes to a scratch array; d'_k overwrites
// the data in place and is replaced by Φ̂_k in the back substitution.
//
// Periodic z (§3: the cyclic system "reduced into two tridiagonal problems"):
// Sherman–Morrison with γ = −b_0, u = (γ, 0, …, 0, c_{n−1}), v = (1, 0, …, 0, a_0/γ):
// solve B y = d and B z = u with one elimination, then Φ̂ = y − (v·y)/(1 + v·z) z.
//
// Singular column (every axis P or NN): (q_x, q_y) = (0, 0) has λ = 0 and a
// singular z matrix. Its right-hand side loses its Δz^f-weighted mean, Φ̂_0 = 0
// is pinned (row 0 dropped), and the solution's weighted mean is removed. A
// separate one-CTA kernel does this column from shared memory.
#include "tridiag_dev.cuh"

namespace ps {

// FP32, non-periodic columns: the forward sweep keeps the eliminated
// (c'_k, d'_k) only at the end of every chunk of ZK planes (1/8 of the data
// volume, in the scratch array); the backward sweep walks the chunks from the top, re-reads each
// chunk's right-hand side, recomputes its (c', d') from the checkpoint in
// registers (the same instructions on the same inputs, so bit-identical to the
// forward sweep) and back-substitutes. HBM traffic: read f̂ twice (the second
// read of a chunk usually hits L2), write Φ̂ once; loads of the next chunk are
// issued before the current chunk is processed.
template <class T>
cudaError_t launch_zsolve(ZArgs<T> a, cudaStream_t st);

constexpr int ZK = 16;
constexpr int ZB = 128;  // columns (threads) per CTA

__global__ void __launch_bounds__(ZB) zsolve_ckpt_kernel(ZArgs<float> a) {
  if (a.skip && *a.skip) return;
  const int ncol = a.nx * a.ny;
  float2* __restrict__ ck = reinterpret_cast<float2*>(a.scr_c);  // [nchunk][ncol]
  const int col = blockIdx.x * ZB + threadIdx.x;
  const bool act = col < ncol && !(a.singular && col == 0);
  const int colc = col < ncol ? col : ncol - 1;
  const int i = colc % a.nx, j = colc / a.nx;
  const float lam = a.lamx[i] + a.lamy[j];
  const size_t st = (size_t)ncol;
  const int nz = a.nz;
  const int nch = (nz + ZK - 1) / ZK;
  float* __restrict__ d = a.data + colc;
  const float* __restrict__ za = a.za;
  const float* __restrict__ zb = a.zb;
  const float* __restrict__ zc = a.zc;

  float cur[ZK], nxt[ZK];
#pragma unroll
  for (int u = 0; u < ZK; ++u) cur[u] = (u < nz) ? d[(size_t)u * st] : 0.f;
  float cp = 0.f, dp = 0.f;
  for (int c = 0; c < nch; ++c) {
    const int k0 = c * ZK;
    if (c + 1 < nch) {
#pragma unroll
      for (int u = 0; u < ZK; ++u) {
        const int k = k0 + ZK + u;
        nxt[u] = (k < nz) ? d[(size_t)k * st] : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < ZK; ++u) {
      const int k = k0 + u;
      if (k < nz) {
        const float ak = (k > 0) ? za[k] : 0.f;
        const float ckk = (k < nz - 1) ? zc[k] : 0.f;
        const float mk = __fdividef(1.f, zb[k] + lam - ak * cp);
        cp = ckk * mk;
        dp = (cur[u] - ak * dp) * mk;
      }
    }
    ck[(size_t)c * ncol + colc] = make_float2(cp, dp);
#pragma unroll
    for (int u = 0; u < ZK; ++u) cur[u] = nxt[u];
  }
  // backward: chunks from the top; prefetch the chunk below
  {
    const int k0 = (nch - 1) * ZK;
#pragma unroll
    for (int u = 0; u < ZK; ++u) {
      const int k = k0 + u;
      cur[u] = (k < nz) ? d[(size_t)k * st] : 0.f;
    }
  }
  float x = 0.f;
  for (int c = nch - 1; c >= 0; --c) {
    const int k0 = c * ZK;
    if (c > 0) {
#pragma unroll
      for (int u = 0; u < ZK; ++u) nxt[u] = d[(size_t)(k0 - ZK + u) * st];
    }
    float2 prev = (c > 0) ? ck[(size_t)(c - 1) * ncol + colc] : make_float2(0.f, 0.f);
    float cpa[ZK], dpa[ZK];
    cp = prev.x;
    dp = prev.y;
#pragma unroll
    for (int u = 0; u < ZK; ++u) {
      const int k = k0 + u;
      if (k < nz) {
        const float ak = (k > 0) ? za[k] : 0.f;
        const float ckk = (k < nz - 1) ? zc[k] : 0.f;
        const float mk = __fdividef(1.f, zb[k] + lam - ak * cp);
        cp = ckk * mk;
        dp = (cur[u] - ak * dp) * mk;
      }
      cpa[u] = cp;
      dpa[u] = dp;
    }
#pragma unroll
    for (int u = ZK - 1; u >= 0; --u) {
      const int k = k0 + u;
      if (k < nz) {
        x = dpa[u] - ((k < nz - 1) ? cpa[u] : 0.f) * x;
        if (act) d[(size_t)k * st] = x;
      }
    }
#pragma unroll
    for (int u = 0; u < ZK; ++u) cur[u] = nxt[u];
  }
}

cudaError_t launch_zsolve_ckpt(ZArgs<float> a, cudaStream_t st) {
  const int ncol = a.nx * a.ny;
  zsolve_ckpt_kernel<<<(ncol + ZB - 1) / ZB, ZB, 0, st>>>(a);
  return cudaGetLastError();
}

template <class T>
__global__ void __launch_bounds__(128) zsolve_kernel(ZArgs<T> a) {
  if (a.skip && *a.skip) return;
  zsolve_column<T>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

template <class T>
__global__ void __launch_bounds__(256) zsingular_kernel(ZArgs<T> a) {
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zsingular_block<T>(a, smem_raw);
}

template <class T>
cudaError_t launch_zsolve(ZArgs<T> a, cudaStream_t st) {
  const int ncol = a.nx * a.ny;
  zsolve_kernel<T><<<(ncol + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_zsingular(ZArgs<T> a, cudaStream_t st) {
  const size_t smem = 2 * (size_t)a.nz * sizeof(T);
  auto k = zsingular_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<1, 256, smem, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_zsolve<double>(ZArgs<double>, cudaStream_t);
template cudaError_t launch_zsolve<float>(ZArgs<float>, cudaStream_t);
template cudaError_t launch_zsingular<double>(ZArgs<double>, cudaStream_t);
template cudaError_t launch_zsingular<float>(ZArgs<float>, cudaStream_t);

}  // namespace ps
