// projection.cu — the velocity projection around the solve (Eqs. 2b–2c) and its adjoint.
//
// Staggered (MAC) grid of §2: the velocity component along an axis lives on the
// cell faces normal to that axis. Storage: each component has the cell array's
// shape [n_z][n_y][n_x]; entry i along its own axis is the face on the low side
// of cell i. On a periodic axis face 0 is the wrap face; on a Neumann-pressure
// axis (prescribed velocity, end of §2) face 0 is the wall (its value is
// carried through unchanged) and the high wall is implicit.
//
//   D u   (cell):  Σ_axes (u[i+1] − u[i]) / Δ_i, wall faces excluded
//   G φ   (face):  (φ[i] − φ[i−1]) / Δc_{i−1} on interior/periodic faces, 0 on walls
// with Δ_i the cell width and Δc the centre distance (Δz^f, Δz^c on the stretched
// z; the periodic wrap distance is (Δ_0 + Δ_{n−1})/2). D·G is the operator of
// Eq. 4. The projection (γΔt cancels): u = u* − G A⁻¹ D u*. Its vector–Jacobian
// product: ḡ* = ḡ − Dᵀ A⁻ᵀ Gᵀ ḡ, with
//   (Gᵀ g)[c] = Σ_axes g[i]/Δc_{i−1} − g[i+1]/Δc_i      (interior/periodic faces)
//   (Dᵀ s)[face i] = s[i−1]/Δ_{i−1} − s[i]/Δ_i         (interior/periodic faces; 0 on walls)
// Only P and NN axes are supported (the pressure BCs of periodic and wall axes).
#include "internal.h"

namespace ps {

// ProjArgs (internal.h): per[] = axis periodic; idx, idy = 1/Δx, 1/Δy; idzf[k] = 1/Δz^f_k;
// idzc[k] = 1/(centre distance between cells k−1 and k), idzc[0] = the periodic wrap.

// x, y, z index helpers
#define PS_IDX(k, j, i) (((size_t)(k) * a.ny + (j)) * a.nx + (i))

template <class T>
__global__ void div_kernel(ProjArgs<T> a, const T* __restrict__ u, T* __restrict__ f) {
  const size_t N = (size_t)a.nx * a.ny * a.nz;
  const T* __restrict__ ux = u;
  const T* __restrict__ uy = u + N;
  const T* __restrict__ uz = u + 2 * N;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(g % a.nx);
    const size_t t = g / a.nx;
    const int j = (int)(t % a.ny), k = (int)(t / a.ny);
    // x: faces i (low) and i+1 (high)
    T hx = (i + 1 < a.nx) ? ux[g + 1] : (a.per[0] ? ux[g + 1 - a.nx] : (T)0);
    T lx = (i > 0 || a.per[0]) ? ux[g] : (T)0;
    T hy = (j + 1 < a.ny) ? uy[g + a.nx] : (a.per[1] ? uy[PS_IDX(k, 0, i)] : (T)0);
    T ly = (j > 0 || a.per[1]) ? uy[g] : (T)0;
    T hz = (k + 1 < a.nz) ? uz[g + (size_t)a.nx * a.ny] : (a.per[2] ? uz[PS_IDX(0, j, i)] : (T)0);
    T lz = (k > 0 || a.per[2]) ? uz[g] : (T)0;
    f[g] = (hx - lx) * a.idx + (hy - ly) * a.idy + (hz - lz) * a.idzf[k];
  }
}

// u = u* − G φ (all three components)
template <class T>
__global__ void grad_correct_kernel(ProjArgs<T> a, const T* __restrict__ us, const T* __restrict__ phi,
                                    T* __restrict__ u) {
  const size_t N = (size_t)a.nx * a.ny * a.nz;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(g % a.nx);
    const size_t t = g / a.nx;
    const int j = (int)(t % a.ny), k = (int)(t / a.ny);
    const T pc = phi[g];
    T gx = 0, gy = 0, gz = 0;
    if (i > 0) gx = (pc - phi[g - 1]) * a.idx;
    else if (a.per[0]) gx = (pc - phi[g + a.nx - 1]) * a.idx;
    if (j > 0) gy = (pc - phi[g - a.nx]) * a.idy;
    else if (a.per[1]) gy = (pc - phi[PS_IDX(k, a.ny - 1, i)]) * a.idy;
    if (k > 0) gz = (pc - phi[g - (size_t)a.nx * a.ny]) * a.idzc[k];
    else if (a.per[2]) gz = (pc - phi[PS_IDX(a.nz - 1, j, i)]) * a.idzc[0];
    u[g] = us[g] - gx;
    u[g + N] = us[g + N] - gy;
    u[g + 2 * N] = us[g + 2 * N] - gz;
  }
}

// h = Gᵀ g (cells)
template <class T>
__global__ void grad_adjoint_kernel(ProjArgs<T> a, const T* __restrict__ gu, T* __restrict__ h) {
  const size_t N = (size_t)a.nx * a.ny * a.nz;
  const T* __restrict__ gx = gu;
  const T* __restrict__ gy = gu + N;
  const T* __restrict__ gz = gu + 2 * N;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(g % a.nx);
    const size_t t = g / a.nx;
    const int j = (int)(t % a.ny), k = (int)(t / a.ny);
    T v = 0;
    // own low face (i) contributes +g/Δc, high face (i+1) contributes −g/Δc
    if (i > 0 || a.per[0]) v += gx[g] * a.idx;
    if (i + 1 < a.nx) v -= gx[g + 1] * a.idx;
    else if (a.per[0]) v -= gx[g + 1 - a.nx] * a.idx;
    if (j > 0 || a.per[1]) v += gy[g] * a.idy;
    if (j + 1 < a.ny) v -= gy[g + a.nx] * a.idy;
    else if (a.per[1]) v -= gy[PS_IDX(k, 0, i)] * a.idy;
    if (k > 0 || a.per[2]) v += gz[g] * a.idzc[k];
    if (k + 1 < a.nz) v -= gz[g + (size_t)a.nx * a.ny] * a.idzc[k + 1];
    else if (a.per[2]) v -= gz[PS_IDX(0, j, i)] * a.idzc[0];
    h[g] = v;
  }
}

// ḡ* = ḡ − Dᵀ s (faces)
template <class T>
__global__ void div_adjoint_correct_kernel(ProjArgs<T> a, const T* __restrict__ gu, const T* __restrict__ s,
                                           T* __restrict__ out) {
  const size_t N = (size_t)a.nx * a.ny * a.nz;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(g % a.nx);
    const size_t t = g / a.nx;
    const int j = (int)(t % a.ny), k = (int)(t / a.ny);
    const T sc = s[g];
    // face i lies between cell i−1 (contributes s/Δ) and cell i (−s/Δ)
    T dx = 0, dy = 0, dz = 0;
    if (i > 0) dx = (s[g - 1] - sc) * a.idx;
    else if (a.per[0]) dx = (s[g + a.nx - 1] - sc) * a.idx;
    if (j > 0) dy = (s[g - a.nx] - sc) * a.idy;
    else if (a.per[1]) dy = (s[PS_IDX(k, a.ny - 1, i)] - sc) * a.idy;
    if (k > 0) dz = s[g - (size_t)a.nx * a.ny] * a.idzf[k - 1] - sc * a.idzf[k];
    else if (a.per[2]) dz = s[PS_IDX(a.nz - 1, j, i)] * a.idzf[a.nz - 1] - sc * a.idzf[0];
    out[g] = gu[g] - dx;
    out[g + N] = gu[g + N] - dy;
    out[g + 2 * N] = gu[g + 2 * N] - dz;
  }
}
#undef PS_IDX

template <class T>
cudaError_t launch_projection(int op, const ProjArgs<T>& a, const void* x0, const void* x1, void* y,
                              cudaStream_t st) {
  const size_t N = (size_t)a.nx * a.ny * a.nz;
  const int threads = 256;
  const int blocks = (int)((N + threads - 1) / threads < 152 * 16 ? (N + threads - 1) / threads : 152 * 16);
  const T* a0 = static_cast<const T*>(x0);
  const T* a1 = static_cast<const T*>(x1);
  T* o = static_cast<T*>(y);
  switch (op) {
    case 0: div_kernel<T><<<blocks, threads, 0, st>>>(a, a0, o); break;
    case 1: grad_correct_kernel<T><<<blocks, threads, 0, st>>>(a, a0, a1, o); break;
    case 2: grad_adjoint_kernel<T><<<blocks, threads, 0, st>>>(a, a0, o); break;
    default: div_adjoint_correct_kernel<T><<<blocks, threads, 0, st>>>(a, a0, a1, o); break;
  }
  return cudaGetLastError();
}

template cudaError_t launch_projection<float>(int, const ProjArgs<float>&, const void*, const void*, void*, cudaStream_t);
template cudaError_t launch_projection<double>(int, const ProjArgs<double>&, const void*, const void*, void*, cudaStream_t);

}  // namespace ps
