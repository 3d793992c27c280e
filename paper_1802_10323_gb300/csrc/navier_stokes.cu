// navier_stokes.cu — the RK3 fractional step around the solve (§2, Eqs. 2a–2d).
//
// Substep k (α = 8/15, 5/12, 3/4; β = 0, −17/60, −5/12; γ = α + β):
//   u* = u^k + Δt (α_k AD^k + β_k AD^{k−1} − γ_k G p^{k−1/2})     (2a; this file, one kernel)
//   A Φ' = D u*,  u^{k+1} = u* − G Φ'                                (2b–2c; the projection kernels
//                                                                      and the solve, Φ' = γΔt·Φ)
//   p^{k+1/2} = p^{k−1/2} + Φ'/(γΔt)                                 (2d; this file)
// with AD = −(u·∇)u + ν∇²u. Staggered layout of the projection: each velocity
// component has the cell array's shape [n_z][n_y][n_x], entry i along its own axis
// being the face on the low side of cell i; the components are stacked [u | v | w].
//
// Discretisation (second-order central, §2 gives no stencil): advection in
// divergence form ∂(u_i u_j)/∂x_j with arithmetic averages for every interpolation —
// the normal products at cell centres, the cross products on cell edges — and the
// flux differences taken over each component's control volume (Δ across a cell, the
// centre distance across a z face); the viscous term is the finite-volume second
// difference of Eq. 4 on the same control volumes. x and y are periodic; z is
// periodic, or bounded by no-slip walls: w = 0 on the wall faces (face 0 stored, the
// top face implicit) and the tangential components see a ghost cell mirrored across
// the wall with the opposite sign. On a wall face AD is not formed and w stays 0.
//
// One thread per cell forms the three face values of that cell (x face i, y face j,
// z face k); x is the fastest index, so every neighbour load of a warp is a
// contiguous row segment, and the 3×3×3 neighbourhoods overlap in L1/L2.
#include "internal.h"

namespace ps {

namespace {

template <class T>
__global__ void __launch_bounds__(256) ns_predict_kernel(NsArgs<T> a, const T* __restrict__ u3,
                                                         const T* __restrict__ p, const T* ad_prev,
                                                         T* __restrict__ ustar, T* ad_out) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t sy = (size_t)nx, sz = (size_t)nx * ny, N = sz * nz;
  const T* __restrict__ U = u3;
  const T* __restrict__ V = u3 + N;
  const T* __restrict__ W = u3 + 2 * N;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(g % nx);
    const size_t t = g / nx;
    const int j = (int)(t % ny), k = (int)(t / ny);
    // periodic x and y neighbours (offsets from g)
    const long dxm = (i > 0) ? -1 : (long)(nx - 1), dxp = (i + 1 < nx) ? 1 : -(long)(nx - 1);
    const long dym = (j > 0) ? -(long)sy : (long)((ny - 1) * sy), dyp = (j + 1 < ny) ? (long)sy : -(long)((ny - 1) * sy);
    // z neighbours: the plane below / above, whether they exist (walls) and the wrap
    const bool per = a.per_z != 0;
    const bool has_dn = k > 0 || per, has_up = k + 1 < nz || per;
    const long dzm = (k > 0) ? -(long)sz : (long)((nz - 1) * sz);
    const long dzp = (k + 1 < nz) ? (long)sz : -(long)((nz - 1) * sz);
    const T idzf = a.idzf[k];
    // 1/(centre distance) below and above cell k; walls: the ghost sits one Δz^f away
    const T ihdn = (k > 0) ? a.idzc[k] : (per ? a.idzc[0] : a.idzf[0]);
    const T ihup = (k + 1 < nz) ? a.idzc[k + 1] : (per ? a.idzc[0] : a.idzf[nz - 1]);

    // loads (W on the wall face 0 is taken as 0; cell-centred ghosts are −value)
    auto Wv = [&](long off, int kk) -> T { return (!per && kk == 0) ? (T)0 : W[g + off]; };
    const T uc = U[g], vc = V[g], wc = Wv(0, k);

    // Every flux below is a product of two sums of neighbours (an average each): the two
    // factors ½ go into one factor ¼ on the flux difference (q* = ¼/Δ), and the normal
    // term d(ū²) = ((a + b)² − (c + a)²)/4 is formed as (b − c)(b + 2a + c)/4.
    // ---------------- x momentum at x face i ----------------
    T adu;
    {
      const T uxp = U[g + dxp], uxm = U[g + dxm];
      const T uyp = U[g + dyp], uym = U[g + dym];
      const T uzp = has_up ? U[g + dzp] : -uc, uzm = has_dn ? U[g + dzm] : -uc;
      const T duu = (uxp - uxm) * (uxp + 2 * uc + uxm) * a.qx;
      // uv on the y faces j and j+1 of this x face
      const T uv0 = (uc + uym) * (vc + V[g + dxm]);
      const T uv1 = (uyp + uc) * (V[g + dyp] + V[g + dyp + dxm]);
      const T duv = (uv1 - uv0) * a.qy;
      // uw on the z faces k and k+1 of this x face (k = 0 on a wall: w = 0)
      const T uw0 = has_dn ? (uc + uzm) * (wc + Wv(dxm, k)) : (T)0;
      const T uw1 = has_up ? (uzp + uc) * (Wv(dzp, k + 1 < nz ? k + 1 : 0) + Wv(dzp + dxm, k + 1 < nz ? k + 1 : 0)) : (T)0;
      const T duw = (uw1 - uw0) * ((T)0.25 * idzf);
      const T lap = (uxp - 2 * uc + uxm) * a.idx2 + (uyp - 2 * uc + uym) * a.idy2 +
                    ((uzp - uc) * ihup - (uc - uzm) * ihdn) * idzf;
      adu = a.nu * lap - (duu + duv + duw);
    }
    // ---------------- y momentum at y face j ----------------
    T adv;
    {
      const T vxp = V[g + dxp], vxm = V[g + dxm];
      const T vyp = V[g + dyp], vym = V[g + dym];
      const T vzp = has_up ? V[g + dzp] : -vc, vzm = has_dn ? V[g + dzm] : -vc;
      const T dvv = (vyp - vym) * (vyp + 2 * vc + vym) * a.qy;
      // uv on the x faces i and i+1 of this y face
      const T uv0 = (uc + U[g + dym]) * (vc + vxm);
      const T uv1 = (U[g + dxp] + U[g + dxp + dym]) * (vxp + vc);
      const T duv = (uv1 - uv0) * a.qx;
      const T vw0 = has_dn ? (vc + vzm) * (wc + Wv(dym, k)) : (T)0;
      const T vw1 = has_up ? (vzp + vc) * (Wv(dzp, k + 1 < nz ? k + 1 : 0) + Wv(dzp + dym, k + 1 < nz ? k + 1 : 0)) : (T)0;
      const T dvw = (vw1 - vw0) * ((T)0.25 * idzf);
      const T lap = (vxp - 2 * vc + vxm) * a.idx2 + (vyp - 2 * vc + vym) * a.idy2 +
                    ((vzp - vc) * ihup - (vc - vzm) * ihdn) * idzf;
      adv = a.nu * lap - (duv + dvv + dvw);
    }
    // ---------------- z momentum at z face k ----------------
    T adw = (T)0;
    if (has_dn) {  // not on a wall face
      const int kup = k + 1 < nz ? k + 1 : 0;
      const T wzp = has_up ? Wv(dzp, kup) : (T)0;
      const int kdn = k > 0 ? k - 1 : nz - 1;
      const T wzm = Wv(dzm, kdn);
      const T wxp = Wv(dxp, k), wxm = Wv(dxm, k), wyp = Wv(dyp, k), wym = Wv(dym, k);
      const T dww = (wzp - wzm) * (wzp + 2 * wc + wzm) * ((T)0.25 * ihdn);
      // uw on the x faces i and i+1 of this z face (u averaged over cells k−1 and k)
      const T uw0 = (uc + U[g + dzm]) * (wc + wxm);
      const T uw1 = (U[g + dxp] + U[g + dxp + dzm]) * (wxp + wc);
      const T duw = (uw1 - uw0) * a.qx;
      const T vw0 = (vc + V[g + dzm]) * (wc + wym);
      const T vw1 = (V[g + dyp] + V[g + dyp + dzm]) * (wyp + wc);
      const T dvw = (vw1 - vw0) * a.qy;
      const T idzf_m = a.idzf[kdn];
      const T lap = (wxp - 2 * wc + wxm) * a.idx2 + (wyp - 2 * wc + wym) * a.idy2 +
                    ((wzp - wc) * idzf - (wc - wzm) * idzf_m) * ihdn;
      adw = a.nu * lap - (duw + dvw + dww);
    }

    // ---------------- predictor (2a) ----------------
    const T pc = p[g];
    const T gpx = (pc - p[g + dxm]) * a.idx;
    const T gpy = (pc - p[g + dym]) * a.idy;
    const T gpz = has_dn ? (pc - p[g + dzm]) * ihdn : (T)0;
    const T bu = a.beta != (T)0 ? ad_prev[g] : (T)0;
    const T bv = a.beta != (T)0 ? ad_prev[g + N] : (T)0;
    const T bw = a.beta != (T)0 ? ad_prev[g + 2 * N] : (T)0;
    ustar[g] = uc + a.dt * (a.alpha * adu + a.beta * bu - a.gamma * gpx);
    ustar[g + N] = vc + a.dt * (a.alpha * adv + a.beta * bv - a.gamma * gpy);
    ustar[g + 2 * N] = has_dn ? wc + a.dt * (a.alpha * adw + a.beta * bw - a.gamma * gpz) : W[g];
    ad_out[g] = adu;
    ad_out[g + N] = adv;
    ad_out[g + 2 * N] = adw;
  }
}

// p += Φ'/(γΔt), and Φ' → Φ in place (2d)
template <class T>
__global__ void __launch_bounds__(256) ns_pressure_kernel(size_t N, T scale, T* __restrict__ p,
                                                          T* __restrict__ phi) {
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
    const T f = phi[g] * scale;
    phi[g] = f;
    p[g] += f;
  }
}

int grid_for(size_t N) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (N + 255) / 256, cap = (size_t)sms * 8;
  return (int)(want < cap ? want : cap);
}

}  // namespace

template <class T>
cudaError_t launch_ns_predict(const NsArgs<T>& a, const void* u3, const void* p, const void* ad_prev,
                              void* ustar, void* ad_out, cudaStream_t st) {
  const size_t N = (size_t)a.nx * a.ny * a.nz;
  ns_predict_kernel<T><<<grid_for(N), 256, 0, st>>>(a, static_cast<const T*>(u3), static_cast<const T*>(p),
                                                    static_cast<const T*>(ad_prev), static_cast<T*>(ustar),
                                                    static_cast<T*>(ad_out));
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_ns_pressure(size_t N, double scale, void* p, void* phi, cudaStream_t st) {
  ns_pressure_kernel<T><<<grid_for(N), 256, 0, st>>>(N, (T)scale, static_cast<T*>(p), static_cast<T*>(phi));
  return cudaGetLastError();
}

template cudaError_t launch_ns_predict<float>(const NsArgs<float>&, const void*, const void*, const void*, void*,
                                              void*, cudaStream_t);
template cudaError_t launch_ns_predict<double>(const NsArgs<double>&, const void*, const void*, const void*, void*,
                                               void*, cudaStream_t);
template cudaError_t launch_ns_pressure<float>(size_t, double, void*, void*, cudaStream_t);
template cudaError_t launch_ns_pressure<double>(size_t, double, void*, void*, cudaStream_t);

}  // namespace ps
