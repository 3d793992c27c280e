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
// difference of Eq. 4 on the same control volumes. Each axis is periodic, or bounded
// by no-slip walls (the duct and cavity cases of Table 3 have walls on x and y): the
// normal component is 0 on the wall faces (face 0 stored, the top face implicit) and
// the tangential components see a ghost cell mirrored across the wall with the
// opposite sign, one cell width away. On a wall face AD is not formed and the normal
// component stays 0. x and y are uniform, z may be stretched.
//
// One thread per cell forms the three face values of that cell (x face i, y face j,
// z face k); x is the fastest index, so every neighbour load of a warp is a
// contiguous row segment, and the 3×3×3 neighbourhoods overlap in L1/L2. Every
// neighbour goes through one loader that applies the axis rules (wrap, mirrored
// ghost, or the zero wall face), so the flux formulas below are those of the
// periodic box; which axes are periodic is a template argument, so the periodic box
// compiles to plain wrapped offsets.
#include "internal.h"
#include "number.cuh"

namespace ps {

namespace {

// ---- the arithmetic of the predictor ------------------------------------------------
// FP32 fields are evaluated in float, FP64 fields in double-float (NumOf, number.cuh):
// an FP64 operation issues at 1/64 of the FP32 rate on this part, so the ~110
// operations per cell of the predictor kept the FP64 pipe saturated (86 %) while HBM
// idled. The FP64 inputs are split on their bit patterns (no FP64 instruction); only
// the outputs are formed in FP64: AD^k rounded once, and u* = u^k + (its increment)
// with one FP64 add.


// One axis of the loader: the neighbour offsets of this cell along the axis (wrapped
// when periodic; 0 past a wall, where the mirrored ghost of the boundary cell is read)
// and whether the cell touches the low or the high wall.
struct NbAxis {
  long om, op;
  int idx, n;
};

template <bool PER>
__device__ __forceinline__ NbAxis nb_axis(int idx, int n, long str) {
  NbAxis a;
  a.idx = idx;
  a.n = n;
  if (PER) {
    a.om = idx > 0 ? -str : (long)(n - 1) * str;
    a.op = idx + 1 < n ? str : -(long)(n - 1) * str;
  } else {
    a.om = idx > 0 ? -str : 0;
    a.op = idx + 1 < n ? str : 0;
  }
  return a;
}

// Contribution of offset o ∈ {−1, 0, 1} along one wall axis: returns false when the
// value is 0 (the normal component ca == this axis on a wall face, stored or implicit)
// and flips s for the ghost of a tangential component.
template <bool PER>
__device__ __forceinline__ bool nb_rule(const NbAxis& a, bool normal, int o, int& s) {
  if (PER) return true;
  if (normal) return !(o < 0 ? a.idx <= 1 : (o == 0 ? a.idx == 0 : a.idx + 1 >= a.n));
  if ((o < 0 && a.idx == 0) || (o > 0 && a.idx + 1 == a.n)) s = -s;
  return true;
}

// CTAs per SM the predictor is compiled for (its register cap), measured on 512×256×256:
// with x and y periodic the uncapped kernel is fastest (3.35 ms, two CTAs per SM; four:
// 3.49 ms); with walls on x or y the wall rules add registers and four CTAs win
// (4.05 ms against 5.24 ms uncapped, walls on every axis).
constexpr int ns_min_blocks(bool px, bool py) { return (px && py) ? 2 : 4; }

template <class T, bool PX, bool PY, bool PZ>
__global__ void __launch_bounds__(256, ns_min_blocks(PX, PY)) ns_predict_kernel(NsArgs<T> a, const T* __restrict__ u3,
                                                         const T* __restrict__ p, const T* ad_prev,
                                                         T* __restrict__ ustar, T* ad_out) {
  using N = NumOf<T>;
  using X = Num<N>;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t sy = (size_t)nx, sz = (size_t)nx * ny, Ncell = sz * nz;
  const T* __restrict__ U = u3;
  const T* __restrict__ V = u3 + Ncell;
  const T* __restrict__ W = u3 + 2 * Ncell;
  // the constants (FP64 fields: the host's hi + lo split, read from the parameter bank)
  auto K = [&](int q, T v) -> N {
    if constexpr (sizeof(T) == 8) return N{a.dc[q].x, a.dc[q].y};
    else return v;
  };
  const N idx = K(0, a.idx), idy = K(1, a.idy), idx2 = K(2, a.idx2), idy2 = K(3, a.idy2);
  const N qx = K(4, a.qx), qy = K(5, a.qy), nu = K(6, a.nu), dt = K(7, a.dt);
  const N alpha = K(8, a.alpha), beta = K(9, a.beta), gamma = K(10, a.gamma);
  const bool use_prev = a.beta != (T)0;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < Ncell; g += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(g % nx);
    const size_t t = g / nx;
    const int j = (int)(t % ny), k = (int)(t / ny);
    const NbAxis ax_x = nb_axis<PX>(i, nx, 1), ax_y = nb_axis<PY>(j, ny, (long)sy),
                 ax_z = nb_axis<PZ>(k, nz, (long)sz);
    // Value of component C (normal to axis ca) at the neighbour (ox, oy, oz) ∈ {−1, 0, 1}³.
    // Along a periodic axis the index wraps; along a wall axis an index beyond either
    // end is the mirrored ghost (−1 times the boundary cell) for a tangential component
    // and 0 for the normal one (the implicit top wall face), and the normal component's
    // own wall face 0 is 0.
    auto ld = [&](const T* __restrict__ C, int ca, int ox, int oy, int oz) -> N {
      const long off = (ox < 0 ? ax_x.om : ox > 0 ? ax_x.op : 0) + (oy < 0 ? ax_y.om : oy > 0 ? ax_y.op : 0) +
                       (oz < 0 ? ax_z.om : oz > 0 ? ax_z.op : 0);
      int s = 1;
      const bool keep = nb_rule<PX>(ax_x, ca == 0, ox, s) && nb_rule<PY>(ax_y, ca == 1, oy, s) &&
                        nb_rule<PZ>(ax_z, ca == 2, oz, s);
      if (!keep) return X::zero();
      const N v = X::in(C[(long)g + off]);
      return s < 0 ? -v : v;
    };
    const bool wall_u = !PX && i == 0, wall_v = !PY && j == 0, wall_w = !PZ && k == 0;
    const N idzf = X::in(a.idzf[k]);
    // 1/(centre distance) below and above cell k; walls: the ghost sits one Δz^f away
    const N ihdn = X::in((k > 0) ? a.idzc[k] : (PZ ? a.idzc[0] : a.idzf[0]));
    const N ihup = X::in((k + 1 < nz) ? a.idzc[k + 1] : (PZ ? a.idzc[0] : a.idzf[nz - 1]));
    const N idzf_m = X::in(a.idzf[k > 0 ? k - 1 : nz - 1]);
    const N qz = X::scale(idzf, 0.25f), qzc = X::scale(ihdn, 0.25f);
    const N uc = ld(U, 0, 0, 0, 0), vc = ld(V, 1, 0, 0, 0), wc = ld(W, 2, 0, 0, 0);
    const N uc2 = X::scale(uc, 2.f), vc2 = X::scale(vc, 2.f), wc2 = X::scale(wc, 2.f);

    // Every flux below is a product of two sums of neighbours (an average each): the two
    // factors ½ go into one factor ¼ on the flux difference (q* = ¼/Δ), and the normal
    // term d(ū²) = ((a + b)² − (c + a)²)/4 is formed as (b − c)(b + 2a + c)/4.
    // ---------------- x momentum at x face i ----------------
    N adu = X::zero();
    if (!wall_u) {
      const N uxp = ld(U, 0, 1, 0, 0), uxm = ld(U, 0, -1, 0, 0);
      const N uyp = ld(U, 0, 0, 1, 0), uym = ld(U, 0, 0, -1, 0);
      const N uzp = ld(U, 0, 0, 0, 1), uzm = ld(U, 0, 0, 0, -1);
      const N duu = (uxp - uxm) * (uxp + uc2 + uxm) * qx;
      // uv on the y faces j and j+1 of this x face
      const N uv0 = (uc + uym) * (vc + ld(V, 1, -1, 0, 0));
      const N uv1 = (uyp + uc) * (ld(V, 1, 0, 1, 0) + ld(V, 1, -1, 1, 0));
      const N duv = (uv1 - uv0) * qy;
      // uw on the z faces k and k+1 of this x face
      const N uw0 = (uc + uzm) * (wc + ld(W, 2, -1, 0, 0));
      const N uw1 = (uzp + uc) * (ld(W, 2, 0, 0, 1) + ld(W, 2, -1, 0, 1));
      const N duw = (uw1 - uw0) * qz;
      const N lap = (uxp - uc2 + uxm) * idx2 + (uyp - uc2 + uym) * idy2 +
                    ((uzp - uc) * ihup - (uc - uzm) * ihdn) * idzf;
      adu = nu * lap - (duu + duv + duw);
    }
    // ---------------- y momentum at y face j ----------------
    N adv = X::zero();
    if (!wall_v) {
      const N vxp = ld(V, 1, 1, 0, 0), vxm = ld(V, 1, -1, 0, 0);
      const N vyp = ld(V, 1, 0, 1, 0), vym = ld(V, 1, 0, -1, 0);
      const N vzp = ld(V, 1, 0, 0, 1), vzm = ld(V, 1, 0, 0, -1);
      const N dvv = (vyp - vym) * (vyp + vc2 + vym) * qy;
      // uv on the x faces i and i+1 of this y face
      const N uv0 = (uc + ld(U, 0, 0, -1, 0)) * (vc + vxm);
      const N uv1 = (ld(U, 0, 1, 0, 0) + ld(U, 0, 1, -1, 0)) * (vxp + vc);
      const N duv = (uv1 - uv0) * qx;
      const N vw0 = (vc + vzm) * (wc + ld(W, 2, 0, -1, 0));
      const N vw1 = (vzp + vc) * (ld(W, 2, 0, 0, 1) + ld(W, 2, 0, -1, 1));
      const N dvw = (vw1 - vw0) * qz;
      const N lap = (vxp - vc2 + vxm) * idx2 + (vyp - vc2 + vym) * idy2 +
                    ((vzp - vc) * ihup - (vc - vzm) * ihdn) * idzf;
      adv = nu * lap - (duv + dvv + dvw);
    }
    // ---------------- z momentum at z face k ----------------
    N adw = X::zero();
    if (!wall_w) {
      const N wzp = ld(W, 2, 0, 0, 1), wzm = ld(W, 2, 0, 0, -1);
      const N wxp = ld(W, 2, 1, 0, 0), wxm = ld(W, 2, -1, 0, 0);
      const N wyp = ld(W, 2, 0, 1, 0), wym = ld(W, 2, 0, -1, 0);
      const N dww = (wzp - wzm) * (wzp + wc2 + wzm) * qzc;
      // uw on the x faces i and i+1 of this z face (u averaged over cells k−1 and k)
      const N uw0 = (uc + ld(U, 0, 0, 0, -1)) * (wc + wxm);
      const N uw1 = (ld(U, 0, 1, 0, 0) + ld(U, 0, 1, 0, -1)) * (wxp + wc);
      const N duw = (uw1 - uw0) * qx;
      const N vw0 = (vc + ld(V, 1, 0, 0, -1)) * (wc + wym);
      const N vw1 = (ld(V, 1, 0, 1, 0) + ld(V, 1, 0, 1, -1)) * (wyp + wc);
      const N dvw = (vw1 - vw0) * qy;
      const N lap = (wxp - wc2 + wxm) * idx2 + (wyp - wc2 + wym) * idy2 +
                    ((wzp - wc) * idzf - (wc - wzm) * idzf_m) * ihdn;
      adw = nu * lap - (duw + dvw + dww);
    }

    // ---------------- predictor (2a) ----------------
    const N pc = X::in(p[g]);
    const N gpx = wall_u ? X::zero() : (pc - X::in(p[g + (i > 0 ? -1 : nx - 1)])) * idx;
    const N gpy = wall_v ? X::zero() : (pc - X::in(p[g + (j > 0 ? -(long)sy : (long)((ny - 1) * sy))])) * idy;
    const N gpz = wall_w ? X::zero() : (pc - X::in(p[g + (k > 0 ? -(long)sz : (long)((nz - 1) * sz))])) * ihdn;
    N incu = alpha * adu - gamma * gpx, incv = alpha * adv - gamma * gpy, incw = alpha * adw - gamma * gpz;
    if (use_prev) {
      incu = incu + beta * X::in(ad_prev[g]);
      incv = incv + beta * X::in(ad_prev[g + Ncell]);
      incw = incw + beta * X::in(ad_prev[g + 2 * Ncell]);
    }
    ustar[g] = wall_u ? U[g] : U[g] + X::out(dt * incu);
    ustar[g + Ncell] = wall_v ? V[g] : V[g] + X::out(dt * incv);
    ustar[g + 2 * Ncell] = wall_w ? W[g] : W[g] + X::out(dt * incw);
    ad_out[g] = X::out(adu);
    ad_out[g + Ncell] = X::out(adv);
    ad_out[g + 2 * Ncell] = X::out(adw);
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
  const int sel = (a.per_x ? 1 : 0) | (a.per_y ? 2 : 0) | (a.per_z ? 4 : 0);
  auto go = [&](auto k) {
    k<<<grid_for(N), 256, 0, st>>>(a, static_cast<const T*>(u3), static_cast<const T*>(p),
                                   static_cast<const T*>(ad_prev), static_cast<T*>(ustar), static_cast<T*>(ad_out));
  };
  switch (sel) {
    case 0: go(ns_predict_kernel<T, false, false, false>); break;
    case 1: go(ns_predict_kernel<T, true, false, false>); break;
    case 2: go(ns_predict_kernel<T, false, true, false>); break;
    case 3: go(ns_predict_kernel<T, true, true, false>); break;
    case 4: go(ns_predict_kernel<T, false, false, true>); break;
    case 5: go(ns_predict_kernel<T, true, false, true>); break;
    case 6: go(ns_predict_kernel<T, false, true, true>); break;
    default: go(ns_predict_kernel<T, true, true, true>); break;
  }
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
