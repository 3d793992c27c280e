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
// z face k). A CTA owns a tile of 32 × 4 cells in (x, y) and marches along z over a
// chunk of planes. Each plane of u, v, w and p enters a four-slot shared ring once,
// with a one-cell halo on every side: loaded, split into the number type, and with
// the axis rules already applied (wrap, mirrored ghost, or the zero wall face), so
// that the flux formulas below are those of the periodic box and every neighbour is
// one shared-memory read. A plane is split once instead of once per neighbour that
// reads it, which was most of the integer work of a cell-per-thread loader. The ring
// holds planes k−1, k and k+1 while the fill of plane k+1 overwrites the slot of
// k−3, so one barrier per plane suffices.
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

// Tile and residency, measured on 512×256×256 (channel; walls on every axis): 32 × 4
// cells at eight CTAs per SM (64 registers, a few spilled) 1.76 / 1.91 ms; 32 × 4 at
// five (no spills) 1.94 / 1.97; 32 × 8 at two, three, four CTAs 2.36 / 2.01 / 1.82 ms.
// The kernel waits on its shared-memory and ring loads, so warps beat registers.
constexpr int PTX = 32, PTY = 4;                  // cells of a tile in x and y
constexpr int PMINB = 8;                          // CTAs per SM the registers are capped for
constexpr int PW = PTX + 2, PCELLS = PW * (PTY + 2);  // the tile with its halo
constexpr int PSLOTS = 4;                         // plane ring
constexpr int PITEMS = (4 * PCELLS + PTX * PTY - 1) / (PTX * PTY);  // ring entries a thread fills

// Where the in-plane halo position pos ∈ [−1, n] of one field reads from along one
// axis: the wrapped index when periodic; past a wall the boundary cell with the sign
// flipped (tangential component), or 0 at and beyond the wall faces (the component
// normal to this axis: face 0 is stored, the top face is implicit).
__device__ __forceinline__ int halo_src(int pos, int n, bool per, bool normal, bool& flip, bool& zero) {
  if (per) return pos < 0 ? pos + n : (pos >= n ? pos - n : pos);
  if (normal) {
    zero |= (pos <= 0 || pos >= n);
    return pos < 0 ? 0 : (pos >= n ? n - 1 : pos);
  }
  if (pos < 0 || pos >= n) flip = !flip;
  return pos < 0 ? 0 : (pos >= n ? n - 1 : pos);
}

template <class T, bool PX, bool PY, bool PZ>
__global__ void __launch_bounds__(PTX * PTY, PMINB) ns_predict_kernel(NsArgs<T> a, const T* __restrict__ u3,
                                                                  const T* __restrict__ p, const T* ad_prev,
                                                                  T* __restrict__ ustar, T* ad_out, int zchunk) {
  using N = NumOf<T>;
  using X = Num<N>;
  struct Slot {
    N f[4][PCELLS];  // u, v, w, p of one plane (tile and halo)
    N m[4];          // the plane's z metrics: 1/Δz^f_k, 1/Δz^c below and above, 1/Δz^f_{k−1}
  };
  __shared__ Slot ring[PSLOTS];
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t sy = (size_t)nx, sz = (size_t)nx * ny, Ncell = sz * nz;
  const T* __restrict__ U = u3;
  const T* __restrict__ V = u3 + Ncell;
  const T* __restrict__ W = u3 + 2 * Ncell;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * PTX + tx;
  const int x0 = blockIdx.x * PTX, y0 = blockIdx.y * PTY;
  const int i = x0 + tx, j = y0 + ty;
  const int k0 = blockIdx.z * zchunk, k1 = min(nz, k0 + zchunk);

  // The ring entries this thread fills in every plane: field, in-plane source
  // offset, and the x/y rule bits (flip the sign, or store 0). Halo positions beyond
  // the ghost of a partial tile are read by no cell and store 0.
  int off[PITEMS];
  uint32_t flipm = 0, zerom = 0;
#pragma unroll
  for (int h = 0; h < PITEMS; ++h) {
    const int e = tid + h * PTX * PTY;
    const int c = e / PCELLS, cell = e - c * PCELLS;
    const int rr = cell / PW, cc = cell - rr * PW;
    const int gi = x0 - 1 + cc, gj = y0 - 1 + rr;
    bool flip = false, zero = e >= 4 * PCELLS || gi > nx || gj > ny;
    int si = 0, sj = 0;
    if (!zero) {
      // p is read only at (−1, 0) and (0, −1), and there only away from a wall: wrap
      si = halo_src(gi, nx, PX || c == 3, c == 0, flip, zero);
      sj = halo_src(gj, ny, PY || c == 3, c == 1, flip, zero);
    }
    off[h] = zero ? 0 : sj * nx + si;
    flipm |= (flip ? 1u : 0u) << h;
    zerom |= (zero ? 1u : 0u) << h;
  }

  // Fill the ring slot of logical plane q ∈ [−1, n_z] (the z rules as in x and y).
  auto fill = [&](int q) {
    Slot& s = ring[q & (PSLOTS - 1)];
    const int qw = q < 0 ? q + nz : (q >= nz ? q - nz : q);  // wrapped
    const int qc = q < 0 ? 0 : (q >= nz ? nz - 1 : q);        // clamped
    const bool out = q < 0 || q >= nz;
    // per field: source plane, sign flip, zero plane
    const size_t pu = (size_t)(PZ ? qw : qc) * sz, pp = (size_t)qw * sz;
    const bool fl = !PZ && out;                   // u, v: the mirrored ghost plane
    const bool zw = !PZ && (q <= 0 || q >= nz);   // w: face 0 and beyond the walls
    T raw[PITEMS];
#pragma unroll
    for (int h = 0; h < PITEMS; ++h) {
      const int e = tid + h * PTX * PTY;
      const int c = e / PCELLS;
      const bool z = ((zerom >> h) & 1u) || (c == 2 && zw);
      const T* __restrict__ src = c == 3 ? p + pp : u3 + (size_t)(c < 3 ? c : 0) * Ncell + pu;
      raw[h] = z ? (T)0 : src[off[h]];
    }
#pragma unroll
    for (int h = 0; h < PITEMS; ++h) {
      const int e = tid + h * PTX * PTY;
      if (h < PITEMS - 1 || e < 4 * PCELLS) {
        const int c = e / PCELLS, cell = e - c * PCELLS;
        const bool f = ((flipm >> h) & 1u) != (c < 2 && fl);
        const N v = X::in(raw[h]);
        s.f[c][cell] = f ? -v : v;
      }
    }
    if (tid < 4 && !out) {
      // 1/(centre distance) below and above cell q; walls: the ghost sits one Δz^f away
      const T mq = tid == 0 ? a.idzf[q]
                 : tid == 1 ? ((q > 0) ? a.idzc[q] : (PZ ? a.idzc[0] : a.idzf[0]))
                 : tid == 2 ? ((q + 1 < nz) ? a.idzc[q + 1] : (PZ ? a.idzc[0] : a.idzf[nz - 1]))
                            : a.idzf[q > 0 ? q - 1 : nz - 1];
      s.m[tid] = X::in(mq);
    }
  };

  // the constants (FP64 fields: the host's hi + lo split, read from the parameter bank)
  auto K = [&](int q, T v) -> N {
    if constexpr (sizeof(T) == 8) return N{a.dc[q].x, a.dc[q].y};
    else return v;
  };
  const bool use_prev = a.beta != (T)0;
  const bool live = i < nx && j < ny;
  const bool wall_u = !PX && i == 0, wall_v = !PY && j == 0;
  const int cc0 = (ty + 1) * PW + tx + 1;  // this cell in a ring plane

  fill(k0 - 1);
  fill(k0);
  for (int k = k0; k < k1; ++k) {
    fill(k + 1);
    __syncthreads();  // plane k+1 published; every read of the slot it replaced is done
    if (!live) continue;
    const N idx = K(0, a.idx), idy = K(1, a.idy), idx2 = K(2, a.idx2), idy2 = K(3, a.idy2);
    const N qx = K(4, a.qx), qy = K(5, a.qy), nu = K(6, a.nu), dt = K(7, a.dt);
    const N alpha = K(8, a.alpha), beta = K(9, a.beta), gamma = K(10, a.gamma);
    const Slot& sm = ring[(k - 1) & (PSLOTS - 1)];
    const Slot& s0 = ring[k & (PSLOTS - 1)];
    const Slot& sp = ring[(k + 1) & (PSLOTS - 1)];
    // component C at the neighbour (ox, oy, oz) ∈ {−1, 0, 1}³
    auto ld = [&](int C, int ox, int oy, int oz) -> N {
      const Slot& s = oz < 0 ? sm : (oz > 0 ? sp : s0);
      return s.f[C][cc0 + oy * PW + ox];
    };
    const bool wall_w = !PZ && k == 0;
    const N idzf = s0.m[0], ihdn = s0.m[1], ihup = s0.m[2], idzf_m = s0.m[3];
    const N qz = X::scale(idzf, 0.25f), qzc = X::scale(ihdn, 0.25f);
    const N uc = ld(0, 0, 0, 0), vc = ld(1, 0, 0, 0), wc = ld(2, 0, 0, 0);
    const N uc2 = X::scale(uc, 2.f), vc2 = X::scale(vc, 2.f), wc2 = X::scale(wc, 2.f);

    // Every flux below is a product of two sums of neighbours (an average each): the two
    // factors ½ go into one factor ¼ on the flux difference (q* = ¼/Δ), and the normal
    // term d(ū²) = ((a + b)² − (c + a)²)/4 is formed as (b − c)(b + 2a + c)/4.
    // ---------------- x momentum at x face i ----------------
    N adu = X::zero();
    if (!wall_u) {
      const N uxp = ld(0, 1, 0, 0), uxm = ld(0, -1, 0, 0);
      const N uyp = ld(0, 0, 1, 0), uym = ld(0, 0, -1, 0);
      const N uzp = ld(0, 0, 0, 1), uzm = ld(0, 0, 0, -1);
      const N duu = (uxp - uxm) * (uxp + uc2 + uxm) * qx;
      // uv on the y faces j and j+1 of this x face
      const N uv0 = (uc + uym) * (vc + ld(1, -1, 0, 0));
      const N uv1 = (uyp + uc) * (ld(1, 0, 1, 0) + ld(1, -1, 1, 0));
      const N duv = (uv1 - uv0) * qy;
      // uw on the z faces k and k+1 of this x face
      const N uw0 = (uc + uzm) * (wc + ld(2, -1, 0, 0));
      const N uw1 = (uzp + uc) * (ld(2, 0, 0, 1) + ld(2, -1, 0, 1));
      const N duw = (uw1 - uw0) * qz;
      const N lap = (uxp - uc2 + uxm) * idx2 + (uyp - uc2 + uym) * idy2 +
                    ((uzp - uc) * ihup - (uc - uzm) * ihdn) * idzf;
      adu = nu * lap - (duu + duv + duw);
    }
    // ---------------- y momentum at y face j ----------------
    N adv = X::zero();
    if (!wall_v) {
      const N vxp = ld(1, 1, 0, 0), vxm = ld(1, -1, 0, 0);
      const N vyp = ld(1, 0, 1, 0), vym = ld(1, 0, -1, 0);
      const N vzp = ld(1, 0, 0, 1), vzm = ld(1, 0, 0, -1);
      const N dvv = (vyp - vym) * (vyp + vc2 + vym) * qy;
      // uv on the x faces i and i+1 of this y face
      const N uv0 = (uc + ld(0, 0, -1, 0)) * (vc + vxm);
      const N uv1 = (ld(0, 1, 0, 0) + ld(0, 1, -1, 0)) * (vxp + vc);
      const N duv = (uv1 - uv0) * qx;
      const N vw0 = (vc + vzm) * (wc + ld(2, 0, -1, 0));
      const N vw1 = (vzp + vc) * (ld(2, 0, 0, 1) + ld(2, 0, -1, 1));
      const N dvw = (vw1 - vw0) * qz;
      const N lap = (vxp - vc2 + vxm) * idx2 + (vyp - vc2 + vym) * idy2 +
                    ((vzp - vc) * ihup - (vc - vzm) * ihdn) * idzf;
      adv = nu * lap - (duv + dvv + dvw);
    }
    // ---------------- z momentum at z face k ----------------
    N adw = X::zero();
    if (!wall_w) {
      const N wzp = ld(2, 0, 0, 1), wzm = ld(2, 0, 0, -1);
      const N wxp = ld(2, 1, 0, 0), wxm = ld(2, -1, 0, 0);
      const N wyp = ld(2, 0, 1, 0), wym = ld(2, 0, -1, 0);
      const N dww = (wzp - wzm) * (wzp + wc2 + wzm) * qzc;
      // uw on the x faces i and i+1 of this z face (u averaged over cells k−1 and k)
      const N uw0 = (uc + ld(0, 0, 0, -1)) * (wc + wxm);
      const N uw1 = (ld(0, 1, 0, 0) + ld(0, 1, 0, -1)) * (wxp + wc);
      const N duw = (uw1 - uw0) * qx;
      const N vw0 = (vc + ld(1, 0, 0, -1)) * (wc + wym);
      const N vw1 = (ld(1, 0, 1, 0) + ld(1, 0, 1, -1)) * (wyp + wc);
      const N dvw = (vw1 - vw0) * qy;
      const N lap = (wxp - wc2 + wxm) * idx2 + (wyp - wc2 + wym) * idy2 +
                    ((wzp - wc) * idzf - (wc - wzm) * idzf_m) * ihdn;
      adw = nu * lap - (duw + dvw + dww);
    }

    // ---------------- predictor (2a) ----------------
    const size_t g = (size_t)k * sz + (size_t)j * sy + i;
    const N pc = ld(3, 0, 0, 0);
    const N gpx = wall_u ? X::zero() : (pc - ld(3, -1, 0, 0)) * idx;
    const N gpy = wall_v ? X::zero() : (pc - ld(3, 0, -1, 0)) * idy;
    const N gpz = wall_w ? X::zero() : (pc - ld(3, 0, 0, -1)) * ihdn;
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
  const int sel = (a.per_x ? 1 : 0) | (a.per_y ? 2 : 0) | (a.per_z ? 4 : 0);
  // (x, y) tiles × chunks of z planes: 32 CTAs per SM in all (four waves), each chunk
  // paying two extra plane fills (8 or 128 per SM measured slower)
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int gx = (a.nx + PTX - 1) / PTX, gy = (a.ny + PTY - 1) / PTY;
  const long tiles = (long)gx * gy, want = 32L * sms;
  long nch = (want + tiles - 1) / tiles;
  if (nch > a.nz) nch = a.nz;
  const int zchunk = (int)((a.nz + nch - 1) / nch);
  const dim3 grid(gx, gy, (a.nz + zchunk - 1) / zchunk);
  auto go = [&](auto k) {
    k<<<grid, dim3(PTX, PTY), 0, st>>>(a, static_cast<const T*>(u3), static_cast<const T*>(p),
                                       static_cast<const T*>(ad_prev), static_cast<T*>(ustar),
                                       static_cast<T*>(ad_out), zchunk);
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
