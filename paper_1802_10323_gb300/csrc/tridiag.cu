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
#include <type_traits>

#include "tridiag_dev.cuh"

namespace ps {

// FP32, non-periodic columns: the forward sweep keeps the eliminated
// (c'_k, d'_k) only at the end of every chunk of ZK planes (1/8 of the data
// volume, in the scratch array); the backward sweep walks the chunks from the top,
// re-reads each chunk's right-hand side, recomputes its (c', d') from the
// checkpoint in registers (the same instructions on the same inputs, so
// bit-identical to the forward sweep) and back-substitutes. HBM traffic: read f̂
// twice (the second read of a chunk often hits L2), write Φ̂ once; loads of the
// next chunk are issued before the current chunk is processed. The coefficients
// (a_k, b_k, c_k), with a_0 = c_{n−1} = 0, sit in a shared table (one broadcast
// load per row) and whole chunks run without per-row bound tests.
template <class T>
cudaError_t launch_zsolve(ZArgs<T> a, cudaStream_t st);

constexpr int ZK = 16;
constexpr int ZB = 128;            // columns (threads) per CTA
constexpr int ZTAB_MAX = 4096;     // planes whose coefficient table fits in shared memory

// The FP32 elimination of a column with a small |λ| (low wavenumbers) errs by about
// ε_32·κ, κ ≈ ‖T_z‖/|λ| up to ~10^7 on the stretched channel grid, and that error
// is smooth in z with a large amplitude: exactly what an FP32 correction solve
// removes worst (its own transform rounding, amplified by ‖A‖, scales with the
// correction's size). Those few columns — a rectangle q_x < lowx, q_y < lowy chosen
// at plan creation from κ — are solved here in double-float arithmetic, ~2^−46
// relative per operation against ε_32 = 2^−24 (Thomas with c' and d' as float pairs in
// the FP64-sized scratch; the singular column (0,0) with its weighted-mean pinning),
// by CTAs of the same launch as the FP32 columns, so they overlap them. Output
// rounded to FP32.
constexpr int ZL = 4;  // rows in flight per rectangle column (keeps the kernel's registers at the FP32 path's)

// Those columns run in double-float arithmetic (pairs of floats, ~48-bit significand)
// rather than in FP64: on this part one FP64 warp instruction occupies its SM
// sub-partition's FP64 pipe for ~33 ns whatever the number of active lanes (measured:
// a dependent FP64 FMA chain 32.8 ns per step with 1, 8 or 32 lanes, 2.3 ns in FP32),
// and a row of the FP64 elimination took about eleven of them, so the rectangle's
// sequential sweeps were the z pass's critical path on small planes. The coefficients
// are split on their bit patterns; no FP64 instruction remains in the row loops. The
// result is rounded to FP32, far above the ~2^−46 relative error of these operations.

// 1/x of a double-float pivot: the FP32 approximation r refined by one Newton step
// carried in double-float, r + r·e with e = 1 − x·r (x.h·r is formed exactly with an
// FMA; 1 − p is exact for p near 1), about 2^−46 relative.
__device__ __forceinline__ df df_rcp(df x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.h));
  const float p = __fmul_rn(x.h, r);
  const float pe = __fmaf_rn(x.h, r, -p);
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p), pe), __fmul_rn(x.l, r));
  return quick_two_sum(r, __fmul_rn(r, e));
}

// Called by all 32 lanes of a warp (t = the warp's first column + lane).
__device__ void zlow_column(const ZArgs<float>& a, int t) {
  const int nrect = a.lowx * a.lowy;
  const size_t st = (size_t)a.nx * a.ny;
  const int nz = a.nz;
  const int lane = threadIdx.x & 31;
  // The singular column (0,0) is t = 0: its Δz^f-weighted mean (and, below, its final
  // shift) is a loop over the whole column, taken by every lane of its warp rather than
  // by lane 0 alone while the others wait.
  const bool sing_warp = a.singular && (t >> 5) == 0;
  double mean = 0.0, wsum = 0.0;
  if (sing_warp) {  // remove the Δz^f-weighted mean of the right-hand side; Φ̂_0 = 0 pinned
    for (int k = lane; k < nz; k += 32) {
      mean += a.dzf64[k] * (double)a.data[k * st];
      wsum += a.dzf64[k];
    }
    for (int o = 16; o > 0; o >>= 1) {
      mean += __shfl_xor_sync(0xffffffffu, mean, o);
      wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    }
    mean /= wsum;
  }
  const unsigned live = __ballot_sync(0xffffffffu, t < nrect);  // lanes with a column
  if (t >= nrect) return;
  const int i = t % a.lowx, j = t / a.lowx;
  const int col = j * a.nx + i;
  float* d = a.data + col;
  // (c'_k, d'_k) as float pairs in the FP64 scratch: [k][nrect] each
  float2* cs = reinterpret_cast<float2*>(a.scr64) + t;
  float2* ds = reinterpret_cast<float2*>(a.scr64) + (size_t)nz * nrect + t;
  const bool sing = a.singular && col == 0;
  const df mn = sing ? df_from_f64(mean) : df{0.f, 0.f};
  const df lam = sing ? df{0.f, 0.f} : df_from_f64(a.lamx64[i] + a.lamy64[j]);
  const int kb = sing ? 1 : 0;
  // forward sweep over chunks of ZL rows, the next chunk's right-hand side in flight
  float cur[ZL], nxt[ZL];
  auto load = [&](int k0, float* buf) {
#pragma unroll
    for (int u = 0; u < ZL; ++u) buf[u] = (k0 + u < nz) ? d[(size_t)(k0 + u) * st] : 0.f;
  };
  load(0, cur);
  df cp = {0.f, 0.f}, dp = {0.f, 0.f};
  for (int k0 = 0; k0 < nz; k0 += ZL) {
    if (k0 + ZL < nz) load(k0 + ZL, nxt);
#pragma unroll
    for (int u = 0; u < ZL; ++u) {
      const int k = k0 + u;
      if (k >= kb && k < nz) {
        const df ak = (k > kb) ? df_from_f64(__ldg(a.za64 + k)) : df{0.f, 0.f};
        const df ck = (k < nz - 1) ? df_from_f64(__ldg(a.zc64 + k)) : df{0.f, 0.f};
        const df bk = df_add(df_from_f64(__ldg(a.zb64 + k)), lam);
        const df mk = df_rcp(df_sub(bk, df_mul(ak, cp)));
        cp = df_mul(ck, mk);
        dp = df_mul(df_sub(df_sub(df{cur[u], 0.f}, mn), df_mul(ak, dp)), mk);
        cs[(size_t)k * nrect] = make_float2(cp.h, cp.l);
        ds[(size_t)k * nrect] = make_float2(dp.h, dp.l);
      }
    }
#pragma unroll
    for (int u = 0; u < ZL; ++u) cur[u] = nxt[u];
  }
  // backward sweep, chunks of (c', d') from the top with the chunk below in flight
  float2 cb[ZL], db[ZL], cn[ZL], dn[ZL];
  const int klast = ((nz - 1) / ZL) * ZL;
  auto loadb = [&](int k0, float2* c_, float2* d_) {
#pragma unroll
    for (int u = 0; u < ZL; ++u) {
      const int k = k0 + u;
      c_[u] = (k < nz) ? cs[(size_t)k * nrect] : make_float2(0.f, 0.f);
      d_[u] = (k < nz) ? ds[(size_t)k * nrect] : make_float2(0.f, 0.f);
    }
  };
  loadb(klast, cb, db);
  df x = {0.f, 0.f}, xs = {0.f, 0.f};
  for (int k0 = klast; k0 >= 0; k0 -= ZL) {
    if (k0 > 0) loadb(k0 - ZL, cn, dn);
#pragma unroll
    for (int u = ZL - 1; u >= 0; --u) {
      const int k = k0 + u;
      if (k >= kb && k < nz) {
        const df ck = (k < nz - 1) ? df{cb[u].x, cb[u].y} : df{0.f, 0.f};
        x = df_sub(df{db[u].x, db[u].y}, df_mul(ck, x));
        db[u] = make_float2(x.h, x.l);
        if (sing) xs = df_add(xs, df_mul(df_from_f64(a.dzf64[k]), x));
      }
    }
    if (!sing) {
#pragma unroll
      for (int u = 0; u < ZL; ++u)
        if (k0 + u < nz) d[(size_t)(k0 + u) * st] = __fadd_rn(db[u].x, db[u].y);
    } else {
#pragma unroll
      for (int u = 0; u < ZL; ++u)
        if (k0 + u >= kb && k0 + u < nz) ds[(size_t)(k0 + u) * nrect] = db[u];
    }
#pragma unroll
    for (int u = 0; u < ZL; ++u) {
      cb[u] = cn[u];
      db[u] = dn[u];
    }
  }
  if (sing_warp) {  // the singular column keeps zero weighted mean (its warp's live lanes)
    const double mx = __shfl_sync(live, ((double)xs.h + (double)xs.l) / wsum, 0);
    __syncwarp(live);  // lane 0's scratch stores are visible to the lanes reading them below
    const int rank = __popc(live & ((1u << lane) - 1u)), nl = __popc(live);
    float* d0 = a.data;
    const float2* ds0 = reinterpret_cast<const float2*>(a.scr64) + (size_t)nz * nrect;  // column t = 0
    const df nmx = df_from_f64(-mx);
    if (rank == 0) d0[0] = nmx.h + nmx.l;
    for (int k = 1 + rank; k < nz; k += nl) {
      const float2 v = ds0[(size_t)k * nrect];
      const df y = df_add(df{v.x, v.y}, nmx);
      d0[(size_t)k * st] = __fadd_rn(y.h, y.l);
    }
  }
}

// 1/x by the hardware approximation (`rcp.approx.ftz.f32`, about 1 ulp): the pivots
// here are normal FP32 numbers far from the overflow range.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <bool TAB>
__global__ void __launch_bounds__(ZB) zsolve_ckpt_kernel(ZArgs<float> a, int nlowb) {
  if (a.skip && *a.skip) return;
  if ((int)blockIdx.x < nlowb) {  // the rectangle of low wavenumbers: one warp per CTA,
    // so that its columns spread over many SMs
    if (threadIdx.x < 32) zlow_column(a, blockIdx.x * 32 + threadIdx.x);
    return;
  }
  extern __shared__ float4 ztab[];  // [nz] (a_k, b_k, c_k, ·) when TAB
  const int nz = a.nz;
  auto coef = [&](int k) -> float4 {
    if constexpr (TAB) {
      return ztab[k];
    } else {
      return make_float4(k > 0 ? __ldg(a.za + k) : 0.f, __ldg(a.zb + k), k < nz - 1 ? __ldg(a.zc + k) : 0.f, 0.f);
    }
  };
  if constexpr (TAB) {
    for (int k = threadIdx.x; k < nz; k += ZB)
      ztab[k] = make_float4(k > 0 ? a.za[k] : 0.f, a.zb[k], k < nz - 1 ? a.zc[k] : 0.f, 0.f);
    __syncthreads();
  }
  const int ncol = a.nx * a.ny;
  float2* __restrict__ ck = reinterpret_cast<float2*>(a.scr_c);  // [nchunk][ncol]
  const int col = (blockIdx.x - nlowb) * ZB + threadIdx.x;
  const int colc = col < ncol ? col : ncol - 1;
  const int i = colc % a.nx, j = colc / a.nx;
  const bool act = col < ncol && !(a.singular && col == 0) && !(i < a.lowx && j < a.lowy);
  const float lam = a.lamx[i] + a.lamy[j];
  const size_t st = (size_t)ncol;
  const int nch = (nz + ZK - 1) / ZK, nfull = nz / ZK;
  float* __restrict__ d = a.data + colc;

  // one chunk of the elimination: rows k0 … k0+ZK−1 (all present when FULL)
  auto eliminate = [&](int k0, const float* cur, float& cp, float& dp, float* cpa, float* dpa,
                       auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
    for (int u = 0; u < ZK; ++u) {
      const int k = k0 + u;
      if (FULL || k < nz) {
        const float4 q = coef(k);
        const float mk = rcp_approx(q.y + lam - q.x * cp);
        cp = q.z * mk;
        dp = (cur[u] - q.x * dp) * mk;
      }
      if (cpa) {
        cpa[u] = cp;
        dpa[u] = dp;
      }
    }
  };
  auto load = [&](int k0, float* buf, auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
    const float* src = d + (size_t)k0 * st;
#pragma unroll
    for (int u = 0; u < ZK; ++u) buf[u] = (FULL || k0 + u < nz) ? src[(size_t)u * st] : 0.f;
  };

  // L2 prefetch of the chunk after next (both sweeps), so that more of the column
  // is in flight than the registers of the next chunk allow
  auto prefetch = [&](int c2) {
    if (c2 >= 0 && c2 < nfull) {
      const float* src = d + (size_t)c2 * ZK * st;
#pragma unroll
      for (int u = 0; u < ZK; ++u) asm volatile("prefetch.global.L2 [%0];" ::"l"(src + (size_t)u * st));
    }
  };
  float cur[ZK], nxt[ZK];
  if (nfull > 0) load(0, cur, std::true_type{});
  else load(0, cur, std::false_type{});
  float cp = 0.f, dp = 0.f;
  for (int c = 0; c < nch; ++c) {
    const int k0 = c * ZK;
    prefetch(c + 2);
    if (c + 1 < nfull) load(k0 + ZK, nxt, std::true_type{});
    else if (c + 1 < nch) load(k0 + ZK, nxt, std::false_type{});
    if (c < nfull) eliminate(k0, cur, cp, dp, nullptr, nullptr, std::true_type{});
    else eliminate(k0, cur, cp, dp, nullptr, nullptr, std::false_type{});
    ck[(size_t)c * ncol + colc] = make_float2(cp, dp);
#pragma unroll
    for (int u = 0; u < ZK; ++u) cur[u] = nxt[u];
  }
  // backward: chunks from the top; prefetch the chunk below
  if (nch - 1 < nfull) load((nch - 1) * ZK, cur, std::true_type{});
  else load((nch - 1) * ZK, cur, std::false_type{});
  float x = 0.f;
  for (int c = nch - 1; c >= 0; --c) {
    const int k0 = c * ZK;
    prefetch(c - 2);
    if (c > 0) load(k0 - ZK, nxt, std::true_type{});  // every chunk below the last is full
    const float2 prev = (c > 0) ? ck[(size_t)(c - 1) * ncol + colc] : make_float2(0.f, 0.f);
    float cpa[ZK], dpa[ZK];
    cp = prev.x;
    dp = prev.y;
    if (c < nfull) eliminate(k0, cur, cp, dp, cpa, dpa, std::true_type{});
    else eliminate(k0, cur, cp, dp, cpa, dpa, std::false_type{});
    float* dst = d + (size_t)k0 * st;
#pragma unroll
    for (int u = ZK - 1; u >= 0; --u) {
      const int k = k0 + u;
      if (c < nfull || k < nz) {
        x = dpa[u] - cpa[u] * x;  // c'_{n−1} = 0: the table holds c_{n−1} = 0
        if (act) dst[(size_t)u * st] = x;
      }
    }
#pragma unroll
    for (int u = 0; u < ZK; ++u) cur[u] = nxt[u];
  }
}

cudaError_t launch_zsolve_ckpt(ZArgs<float> a, cudaStream_t st) {
  const int ncol = a.nx * a.ny;
  const int nlowb = (a.lowx * a.lowy + 31) / 32;  // FP64 CTAs first (they run longest)
  const int grid = nlowb + (ncol + ZB - 1) / ZB;
  if (a.nz <= ZTAB_MAX) {
    const size_t smem = (size_t)a.nz * sizeof(float4);
    static size_t smem_set = 0;
    if (smem > smem_set) {
      cudaError_t e = cudaFuncSetAttribute(zsolve_ckpt_kernel<true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZTAB_MAX * 16);
      if (e != cudaSuccess) return e;
      smem_set = (size_t)ZTAB_MAX * 16;
    }
    zsolve_ckpt_kernel<true><<<grid, ZB, smem, st>>>(a, nlowb);
  } else {
    zsolve_ckpt_kernel<false><<<grid, ZB, 0, st>>>(a, nlowb);
  }
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
