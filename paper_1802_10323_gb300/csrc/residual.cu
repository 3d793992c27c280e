// residual.cu — r = f − A·Φ (Eq. 4) for the iterative refinement, in double-float.
//
// Φ and f are FP64 fields. FP64 arithmetic and f64<->f32 conversions issue at
// ~1/64 of the FP32 rate on this part, so each value is split on its bit pattern
// into hi + lo floats (48 significant bits) and the 7-point stencil is evaluated
// with error-free transformations (TwoSum, FMA products). The residual is
// rounded once to FP32 (the right-hand side of the next FP32 correction solve).
//
// Blocking: a CTA of 32 × 8 threads owns a 32 × 8 (x, y) tile and marches along
// z over a chunk of planes, keeping Φ_{k−1}, Φ_k, Φ_{k+1} of its column in
// registers; x and y neighbours come from a double-buffered shared plane with
// one halo column/row per side. Every FP64 value is loaded from HBM and split
// once (halos aside).
//
// Ends of each axis (staggered ghost rules of Table 1): periodic wraps; a
// Neumann end contributes nothing; a Dirichlet end contributes
// coef·(ghost − Φ) = coef·(−2Φ). In z the coefficients zlo/zhi already hold
// a_k, c_k, the wrap couplings, or 1/(Δz^f)² at a Dirichlet end.
//
// Reductions per pass (deterministic): max and min of r and of f (order-
// preserving integer keys, atomicMax/atomicMin), and, for singular problems,
// per-block double-float sums of Δz^f·r and Δz^f·f for the weighted means. The
// finalize kernel forms ‖r_c‖∞ = max(max r − μ_r, μ_r − min r) and the same for
// f, compares with rtol and sets the convergence flag that makes every later
// kernel of the solve return at once.
#include "internal.h"

namespace ps {

enum { END_WRAP = 0, END_N = 1, END_D = 2 };
constexpr int RTX = 32, RTY = 8;

__device__ __forceinline__ int end_lo(int bc) { return bc == BC_P ? END_WRAP : (bc == BC_DD ? END_D : END_N); }
__device__ __forceinline__ int end_hi(int bc) { return bc == BC_P ? END_WRAP : ((bc == BC_DD || bc == BC_ND) ? END_D : END_N); }

// (a + b) − 2c as an unevaluated double-float (two TwoSums on the high parts)
__device__ __forceinline__ df second_diff(df a, df b, df c) {
  df s1 = two_sum(a.h, b.h);
  df s2 = two_sum(s1.h, -2.f * c.h);
  return {s2.h, s1.l + s2.l + (a.l + b.l - 2.f * c.l)};
}
// b − c as an unevaluated double-float
__device__ __forceinline__ df diff(df b, df c) {
  df s = two_sum(b.h, -c.h);
  return {s.h, s.l + (b.l - c.l)};
}
// s · w (w a double-float coefficient), unevaluated
__device__ __forceinline__ df mul_coef(df s, df w) {
  const float p = __fmul_rn(s.h, w.h);
  float e = __fmaf_rn(s.h, w.h, -p);
  e = __fmaf_rn(s.l, w.h, __fmaf_rn(s.h, w.l, e));
  return {p, e};
}
// unevaluated double-float sum
__device__ __forceinline__ df add_u(df a, df b) {
  df s = two_sum(a.h, b.h);
  return {s.h, s.l + a.l + b.l};
}

__device__ __forceinline__ df ld_df(const double* p) { return df_from_f64(__ldg(p)); }

__global__ void __launch_bounds__(RTX * RTY) residual_kernel(ResidArgs a) {
  if (a.skip && *a.skip) return;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t sxy = (size_t)nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * RTX + tx, j = blockIdx.y * RTY + ty;
  const bool in = (i < nx) && (j < ny);
  const int k0 = blockIdx.z * a.zchunk, k1 = min(nz, k0 + a.zchunk);
  const int xl = end_lo(a.bcx), xh = end_hi(a.bcx);
  const int yl = end_lo(a.bcy), yh = end_hi(a.bcy);
  const int zl = end_lo(a.bcz), zh = end_hi(a.bcz);
  __shared__ df sp[2][RTY + 2][RTX + 2];
  // column of this thread (clamped inside the domain)
  const int ic = min(i, nx - 1), jc = min(j, ny - 1);
  const size_t col = (size_t)jc * nx + ic;
  // halo columns / rows loaded by edge threads (periodic wrap; the N/D ends are
  // resolved in the arithmetic, so their halo value is never used)
  const bool hx_lo = (tx == 0), hx_hi = (tx == RTX - 1) || (i == nx - 1);
  const bool hy_lo = (ty == 0), hy_hi = (ty == RTY - 1) || (j == ny - 1);
  const int ixl = (ic > 0) ? ic - 1 : nx - 1, ixh = (ic < nx - 1) ? ic + 1 : 0;
  const int jyl = (jc > 0) ? jc - 1 : ny - 1, jyh = (jc < ny - 1) ? jc + 1 : 0;
  const size_t cxl = (size_t)jc * nx + ixl, cxh = (size_t)jc * nx + ixh;
  const size_t cyl = (size_t)jyl * nx + ic, cyh = (size_t)jyh * nx + ic;

  const int km = (k0 > 0) ? k0 - 1 : nz - 1;
  df pm = ld_df(a.p + (size_t)km * sxy + col);
  df pc = ld_df(a.p + (size_t)k0 * sxy + col);
  float rmax = -INFINITY, rmin = INFINITY, fmax_ = -INFINITY, fmin_ = INFINITY;
  df wr = {0.f, 0.f}, wf = {0.f, 0.f};
  const df mu = a.singular ? df{a.mu[0], a.mu[1]} : df{0.f, 0.f};

  for (int k = k0; k < k1; ++k) {
    const int b = k & 1;
    const size_t plane = (size_t)k * sxy;
    // this plane into shared memory (centre + halos)
    // (only in-domain threads write: every cell an in-domain thread reads is
    // written by an in-domain thread, and out-of-domain clamped copies would race)
    if (in) {
      sp[b][ty + 1][tx + 1] = pc;
      if (hx_lo) sp[b][ty + 1][tx] = ld_df(a.p + plane + cxl);
      if (hx_hi) sp[b][ty + 1][tx + 2] = ld_df(a.p + plane + cxh);
      if (hy_lo) sp[b][ty][tx + 1] = ld_df(a.p + plane + cyl);
      if (hy_hi) sp[b][ty + 2][tx + 1] = ld_df(a.p + plane + cyh);
    }
    // next plane and f while the shared plane settles
    const int kp = (k + 1 < nz) ? k + 1 : 0;
    const df pp = ld_df(a.p + (size_t)kp * sxy + col);
    const df fv = ld_df(a.f + plane + col);
    __syncthreads();
    df xm = sp[b][ty + 1][tx], xp = sp[b][ty + 1][tx + 2];
    df ym = sp[b][ty][tx + 1], yp = sp[b][ty + 2][tx + 1];
    const df nc = {-pc.h, -pc.l};
    if (i == 0 && xl != END_WRAP) xm = (xl == END_N) ? pc : nc;
    if (i == nx - 1 && xh != END_WRAP) xp = (xh == END_N) ? pc : nc;
    if (j == 0 && yl != END_WRAP) ym = (yl == END_N) ? pc : nc;
    if (j == ny - 1 && yh != END_WRAP) yp = (yh == END_N) ? pc : nc;
    df zm = pm, zp = pp;
    if (k == 0 && zl != END_WRAP) zm = (zl == END_N) ? pc : nc;
    if (k == nz - 1 && zh != END_WRAP) zp = (zh == END_N) ? pc : nc;
    const df tx2 = mul_coef(second_diff(xm, xp, pc), a.idx2);
    const df ty2 = mul_coef(second_diff(ym, yp, pc), a.idy2);
    const float2 cl = a.zlo[k], ch = a.zhi[k];
    const df tz = add_u(mul_coef(diff(zm, pc), df{cl.x, cl.y}), mul_coef(diff(zp, pc), df{ch.x, ch.y}));
    const df ap = add_u(add_u(tx2, ty2), tz);
    const df r = add_u(add_u(fv, df{-mu.h, -mu.l}), df{-ap.h, -ap.l});
    const float rf = r.h + r.l;
    if (in) {
      if (a.r) a.r[plane + col] = rf;
      const float ff = fv.h + fv.l;
      rmax = fmaxf(rmax, rf);
      rmin = fminf(rmin, rf);
      fmax_ = fmaxf(fmax_, ff);
      fmin_ = fminf(fmin_, ff);
      if (a.singular) {
        const df w = {a.wz[k], 0.f};
        wr = add_u(wr, mul_coef(r, w));
        wf = add_u(wf, mul_coef(fv, w));
      }
    }
    pm = pc;
    pc = pp;
  }

  // block reductions: warp shuffles, then one thread over the warps
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rmax = fmaxf(rmax, __shfl_xor_sync(full, rmax, o));
    rmin = fminf(rmin, __shfl_xor_sync(full, rmin, o));
    fmax_ = fmaxf(fmax_, __shfl_xor_sync(full, fmax_, o));
    fmin_ = fminf(fmin_, __shfl_xor_sync(full, fmin_, o));
    wr = add_u(wr, df{__shfl_xor_sync(full, wr.h, o), __shfl_xor_sync(full, wr.l, o)});
    wf = add_u(wf, df{__shfl_xor_sync(full, wf.h, o), __shfl_xor_sync(full, wf.l, o)});
  }
  __shared__ float red[RTY][8];
  if (tx == 0) {
    red[ty][0] = rmax; red[ty][1] = rmin; red[ty][2] = fmax_; red[ty][3] = fmin_;
    red[ty][4] = wr.h; red[ty][5] = wr.l; red[ty][6] = wf.h; red[ty][7] = wf.l;
  }
  __syncthreads();
  if (ty == 0 && tx == 0) {
    for (int w = 1; w < RTY; ++w) {
      rmax = fmaxf(rmax, red[w][0]);
      rmin = fminf(rmin, red[w][1]);
      fmax_ = fmaxf(fmax_, red[w][2]);
      fmin_ = fminf(fmin_, red[w][3]);
      wr = add_u(wr, df{red[w][4], red[w][5]});
      wf = add_u(wf, df{red[w][6], red[w][7]});
    }
    atomicMax(&a.red[0], f32_key(rmax));
    atomicMin(&a.red[1], f32_key(rmin));
    atomicMax(&a.red[2], f32_key(fmax_));
    atomicMin(&a.red[3], f32_key(fmin_));
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    reinterpret_cast<float4*>(a.partial)[bid] = make_float4(wr.h, wr.l, wf.h, wf.l);
  }
}

// Resets the reduction words before a residual pass.
__global__ void reset_red_kernel(int* red, const int* skip) {
  if (skip && *skip) return;
  red[0] = f32_key(-INFINITY);
  red[1] = f32_key(INFINITY);
  red[2] = f32_key(-INFINITY);
  red[3] = f32_key(INFINITY);
}

int residual_blocks(int nx, int ny, int nz) {
  const int zc = nz < 32 ? nz : 32;
  return ((nx + RTX - 1) / RTX) * ((ny + RTY - 1) / RTY) * ((nz + zc - 1) / zc);
}

cudaError_t launch_residual(const ResidArgs& a, cudaStream_t st) {
  reset_red_kernel<<<1, 1, 0, st>>>(a.red, a.skip);
  ResidArgs b = a;
  b.zchunk = a.nz < 32 ? a.nz : 32;
  const dim3 grid((a.nx + RTX - 1) / RTX, (a.ny + RTY - 1) / RTY, (a.nz + b.zchunk - 1) / b.zchunk);
  residual_kernel<<<grid, dim3(RTX, RTY), 0, st>>>(b);
  return cudaGetLastError();
}

// One CTA: weighted means (singular), norms, convergence test, info record.
__global__ void __launch_bounds__(1024) finalize_kernel(Ctrl* c, const float* partial, int nblocks,
                                                        double wsum_total, int singular, double rtol,
                                                        int iteration, int last, ps_info* info) {
  if (c->converged) return;
  __shared__ df sr[32], sf[32];
  if (singular) {
    df ar = {0.f, 0.f}, af = {0.f, 0.f};
    const float4* pv = reinterpret_cast<const float4*>(partial);
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      const float4 v = pv[b];
      ar = add_u(ar, df{v.x, v.y});
      af = add_u(af, df{v.z, v.w});
    }
    for (int o = 16; o > 0; o >>= 1) {
      ar = add_u(ar, df{__shfl_xor_sync(0xffffffffu, ar.h, o), __shfl_xor_sync(0xffffffffu, ar.l, o)});
      af = add_u(af, df{__shfl_xor_sync(0xffffffffu, af.h, o), __shfl_xor_sync(0xffffffffu, af.l, o)});
    }
    if ((threadIdx.x & 31) == 0) {
      sr[threadIdx.x >> 5] = ar;
      sf[threadIdx.x >> 5] = af;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double mr = 0.0, mf = 0.0;
  if (singular) {
    double s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s1 += (double)sr[w].h + (double)sr[w].l;
      s2 += (double)sf[w].h + (double)sf[w].l;
    }
    mr = s1 / wsum_total;
    mf = s2 / wsum_total;
    if (iteration == 0) {
      const float h = (float)mf;
      c->mu[0] = h;
      c->mu[1] = (float)(mf - (double)h);
    }
  }
  const double rmax = key_f32(c->red[0]), rmin = key_f32(c->red[1]);
  const double vfmax = key_f32(c->red[2]), vfmin = key_f32(c->red[3]);
  const double rn = fmax(rmax - mr, mr - rmin);
  const double fn = fmax(vfmax - mf, mf - vfmin);  // f's sums are of the raw f
  const double rel = fn > 0 ? rn / fn : (rn > 0 ? INFINITY : 0.0);
  c->rnorm = rn;
  c->fnorm = fn;
  c->rel = rel;
  c->iterations = iteration;
  const bool ok = rel <= rtol;
  if (ok) c->converged = 1;
  if (info && (ok || last)) {
    info->status = ok ? PS_OK : PS_NOT_CONVERGED;
    info->iterations = iteration;
    info->rel_residual = rel;
    info->r_norm = rn;
    info->f_norm = fn;
  }
}

cudaError_t launch_finalize(Ctrl* ctrl, const float* partial, int nblocks, double wsum_total,
                            int singular, double rtol, int iteration, int last, ps_info* info,
                            cudaStream_t st) {
  finalize_kernel<<<1, 1024, 0, st>>>(ctrl, partial, nblocks, wsum_total, singular, rtol, iteration,
                                      last, info);
  return cudaGetLastError();
}

__global__ void info_plain_kernel(ps_info* info) {
  info->status = PS_OK;
  info->iterations = 0;
  info->rel_residual = -1.0;
  info->r_norm = -1.0;
  info->f_norm = -1.0;
}

cudaError_t launch_info_plain(ps_info* info, cudaStream_t st) {
  info_plain_kernel<<<1, 1, 0, st>>>(info);
  return cudaGetLastError();
}

}  // namespace ps
