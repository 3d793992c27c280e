// residual.cu — r = f − A·Φ (Eq. 4) for the iterative refinement, in double-float.
//
// Φ and f are FP64 fields. FP64 arithmetic and f64<->f32 conversions issue at
// ~1/64 of the FP32 rate on this part, so each value is split on its bit pattern
// into hi + lo floats (48 significant bits) and the 7-point stencil is evaluated
// with error-free transformations (TwoSum, FMA products). The residual is
// rounded once to FP32 (the right-hand side of the next FP32 correction solve).
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

__device__ __forceinline__ df nb_diff(int kind, const double* q, bool inner, df pc) {
  // (neighbour − Φ_c) with the ghost rule for the end; q points at the neighbour
  if (inner || kind == END_WRAP) return df_sub(df_from_f64(*q), pc);
  if (kind == END_N) return df{0.f, 0.f};
  return df{-2.f * pc.h, -2.f * pc.l};  // Dirichlet: ghost = −Φ_c
}

__device__ __forceinline__ int end_lo(int bc) { return bc == BC_P ? END_WRAP : (bc == BC_DD ? END_D : END_N); }
__device__ __forceinline__ int end_hi(int bc) { return bc == BC_P ? END_WRAP : ((bc == BC_DD || bc == BC_ND) ? END_D : END_N); }

__global__ void __launch_bounds__(256) residual_kernel(ResidArgs a) {
  if (a.skip && *a.skip) return;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t N = (size_t)nx * ny * nz;
  const size_t sxy = (size_t)nx * ny;
  const int xl = end_lo(a.bcx), xh = end_hi(a.bcx);
  const int yl = end_lo(a.bcy), yh = end_hi(a.bcy);
  const int zl = end_lo(a.bcz), zh = end_hi(a.bcz);
  float rmax = -INFINITY, rmin = INFINITY, fmax = -INFINITY, fmin = INFINITY;
  df wr = {0.f, 0.f}, wf = {0.f, 0.f};
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(g % nx);
    const size_t t = g / nx;
    const int j = (int)(t % ny);
    const int k = (int)(t / ny);
    const double* pp = a.p + g;
    const df pc = df_from_f64(*pp);
    // x
    df dxm = nb_diff(xl, (i > 0) ? pp - 1 : pp + (nx - 1), i > 0, pc);
    df dxp = nb_diff(xh, (i < nx - 1) ? pp + 1 : pp - (nx - 1), i < nx - 1, pc);
    df tx = df_mul(df_add(dxm, dxp), a.idx2);
    // y
    df dym = nb_diff(yl, (j > 0) ? pp - nx : pp + (size_t)(ny - 1) * nx, j > 0, pc);
    df dyp = nb_diff(yh, (j < ny - 1) ? pp + nx : pp - (size_t)(ny - 1) * nx, j < ny - 1, pc);
    df ty = df_mul(df_add(dym, dyp), a.idy2);
    // z (stretched): zlo[k]·(Φ_{k−1} − Φ_k) + zhi[k]·(Φ_{k+1} − Φ_k)
    df dzm = nb_diff(zl, (k > 0) ? pp - sxy : pp + (size_t)(nz - 1) * sxy, k > 0, pc);
    df dzp = nb_diff(zh, (k < nz - 1) ? pp + sxy : pp - (size_t)(nz - 1) * sxy, k < nz - 1, pc);
    const float2 cl = a.zlo[k], ch = a.zhi[k];
    df tz = df_add(df_mul(dzm, df{cl.x, cl.y}), df_mul(dzp, df{ch.x, ch.y}));
    df ap = df_add(df_add(tx, ty), tz);
    df fv = df_from_f64(a.f[g]);
    // singular problems: r_c = (f − μ_f) − A·Φ, so that the FP32 rounding of r is
    // relative to its compatible part, not to the (possibly large) mean of f
    df r = a.singular ? df_sub(df_sub(fv, df{a.mu[0], a.mu[1]}), ap) : df_sub(fv, ap);
    const float rf = df_to_f32(r);
    if (a.r) a.r[g] = rf;
    const float ff = df_to_f32(fv);
    rmax = fmaxf(rmax, rf);
    rmin = fminf(rmin, rf);
    fmax = fmaxf(fmax, ff);
    fmin = fminf(fmin, ff);
    if (a.singular) {
      const df w = {a.wz[k], 0.f};
      wr = df_add(wr, df_mul(r, w));
      wf = df_add(wf, df_mul(fv, w));
    }
  }
  // block reductions
  __shared__ float s4[4][256];
  __shared__ df s2[2][256];
  s4[0][threadIdx.x] = rmax;
  s4[1][threadIdx.x] = rmin;
  s4[2][threadIdx.x] = fmax;
  s4[3][threadIdx.x] = fmin;
  s2[0][threadIdx.x] = wr;
  s2[1][threadIdx.x] = wf;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s4[0][threadIdx.x] = fmaxf(s4[0][threadIdx.x], s4[0][threadIdx.x + w]);
      s4[1][threadIdx.x] = fminf(s4[1][threadIdx.x], s4[1][threadIdx.x + w]);
      s4[2][threadIdx.x] = fmaxf(s4[2][threadIdx.x], s4[2][threadIdx.x + w]);
      s4[3][threadIdx.x] = fminf(s4[3][threadIdx.x], s4[3][threadIdx.x + w]);
      s2[0][threadIdx.x] = df_add(s2[0][threadIdx.x], s2[0][threadIdx.x + w]);
      s2[1][threadIdx.x] = df_add(s2[1][threadIdx.x], s2[1][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicMax(&a.red[0], f32_key(s4[0][0]));
    atomicMin(&a.red[1], f32_key(s4[1][0]));
    atomicMax(&a.red[2], f32_key(s4[2][0]));
    atomicMin(&a.red[3], f32_key(s4[3][0]));
    float* pb = a.partial + 4 * blockIdx.x;
    pb[0] = s2[0][0].h;
    pb[1] = s2[0][0].l;
    pb[2] = s2[1][0].h;
    pb[3] = s2[1][0].l;
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

cudaError_t launch_residual(const ResidArgs& a, cudaStream_t st) {
  reset_red_kernel<<<1, 1, 0, st>>>(a.red, a.skip);
  residual_kernel<<<a.nblocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// One thread: weighted means (singular), norms, convergence test, info record.
__global__ void finalize_kernel(Ctrl* c, const float* partial, int nblocks, double wsum_total,
                                int singular, double rtol, int iteration, int last, ps_info* info) {
  if (c->converged) return;
  double mr = 0.0, mf = 0.0;
  if (singular) {
    double sr = 0.0, sf = 0.0;
    for (int b = 0; b < nblocks; ++b) {
      sr += (double)partial[4 * b] + (double)partial[4 * b + 1];
      sf += (double)partial[4 * b + 2] + (double)partial[4 * b + 3];
    }
    mr = sr / wsum_total;
    mf = sf / wsum_total;
    if (iteration == 0) {
      const float h = (float)mf;
      c->mu[0] = h;
      c->mu[1] = (float)(mf - (double)h);
    }
  }
  const double rmax = key_f32(c->red[0]), rmin = key_f32(c->red[1]);
  const double vfmax = key_f32(c->red[2]), vfmin = key_f32(c->red[3]);
  const double rn = fmax(rmax - mr, mr - rmin);
  const double fn = fmax(vfmax - mf, mf - vfmin);
  const double rel = fn > 0 ? rn / fn : (rn > 0 ? INFINITY : 0.0);
  c->rnorm = rn;
  c->fnorm = fn;  // f's own sums are of the raw f, so μ_f is measured afresh each pass
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
  finalize_kernel<<<1, 1, 0, st>>>(ctrl, partial, nblocks, wsum_total, singular, rtol, iteration,
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
