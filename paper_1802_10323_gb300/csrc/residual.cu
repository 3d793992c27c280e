// residual.cu — r = f − A·Φ (Eq. 4) for the iterative refinement, in double-float.
//
// Φ and f are FP64 fields. FP64 arithmetic and f64<->f32 conversions issue at
// ~1/64 of the FP32 rate on this part, so each value is split on its bit pattern
// into hi + lo floats (48 significant bits) and the 7-point stencil is evaluated
// with error-free transformations (TwoSum, FMA products). The residual is
// rounded once to FP32 (the right-hand side of the next FP32 correction solve).
//
// Splitting: Φ = ph + pl with ph on a fixed-point grid 2^−s common to the whole
// field (s from max|Φ|, so |ph|·2^s < 2^20): the stencil sums of ph are exact
// in FP32, the four products with the double-float coefficients are made exact
// with FMA, and the small pl part only needs FP32. f is split into hi + lo.
//
// Blocking: a CTA of 32 × 8 threads owns a 32 × 8 (x, y) tile and marches along
// z over a chunk of planes. Raw FP64 planes of Φ (tile plus one halo cell per
// side, periodic wrap resolved in the addresses) and of f stream into a
// six-stage shared-memory ring with cp.async, up to four planes ahead of the one
// being computed; each Φ value is split once into a three-plane ring of fixed-point
// pairs from which the 7-point stencil reads all its neighbours.
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

// unevaluated double-float sum
__device__ __forceinline__ df add_u(df a, df b) {
  df s = two_sum(a.h, b.h);
  return {s.h, s.l + a.l + b.l};
}

// Φ on a fixed-point grid: ph = rint(Φ·2^s)·2^−s (|Φ·2^s| < 2^20 for every Φ of
// the field, so sums and differences of a few ph are exact in FP32) and
// pl = Φ − ph rounded to FP32 (|pl| ≤ 2^−s−1). A·ph is then exact up to the
// coefficient products, and A·pl only needs FP32.
struct fxp {
  float h, l;
};
__device__ __forceinline__ fxp to_fxp(double d, float S, float iS) {
  float h, l;
  split_f64(d, h, l);
  const float ph = __fmul_rn(rintf(__fmul_rn(h, S)), iS);
  return {ph, __fadd_rn(__fsub_rn(h, ph), l)};
}
// exact product of an FP32 value and a double-float coefficient, unevaluated
__device__ __forceinline__ df prod(float x, df w) {
  const float p = __fmul_rn(x, w.h);
  return {p, __fmaf_rn(x, w.l, __fmaf_rn(x, w.h, -p))};
}

// 8-byte asynchronous global→shared copy; a zero source size fills zeros and
// reads nothing (used for cells outside the domain).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem),
               "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

constexpr int RW = RTX + 2, RH = RTY + 2;  // tile with one halo cell per side
constexpr int RECT = RW * RH;               // 340 cells
constexpr int NSTG = 6;                     // raw planes in flight (ring)

__global__ void __launch_bounds__(RTX * RTY) residual_kernel(ResidArgs a) {
  if (a.skip && *a.skip) return;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t sxy = (size_t)nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RTX + tx;
  const int x0 = blockIdx.x * RTX, y0 = blockIdx.y * RTY;
  const int i = x0 + tx, j = y0 + ty;
  const bool in = (i < nx) && (j < ny);
  const int k0 = blockIdx.z * a.zchunk, k1 = min(nz, k0 + a.zchunk);
  const int xl = end_lo(a.bcx), xh = end_hi(a.bcx);
  const int yl = end_lo(a.bcy), yh = end_hi(a.bcy);
  const int zl = end_lo(a.bcz), zh = end_hi(a.bcz);
  const bool perz = (a.bcz == BC_P);
  float S, iS;
  {
    const int e = (int)((*a.pmax_bits >> 52) & 0x7FF) - 1023;  // max|Φ| ∈ [2^e, 2^(e+1))
    int sc = max(-100, min(100, 19 - e));
    S = __uint_as_float((uint32_t)(sc + 127) << 23);
    iS = __uint_as_float((uint32_t)(127 - sc) << 23);
  }
  __shared__ __align__(16) double rawp[NSTG][RECT];   // Φ tile + halo, by plane
  __shared__ __align__(16) double rawf[NSTG][RTY * RTX];  // f tile, by plane
  __shared__ fxp fx[3][RECT];                         // split Φ planes k−1, k, k+1
  const double* __restrict__ P = a.p;
  const double* __restrict__ F = a.f;

  // the (up to) two halo-rectangle cells this thread copies and converts
  int rc_off[2];
  bool rc_ok[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = tid + h * (RTX * RTY);
    const int rr = e / RW, cc = e - rr * RW;
    int gi = x0 - 1 + cc, gj = y0 - 1 + rr;
    bool ok = e < RECT && !((rr == 0 || rr == RH - 1) && (cc == 0 || cc == RW - 1));
    if (gi < 0) { if (a.bcx == BC_P) gi += nx; else ok = false; }
    if (gi >= nx) { if (a.bcx == BC_P && gi - nx < nx && x0 + RTX >= nx) gi -= nx; else ok = false; }
    if (gj < 0) { if (a.bcy == BC_P) gj += ny; else ok = false; }
    if (gj >= ny) { if (a.bcy == BC_P && gj - ny < ny && y0 + RTY >= ny) gj -= ny; else ok = false; }
    rc_ok[h] = ok;
    rc_off[h] = ok ? gj * nx + gi : 0;
  }
  auto plane_of = [&](int q) {  // source plane of logical plane q (wrap or clamp)
    if (q < 0) return perz ? q + nz : 0;
    if (q >= nz) return perz ? q - nz : nz - 1;
    return q;
  };
  auto issue = [&](int q) {  // raw loads of logical plane q into its ring slot
    const int slot = (q - k0 + 1) % NSTG;
    const size_t pl = (size_t)plane_of(q) * sxy;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + h * (RTX * RTY);
      if (e < RECT) cp_async8(&rawp[slot][e], P + pl + rc_off[h], rc_ok[h]);
    }
    const size_t fo = in ? (size_t)j * nx + i : 0;
    cp_async8(&rawf[slot][tid], F + pl + fo, in && q >= 0 && q < nz);
    cp_commit();
  };
  auto convert = [&](int q) {  // split raw plane q into fx[(q − k0 + 1) % 3]
    const int slot = (q - k0 + 1) % NSTG, fs = (q - k0 + 1) % 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + h * (RTX * RTY);
      if (e < RECT) fx[fs][e] = to_fxp(rawp[slot][e], S, iS);
    }
  };

  // prologue: planes k0−1 … k0+NSTG−2 in flight; convert k0−1 and k0
#pragma unroll
  for (int q = 0; q < NSTG - 1; ++q) issue(k0 - 1 + q);
  cp_wait<NSTG - 3>();
  __syncthreads();
  convert(k0 - 1);
  convert(k0);

  float rmax = -INFINITY, rmin = INFINITY, fmax_ = -INFINITY, fmin_ = INFINITY;
  float wr = 0.f;
  df wf = {0.f, 0.f};
  const bool first = a.singular && a.first;
  const df mu = a.singular ? df{a.mu[0], a.mu[1]} : df{0.f, 0.f};
  const int c = (ty + 1) * RW + (tx + 1);  // this thread's cell in the rectangle

  for (int k = k0; k < k1; ++k) {
    // keep NSTG−1 planes in flight (an empty group keeps the wait count uniform)
    if (k + NSTG - 2 <= k1) issue(k + NSTG - 2);
    else cp_commit();
    cp_wait<NSTG - 3>();  // plane k+1 has landed (planes k+2 … k+NSTG−2 may be pending)
    __syncthreads();
    convert(k + 1);
    __syncthreads();
    const fxp* Pm = fx[(k - k0) % 3];
    const fxp* Pc = fx[(k - k0 + 1) % 3];
    const fxp* Pp = fx[(k - k0 + 2) % 3];
    const fxp pc = Pc[c];
    fxp xm = Pc[c - 1], xp = Pc[c + 1], ym = Pc[c - RW], yp = Pc[c + RW];
    fxp zm = Pm[c], zp = Pp[c];
    const fxp nc = {-pc.h, -pc.l};
    if (i == 0 && xl != END_WRAP) xm = (xl == END_N) ? pc : nc;
    if (i == nx - 1 && xh != END_WRAP) xp = (xh == END_N) ? pc : nc;
    if (j == 0 && yl != END_WRAP) ym = (yl == END_N) ? pc : nc;
    if (j == ny - 1 && yh != END_WRAP) yp = (yh == END_N) ? pc : nc;
    if (k == 0 && zl != END_WRAP) zm = (zl == END_N) ? pc : nc;
    if (k == nz - 1 && zh != END_WRAP) zp = (zh == END_N) ? pc : nc;
    const df fv = df_from_f64(rawf[(k - k0 + 1) % NSTG][tid]);
    // exact high-part stencil sums (fixed-point grid), FP32 low parts
    const float sx = (xm.h + xp.h) - 2.f * pc.h, sy = (ym.h + yp.h) - 2.f * pc.h;
    const float dm = zm.h - pc.h, dpz = zp.h - pc.h;
    const float lx = (xm.l + xp.l) - 2.f * pc.l, ly = (ym.l + yp.l) - 2.f * pc.l;
    const float2 cl = a.zlo[k], ch = a.zhi[k];
    const float lo_terms = lx * a.idx2.h + ly * a.idy2.h + cl.x * (zm.l - pc.l) + ch.x * (zp.l - pc.l);
    const df t1 = prod(sx, a.idx2), t2 = prod(sy, a.idy2);
    const df t3 = prod(dm, df{cl.x, cl.y}), t4 = prod(dpz, df{ch.x, ch.y});
    const df s12 = two_sum(t1.h, t2.h);
    const df s123 = two_sum(s12.h, t3.h);
    const df s1234 = two_sum(s123.h, t4.h);
    const float ap_lo = ((s12.l + s123.l) + (s1234.l + t1.l)) + ((t2.l + t3.l) + (t4.l + lo_terms));
    df r;
    if (a.singular) {
      const df d1 = two_sum(fv.h, -mu.h);
      const df d2 = two_sum(d1.h, -s1234.h);
      r = {d2.h, ((d1.l + d2.l) + (fv.l - mu.l)) - ap_lo};
    } else {
      const df d2 = two_sum(fv.h, -s1234.h);
      r = {d2.h, (d2.l + fv.l) - ap_lo};
    }
    const float rf = r.h + r.l;
    if (in) {
      const size_t g = (size_t)k * sxy + (size_t)j * nx + i;
      if (a.r) a.r[g] = rf;
      const float ff = fv.h + fv.l;
      rmax = fmaxf(rmax, rf);
      rmin = fminf(rmin, rf);
      fmax_ = fmaxf(fmax_, ff);
      fmin_ = fminf(fmin_, ff);
      if (a.singular) {
        const float w = a.wz[k];
        wr = fmaf(w, rf, wr);
        if (first) {  // Σ Δz^f·f in double-float (only the first pass needs μ_f)
          wf = add_u(wf, prod(fv.h, df{w, 0.f}));
          wf.l = fmaf(w, fv.l, wf.l);
        }
      }
    }
  }
  cp_wait<0>();

  // block reductions: warp shuffles, then one thread over the warps
  const unsigned full = 0xffffffffu;
  df wrd = {wr, 0.f};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rmax = fmaxf(rmax, __shfl_xor_sync(full, rmax, o));
    rmin = fminf(rmin, __shfl_xor_sync(full, rmin, o));
    fmax_ = fmaxf(fmax_, __shfl_xor_sync(full, fmax_, o));
    fmin_ = fminf(fmin_, __shfl_xor_sync(full, fmin_, o));
    wrd = add_u(wrd, df{__shfl_xor_sync(full, wrd.h, o), __shfl_xor_sync(full, wrd.l, o)});
    wf = add_u(wf, df{__shfl_xor_sync(full, wf.h, o), __shfl_xor_sync(full, wf.l, o)});
  }
  __shared__ float red[RTY][8];
  if (tx == 0) {
    red[ty][0] = rmax; red[ty][1] = rmin; red[ty][2] = fmax_; red[ty][3] = fmin_;
    red[ty][4] = wrd.h; red[ty][5] = wrd.l; red[ty][6] = wf.h; red[ty][7] = wf.l;
  }
  __syncthreads();
  if (ty == 0 && tx == 0) {
    for (int w = 1; w < RTY; ++w) {
      rmax = fmaxf(rmax, red[w][0]);
      rmin = fminf(rmin, red[w][1]);
      fmax_ = fmaxf(fmax_, red[w][2]);
      fmin_ = fminf(fmin_, red[w][3]);
      wrd = add_u(wrd, df{red[w][4], red[w][5]});
      wf = add_u(wf, df{red[w][6], red[w][7]});
    }
    atomicMax(&a.red[0], f32_key(rmax));
    atomicMin(&a.red[1], f32_key(rmin));
    atomicMax(&a.red[2], f32_key(fmax_));
    atomicMin(&a.red[3], f32_key(fmin_));
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    reinterpret_cast<float4*>(a.partial)[bid] = make_float4(wrd.h, wrd.l, wf.h, wf.l);
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
    if (iteration == 0) {  // μ_f is measured once, on the first pass
      mf = s2 / wsum_total;
      c->mf = mf;
      const float h = (float)mf;
      c->mu[0] = h;
      c->mu[1] = (float)(mf - (double)h);
    } else {
      mf = c->mf;
    }
  }
  const double rmax = key_f32(c->red[0]), rmin = key_f32(c->red[1]);
  const double vfmax = key_f32(c->red[2]), vfmin = key_f32(c->red[3]);
  const double rn = fmax(rmax - mr, mr - rmin);
  const double fn = fmax(vfmax - mf, mf - vfmin);
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
