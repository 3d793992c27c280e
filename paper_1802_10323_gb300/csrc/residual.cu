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
// Blocking: a CTA of 32 × 8 threads owns a 32 × (8·RPT) (x, y) tile and
// marches along z over a chunk of planes; each thread computes RPT consecutive
// rows of one x column. Raw FP64 planes of Φ (tile plus one halo cell per side)
// stream into a shared-memory ring with cp.async, RDEPTH − 2 planes ahead of
// the one being split; each plane is split once into fixed-point pairs (two
// plane slots), from which the in-plane neighbours are read. The z neighbours
// of a thread's own cells stay in registers (planes k−1, k, k+1), and f streams
// through registers one plane ahead with plain loads. The kernel is bound by
// instruction issue rather than bytes, so the per-plane work that does not
// scale with the points (ring control, barriers, coefficient loads) is shared
// by RPT points and the ring slots advance by counters, not by division.
//
// Ends of each axis (staggered ghost rules of Table 1) are folded into the halo
// load: a periodic end wraps; a Neumann end loads the adjacent interior cell
// (ghost = Φ, so its term vanishes); a Dirichlet end loads it with the sign
// flipped (ghost = −Φ, term coef·(−2Φ)). In z the same holds for the ghost
// planes below k = 0 and above k = n_z − 1, and the coefficients zlo/zhi hold
// a_k, c_k, the wrap couplings, or 1/(Δz^f)² at a Dirichlet end.
//
// Reductions per pass (deterministic): max and min of r and of f (order-
// preserving integer keys, atomicMax/atomicMin), and, for singular problems,
// per-block double-float sums of Δz^f·r and Δz^f·f for the weighted means. The
// finalize kernel forms ‖r_c‖∞ = max(max r − μ_r, μ_r − min r) and the same for
// f, compares with rtol and sets the convergence flag that makes every later
// kernel of the solve return at once.
#include <type_traits>

#include "internal.h"

namespace ps {

enum { END_WRAP = 0, END_N = 1, END_D = 2 };
constexpr int RTX = 32, RWARPS = 8, RTHREADS = RTX * RWARPS;
constexpr int RDEPTH = 4;  // raw-plane ring: k+1 being split, k+2 … k+3 in flight

__host__ __device__ constexpr int resid_cells(int rpt) { return (RTX + 2) * (RWARPS * rpt + 2); }
__host__ __device__ constexpr size_t resid_smem(int rpt) {
  return (size_t)(RDEPTH + 2) * resid_cells(rpt) * sizeof(double);
}

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
__device__ __forceinline__ double flip_sign(double d, uint32_t sgn) {
  return __hiloint2double(__double2hiint(d) ^ (int)sgn, __double2loint(d));
}

// 8-byte asynchronous global→shared copy; a zero source size fills zeros and
// reads nothing (used for cells that no in-domain point needs).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem),
               "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// MODE: 0 non-singular; 1 singular (subtract μ_f, weighted sum of r); 2 the
// singular problem's first pass (also the weighted sum of f that gives μ_f).
template <int RPT, int MODE>
__global__ void __launch_bounds__(RTHREADS, RPT >= 4 ? 3 : 4) residual_kernel(ResidArgs a) {
  constexpr bool SING = MODE >= 1, FIRST = MODE == 2;
  constexpr int TY = RWARPS * RPT, W = RTX + 2, CELLS = resid_cells(RPT);
  constexpr int CPT = (CELLS + RTHREADS - 1) / RTHREADS;  // halo cells per thread
  if (a.skip && *a.skip) return;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t sxy = (size_t)nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RTX + tx;
  const int x0 = blockIdx.x * RTX, y0 = blockIdx.y * TY;
  const int i = x0 + tx, jb = y0 + ty * RPT;  // rows jb … jb+RPT−1 of column i
  const int k0 = blockIdx.z * a.zchunk, k1 = min(nz, k0 + a.zchunk);
  const bool perz = (a.bcz == BC_P);
  const uint32_t zsg_lo = end_lo(a.bcz) == END_D ? 0x80000000u : 0u;
  const uint32_t zsg_hi = end_hi(a.bcz) == END_D ? 0x80000000u : 0u;
  float S, iS;
  {
    const int e = (int)((*a.pmax_bits >> 52) & 0x7FF) - 1023;  // max|Φ| ∈ [2^e, 2^(e+1))
    const int sc = max(-100, min(100, 19 - e));
    S = __uint_as_float((uint32_t)(sc + 127) << 23);
    iS = __uint_as_float((uint32_t)(127 - sc) << 23);
  }
  extern __shared__ __align__(16) double rsm[];
  double* raw = rsm;                                       // [RDEPTH][CELLS] raw Φ planes
  fxp* fx = reinterpret_cast<fxp*>(rsm + RDEPTH * CELLS);  // [2][CELLS] split planes
  const double* __restrict__ P = a.p;
  const double* __restrict__ F = a.f;

  // The halo-rectangle cells this thread copies and splits: in-plane offset of
  // the source cell, and per-cell bits "copy" and "flip sign" (Dirichlet ghost).
  int off[CPT];
  uint32_t okm = 0, negm = 0;
  {
    const int xl = end_lo(a.bcx), xh = end_hi(a.bcx), yl = end_lo(a.bcy), yh = end_hi(a.bcy);
#pragma unroll
    for (int h = 0; h < CPT; ++h) {
      const int e = tid + h * RTHREADS;
      const int rr = e / W, cc = e - rr * W;
      int gi = x0 - 1 + cc, gj = y0 - 1 + rr;
      bool ok = e < CELLS && !((gi < 0 || gi >= nx) && (gj < 0 || gj >= ny));  // corners unused
      bool neg = false;
      if (gi < 0) {
        if (a.bcx == BC_P) gi = nx - 1; else { gi = 0; neg ^= (xl == END_D); }
      } else if (gi == nx) {
        if (a.bcx == BC_P) gi = 0; else { gi = nx - 1; neg ^= (xh == END_D); }
      } else if (gi > nx) {
        ok = false;
      }
      if (gj < 0) {
        if (a.bcy == BC_P) gj = ny - 1; else { gj = 0; neg ^= (yl == END_D); }
      } else if (gj == ny) {
        if (a.bcy == BC_P) gj = 0; else { gj = ny - 1; neg ^= (yh == END_D); }
      } else if (gj > ny) {
        ok = false;
      }
      off[h] = ok ? gj * nx + gi : 0;
      okm |= (ok ? 1u : 0u) << h;
      negm |= (neg ? 1u : 0u) << h;
    }
  }
  auto issue = [&](int q, int slot) {  // raw copies of logical plane q (wrap or clamp in z)
    const int pq = q < 0 ? (perz ? q + nz : 0) : (q >= nz ? (perz ? q - nz : nz - 1) : q);
    const double* src = P + (size_t)pq * sxy;
    double* dst = raw + slot * CELLS;
#pragma unroll
    for (int h = 0; h < CPT; ++h) {
      const int e = tid + h * RTHREADS;
      if (h < CPT - 1 || e < CELLS) cp_async8(dst + e, src + off[h], (okm >> h) & 1u);
    }
    cp_commit();
  };
  auto convert = [&](int q, int slot, int fslot) {  // split logical plane q
    const uint32_t zs = q < 0 ? zsg_lo : (q >= nz ? zsg_hi : 0u);
    const double* src = raw + slot * CELLS;
    fxp* dst = fx + fslot * CELLS;
#pragma unroll
    for (int h = 0; h < CPT; ++h) {
      const int e = tid + h * RTHREADS;
      if (h < CPT - 1 || e < CELLS)
        dst[e] = to_fxp(flip_sign(src[e], (((negm >> h) & 1u) << 31) ^ zs), S, iS);
    }
  };

  int cidx[RPT];
  bool in[RPT];
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    cidx[m] = (ty * RPT + m + 1) * W + tx + 1;
    in[m] = (i < nx) && (jb + m < ny);
  }
  // Interior tiles (every row and column in the domain) take a copy of the
  // march without the per-point domain tests.
  const bool interior = (x0 + RTX <= nx) && (y0 + TY <= ny);
  const double* fcol = F + (size_t)jb * nx + i;  // this thread's column, row jb, plane 0
  auto load_f = [&](int k, double* fv, auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
    for (int m = 0; m < RPT; ++m)
      fv[m] = (FULL || in[m]) ? __ldg(fcol + (size_t)k * sxy + (size_t)m * nx) : 0.0;
  };

  // prologue: planes k0−1 … k0+RDEPTH−2 in flight; split k0−1 and k0
#pragma unroll
  for (int q = 0; q < RDEPTH; ++q) {
    if (k0 - 1 + q <= k1) issue(k0 - 1 + q, q);
    else cp_commit();
  }
  double fcur[RPT], fnext[RPT];
  if (interior) load_f(k0, fcur, std::true_type{});
  else load_f(k0, fcur, std::false_type{});
  cp_wait<RDEPTH - 2>();
  __syncthreads();
  convert(k0 - 1, 0, 0);
  convert(k0, 1, 1);
  __syncthreads();
  fxp zm[RPT], zc[RPT], zp[RPT];
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    zm[m] = fx[cidx[m]];
    zc[m] = fx[CELLS + cidx[m]];
  }

  float rmax = -INFINITY, rmin = INFINITY, fmax_ = -INFINITY, fmin_ = INFINITY;
  float wr = 0.f;
  df wf = {0.f, 0.f};
  const df mu = SING ? df{a.mu[0], a.mu[1]} : df{0.f, 0.f};
  int islot = 0;                 // raw slot of plane k + RDEPTH − 1 (≡ k − k0 mod RDEPTH)
  int cslot = 2 % RDEPTH;        // raw slot of plane k + 1
  auto march = [&](auto full_tag) {
  constexpr bool FULL = decltype(full_tag)::value;
  for (int k = k0; k < k1; ++k) {
    const int par = (k - k0) & 1;  // split slot of plane k+1; plane k is in 1 − par
    if (k + 1 < k1) load_f(k + 1, fnext, full_tag);
    // keep the ring full (an empty group keeps the wait count uniform)
    if (k + RDEPTH - 1 <= k1) issue(k + RDEPTH - 1, islot);
    else cp_commit();
    cp_wait<RDEPTH - 2>();  // plane k+1 has landed
    __syncthreads();
    convert(k + 1, cslot, par);
    __syncthreads();
    islot = (islot + 1 == RDEPTH) ? 0 : islot + 1;
    cslot = (cslot + 1 == RDEPTH) ? 0 : cslot + 1;
    const fxp* Fc = fx + (1 - par) * CELLS;
    const fxp* Fn = fx + par * CELLS;
#pragma unroll
    for (int m = 0; m < RPT; ++m) zp[m] = Fn[cidx[m]];
    const float2 cl = __ldg(a.zlo + k), ch = __ldg(a.zhi + k);
    const float w = SING ? __ldg(a.wz + k) : 0.f;
    float* rcol = a.r + (size_t)k * sxy + (size_t)jb * nx + i;
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      const fxp pc = zc[m];
      const fxp xm = Fc[cidx[m] - 1], xp = Fc[cidx[m] + 1];
      const fxp ym = (m == 0) ? Fc[cidx[0] - W] : zc[m > 0 ? m - 1 : 0];
      const fxp yp = (m == RPT - 1) ? Fc[cidx[RPT - 1] + W] : zc[m + 1 < RPT ? m + 1 : 0];
      const fxp zmv = zm[m], zpv = zp[m];
      const df fv = df_from_f64(fcur[m]);
      // exact high-part stencil sums (fixed-point grid), FP32 low parts
      const float sx = (xm.h + xp.h) - 2.f * pc.h, sy = (ym.h + yp.h) - 2.f * pc.h;
      const float dm = zmv.h - pc.h, dpz = zpv.h - pc.h;
      const float lx = (xm.l + xp.l) - 2.f * pc.l, ly = (ym.l + yp.l) - 2.f * pc.l;
      const float lo_terms = lx * a.idx2.h + ly * a.idy2.h + cl.x * (zmv.l - pc.l) + ch.x * (zpv.l - pc.l);
      const df t1 = prod(sx, a.idx2), t2 = prod(sy, a.idy2);
      const df t3 = prod(dm, df{cl.x, cl.y}), t4 = prod(dpz, df{ch.x, ch.y});
      const df s12 = two_sum(t1.h, t2.h);
      const df s123 = two_sum(s12.h, t3.h);
      const df s1234 = two_sum(s123.h, t4.h);
      const float ap_lo = ((s12.l + s123.l) + (s1234.l + t1.l)) + ((t2.l + t3.l) + (t4.l + lo_terms));
      df r;
      if (SING) {
        const df d1 = two_sum(fv.h, -mu.h);
        const df d2 = two_sum(d1.h, -s1234.h);
        r = {d2.h, ((d1.l + d2.l) + (fv.l - mu.l)) - ap_lo};
      } else {
        const df d2 = two_sum(fv.h, -s1234.h);
        r = {d2.h, (d2.l + fv.l) - ap_lo};
      }
      const float rf = r.h + r.l;
      if (FULL || in[m]) {
        rcol[(size_t)m * nx] = rf;
        const float ff = fv.h + fv.l;
        rmax = fmaxf(rmax, rf);
        rmin = fminf(rmin, rf);
        fmax_ = fmaxf(fmax_, ff);
        fmin_ = fminf(fmin_, ff);
        if (SING) {
          wr = fmaf(w, rf, wr);
          if (FIRST) {  // Σ Δz^f·f in double-float (only the first pass needs μ_f)
            wf = add_u(wf, prod(fv.h, df{w, 0.f}));
            wf.l = fmaf(w, fv.l, wf.l);
          }
        }
      }
    }
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      zm[m] = zc[m];
      zc[m] = zp[m];
      fcur[m] = fnext[m];
    }
  }
  };
  if (interior) march(std::true_type{});
  else march(std::false_type{});
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
  __shared__ float red[RWARPS][8];
  if (tx == 0) {
    red[ty][0] = rmax; red[ty][1] = rmin; red[ty][2] = fmax_; red[ty][3] = fmin_;
    red[ty][4] = wrd.h; red[ty][5] = wrd.l; red[ty][6] = wf.h; red[ty][7] = wf.l;
  }
  __syncthreads();
  if (ty == 0 && tx == 0) {
    for (int w = 1; w < RWARPS; ++w) {
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

namespace {
// Launch shape of one residual pass: rows per thread, planes per CTA, grid.
struct ResidShape {
  int rpt, zchunk;
  dim3 grid;
};
ResidShape resid_shape(int nx, int ny, int nz) {
  ResidShape s;
  s.rpt = ny >= 4 * RWARPS ? 4 : 2;
  const int tiles = ((nx + RTX - 1) / RTX) * ((ny + RWARPS * s.rpt - 1) / (RWARPS * s.rpt));
  // about four waves of three CTAs per SM, 8 … 64 planes per CTA
  const long long want = 152LL * 3 * 4;
  long long zc = ((long long)nz * tiles) / want;
  zc = zc < 8 ? 8 : (zc > 64 ? 64 : zc);
  s.zchunk = (int)(zc < nz ? zc : nz);
  s.grid = dim3((nx + RTX - 1) / RTX, (ny + RWARPS * s.rpt - 1) / (RWARPS * s.rpt),
                (nz + s.zchunk - 1) / s.zchunk);
  return s;
}
template <int RPT, int MODE>
cudaError_t launch_resid_mode(const ResidArgs& b, dim3 grid, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(residual_kernel<RPT, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)resid_smem(RPT));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  residual_kernel<RPT, MODE><<<grid, dim3(RTX, RWARPS), resid_smem(RPT), st>>>(b);
  return cudaGetLastError();
}
template <int RPT>
cudaError_t launch_resid_rpt(const ResidArgs& b, dim3 grid, cudaStream_t st) {
  if (!b.singular) return launch_resid_mode<RPT, 0>(b, grid, st);
  return b.first ? launch_resid_mode<RPT, 2>(b, grid, st) : launch_resid_mode<RPT, 1>(b, grid, st);
}
}  // namespace

int residual_blocks(int nx, int ny, int nz) {
  const ResidShape s = resid_shape(nx, ny, nz);
  return (int)(s.grid.x * s.grid.y * s.grid.z);
}

cudaError_t launch_residual(const ResidArgs& a, cudaStream_t st) {
  if (!a.r) return cudaErrorInvalidValue;
  reset_red_kernel<<<1, 1, 0, st>>>(a.red, a.skip);
  const ResidShape s = resid_shape(a.nx, a.ny, a.nz);
  ResidArgs b = a;
  b.zchunk = s.zchunk;
  return s.rpt == 4 ? launch_resid_rpt<4>(b, s.grid, st) : launch_resid_rpt<2>(b, s.grid, st);
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
