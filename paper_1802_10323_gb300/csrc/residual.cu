// residual.cu — residuals r = f − A·Φ (Eq. 4) of the iterative refinement, in double-float.
//
// FP64 arithmetic and f64<->f32 conversions issue at ~1/64 of the FP32 rate on
// this part, so the 7-point stencil is evaluated in FP32 with error-free
// transformations (TwoSum, FMA products; "double-float", ~48 significant bits).
// The refinement loop evaluates
//       pass 0:  r_0 = f − A·Φ_0                 (f FP64, split on its bit pattern)
//       pass m:  r_m = r_{m−1} − c_m − A·e_{m−1}  (r_{m−1} stored as FP32 hi + lo)
// with Φ_0 the FP32 solve (its FP64 widening is the stored Φ, exactly), e the last
// FP32 correction, c_1 = μ_f (singular problems) and c_m = 0 otherwise; r is stored
// as hi + lo (the hi part is the right-hand side of the next FP32 correction solve).
// Since e is small, A·e needs accuracy relative to |e| only, not to |Φ|, so later
// passes are more accurate than a fresh evaluation. Two kernels:
//   * residual_kernel (pass 0, and an optional exact confirmation at the end,
//     r = f − μ_f − A·Φ from the stored FP64 Φ): the operand is split on a
//     fixed-point grid (below) and the stencil evaluated in double-float,
//     ~2^-44·‖A‖·max|U|, three levels when that is not enough;
//   * residual_acc_kernel (passes m ≥ 1): the sum-form stencil accumulated in a
//     single FP32 word offset into a fixed binade (see there), ~2^-39·‖A‖·max|e|.
//
// Splitting the operand: U = ph + pl with ph on a fixed-point grid 2^−s common to
// the whole field (s from max|U|, so |ph|·2^s < 2^20): the stencil sums of ph are
// exact in FP32, the four products with the double-float coefficients are made
// exact with FMA, and the small pl part only needs FP32. For an FP32 U the split
// is exact (pl = U − ph has at most 24 bits); for an FP64 U, pl is rounded.
//
// Blocking: a CTA of 32 × 8 threads owns a 32 × (8·RPT) (x, y) tile and marches
// along z over a chunk of planes; each thread computes RPT consecutive rows of one
// x column. Raw planes of U (tile plus one halo cell per side) stream into a
// shared-memory ring with cp.async, RDEPTH − 2 planes ahead of the one being
// split; each plane is split once into fixed-point pairs (two plane slots), from
// which the in-plane neighbours are read. The z neighbours of a thread's own
// cells stay in registers (planes k−1, k, k+1), and the base (f or r) streams
// through registers one plane ahead with plain loads. The kernel is bound by
// instruction issue rather than bytes, so the per-plane work that does not scale
// with the points is shared by RPT points, the ring slots advance by counters,
// the pass kind is compile-time and interior tiles skip the per-point domain tests.
//
// Ends of each axis (staggered ghost rules of Table 1) are folded into the halo
// load: a periodic end wraps; a Neumann end loads the adjacent interior cell
// (ghost = Φ, so its term vanishes); a Dirichlet end loads it with the sign
// flipped (ghost = −Φ, term coef·(−2Φ)). In z the same holds for the ghost
// planes below k = 0 and above k = n_z − 1, and the coefficients zlo/zhi hold
// a_k, c_k, the wrap couplings, or 1/(Δz^f)² at a Dirichlet end.
//
// Reductions per pass (deterministic): max and min of r (and of f in pass 0)
// through order-preserving integer keys, and, for singular problems, per-block
// double-float sums of Δz^f·r (and Δz^f·f in pass 0) for the weighted means. The
// finalize kernels form ‖r_c‖∞ = max(max r − μ_r, μ_r − min r) and the same for
// f, compare with rtol and set the flags that make later kernels return at once.
#include <type_traits>

#include "internal.h"

namespace ps {

enum { END_WRAP = 0, END_N = 1, END_D = 2 };
constexpr int RTX = 32, RWARPS = 8, RTHREADS = RTX * RWARPS;
constexpr int RDEPTH = 4;  // raw-plane ring: k+1 being split, k+2 … k+3 in flight

// Pass kinds (bit flags of the kernel template).
enum : int {
  RK_SING = 1,    // singular problem: weighted sum of r
  RK_FIRST = 2,   // pass 0: max/min of f, and (singular) the weighted sum of f
  RK_SUBMU = 4,   // subtract μ_f (double-float) from the base
  RK_U32 = 8,     // operand U is FP32 (else FP64)
  RK_SHIFT = 16,  // Helmholtz plan: the row also holds −α·U (exact product with each level)
  RK_SPLIT3 = 32,  // three-level split of U (pass 0 and the exact pass; see below)
  RK_FACE = 64     // x or y face unknowns (BC_FD): the wall rows of face_rows
};

__host__ __device__ constexpr int resid_cells(int rpt) { return (RTX + 2) * (RWARPS * rpt + 2); }
__host__ __device__ constexpr size_t resid_smem(int rpt, int usize, int csize) {
  return (size_t)RDEPTH * resid_cells(rpt) * usize + (size_t)2 * resid_cells(rpt) * csize;
}

// (face unknowns in z, BC_FD: both ends take the Dirichlet ghost rule; the plan scales the
// end coefficients so that row 0 reads −p_0 and the top row sees a zero wall node)
__device__ __forceinline__ int end_lo(int bc) {
  return bc == BC_P ? END_WRAP : ((bc == BC_DD || bc == BC_DN || bc == BC_FD) ? END_D : END_N);
}
__device__ __forceinline__ int end_hi(int bc) {
  return bc == BC_P ? END_WRAP : ((bc == BC_DD || bc == BC_ND || bc == BC_FD) ? END_D : END_N);
}

// unevaluated double-float sum
__device__ __forceinline__ df add_u(df a, df b) {
  df s = two_sum(a.h, b.h);
  return {s.h, s.l + a.l + b.l};
}

// U on a fixed-point grid: ph = rint(U·2^s)·2^−s (|U·2^s| < 2^20 for every U of
// the field, so sums and differences of a few ph are exact in FP32) and
// pl = U − ph (|pl| ≤ 2^−s−1), exact for an FP32 U and rounded to FP32 for an FP64
// U. A·ph is then exact up to the coefficient products, and A·pl only needs FP32.
//
// The FP32 evaluation of A·pl errs by ~2^−24·‖A‖·2^−s ≈ 2^−44·‖A‖·max|U|: pl is
// noise-like, so its second differences do not cancel before they meet the large
// z coefficients. That is small against the residual when U is a correction, but
// not when U is the whole solution of an ill-conditioned problem (‖A‖·max|Φ| ≫
// max|f|). Pass 0 and the exact pass therefore split three ways, U = ph + pm + pr
// with pm on the grid 2^−s−20 as well: the sums of pm are exact too, their
// products with the coefficients are made exact with FMA and summed in
// double-float, and only pr (≤ 2^−s−21) is evaluated in FP32.
struct fxp {
  float h, l;
};
struct __align__(16) fxp3 {
  float h, m, l, pad;
};
__device__ __forceinline__ fxp to_fxp(double d, float S, float iS) {
  float h, l;
  split_f64(d, h, l);
  const float ph = __fmul_rn(rintf(__fmul_rn(h, S)), iS);
  return {ph, __fadd_rn(__fsub_rn(h, ph), l)};
}
// (float operand: rounding to the grid 2^−s by adding and removing C = 1.5·2^(23−s),
// whose unit in the last place is 2^−s; |u| < 2^(20−s) keeps u + C in C's binade, so
// this is round-to-nearest-even onto the grid, as rint(u·2^s)·2^−s, in two additions)
__device__ __forceinline__ float to_grid(float u, float C) { return __fsub_rn(__fadd_rn(u, C), C); }
__device__ __forceinline__ fxp to_fxp(float u, float C) {
  const float ph = to_grid(u, C);
  return {ph, __fsub_rn(u, ph)};
}
// Three levels of an FP64 value from its 53-bit significand M (x = ±M·2^(eb−1075)):
// x·2^(s+20) = I + F·2^−sh with the integer I < 2^40 and sh ≥ 13 fraction bits;
// ph = ⌊I/2^20⌋·2^−s, pm = (I mod 2^20)·2^−s−20 and pr = F·2^(eb−1075) are exact in
// FP32 for |x| near max|x| (pr then has ≤ 13 bits); smaller values round only pr,
// by 2^−24 of itself. (Truncating x to 48 bits instead would leave ~2^−48·|x| of
// noise, which ‖A‖ amplifies.)
__device__ __forceinline__ fxp3 to_fxp3(double x, int sc, float iS, float iS2) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((b >> 52) & 0x7FF);
  const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = max(0, 1075 - 20 - sc - eb);
  const unsigned long long I = sh >= 64 ? 0ull : (M >> sh);
  const unsigned long long F = sh >= 64 ? M : (M - (I << sh));
  const int er = eb - 948;  // biased FP32 exponent of 2^(eb−1075)
  const float scale = __uint_as_float((uint32_t)(er > 0 ? er : 0) << 23);
  float ph = __fmul_rn(__ull2float_rn(I >> 20), iS);
  float pm = __fmul_rn((float)(uint32_t)(I & 0xFFFFFull), iS2);
  float pr = __fmul_rn(__ull2float_rn(F), scale);
  if (eb == 0) ph = pm = pr = 0.f;  // zero (and subnormals, below every grid here)
  if (b >> 63) {
    ph = -ph;
    pm = -pm;
    pr = -pr;
  }
  return {ph, pm, pr, 0.f};
}
// three levels of an FP32 value (exact); C2 = C·2^−20 (the grid 2^−s−20)
__device__ __forceinline__ fxp3 to_fxp3(float u, float C, float C2) {
  const float ph = to_grid(u, C);
  const float d = __fsub_rn(u, ph);  // exact
  const float pm = to_grid(d, C2);
  return {ph, pm, __fsub_rn(d, pm), 0.f};
}
// exact product of an FP32 value and a double-float coefficient, unevaluated
__device__ __forceinline__ df prod(float x, df w) {
  const float p = __fmul_rn(x, w.h);
  return {p, __fmaf_rn(x, w.l, __fmaf_rn(x, w.h, -p))};
}
// flip the sign (bit 31 of the float, of the high word of the double) when sgn is set
__device__ __forceinline__ double flip_sign(double d, uint32_t sgn) {
  return __hiloint2double(__double2hiint(d) ^ (int)sgn, __double2loint(d));
}
__device__ __forceinline__ float flip_sign(float u, uint32_t sgn) {
  return __uint_as_float(__float_as_uint(u) ^ sgn);
}

// Asynchronous global→shared copy of B bytes; a zero source size fills zeros and
// reads nothing (used for cells that no in-domain point needs).
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(gmem), "n"(B),
               "r"(valid ? B : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Block reductions of one pass (warp shuffles, then one thread over the warps):
// max and min of r (and of f when FIRST) into the reduction words, and the
// per-block double-float weighted sums into the partials.
template <bool FIRST>
__device__ __forceinline__ void resid_reduce(const ResidArgs& a, float rmax, float rmin, float fmax_,
                                             float fmin_, float wr, df wf) {
  const int tx = threadIdx.x, ty = threadIdx.y;
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
    if (FIRST) {
      atomicMax(&a.red[2], f32_key(fmax_));
      atomicMin(&a.red[3], f32_key(fmin_));
    }
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    reinterpret_cast<float4*>(a.partial)[bid] = make_float4(wrd.h, wrd.l, wf.h, wf.l);
  }
}

// x/y face unknowns (BC_FD): the wall entry's row has the x (or y) part −u_0/Δ²,
// i.e. the neighbours (u_0, 0) in the second difference, and the first interior
// row sees the wall node 0 instead of the stored entry. Only tiles that touch the
// low end of such an axis run this (they are never "interior").
template <class CT>
__device__ __forceinline__ void face_rows(const ResidArgs& a, int i, int j, const CT& pc, CT& xm, CT& xp, CT& ym,
                                          CT& yp) {
  const CT zero{};
  if (a.bcx == BC_FD) {
    if (i == 0) { xm = pc; xp = zero; }
    else if (i == 1) xm = zero;
  }
  if (a.bcy == BC_FD) {
    if (j == 0) { ym = pc; yp = zero; }
    else if (j == 1) ym = zero;
  }
}

template <int RPT, int KIND>
__global__ void __launch_bounds__(RTHREADS, RPT >= 4 ? 3 : 4) residual_kernel(ResidArgs a) {
  constexpr bool SING = KIND & RK_SING, FIRST = KIND & RK_FIRST, SUBMU = KIND & RK_SUBMU;
  constexpr bool U32 = KIND & RK_U32, SPLIT3 = KIND & RK_SPLIT3, SHIFT = KIND & RK_SHIFT, FACE = KIND & RK_FACE;
  using UT = typename std::conditional<U32, float, double>::type;
  using CT = typename std::conditional<SPLIT3, fxp3, fxp>::type;  // a split cell
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
  float S, iS, iS2, C, C2;
  int sc;
  {
    const int e = (int)((*a.pmax_bits >> 52) & 0x7FF) - 1023;  // max|U| ∈ [2^e, 2^(e+1))
    sc = max(-100, min(100, 19 - e));
    S = __uint_as_float((uint32_t)(sc + 127) << 23);
    iS = __uint_as_float((uint32_t)(127 - sc) << 23);
    iS2 = __uint_as_float((uint32_t)(127 - sc - 20) << 23);
    C = __uint_as_float(((uint32_t)(23 - sc + 127) << 23) | 0x400000u);       // 1.5·2^(23−s)
    C2 = __uint_as_float(((uint32_t)(23 - sc - 20 + 127) << 23) | 0x400000u); // 1.5·2^(3−s)
  }
  extern __shared__ __align__(16) double rsm[];
  UT* raw = reinterpret_cast<UT*>(rsm);  // [RDEPTH][CELLS]
  CT* fx = reinterpret_cast<CT*>(reinterpret_cast<char*>(rsm) + RDEPTH * CELLS * sizeof(UT));  // [2][CELLS]
  const UT* __restrict__ P = static_cast<const UT*>(U32 ? static_cast<const void*>(a.u) : a.p);

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
      const bool gout = (gi < 0 || gi == nx), hout = (gj < 0 || gj == ny);
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
      if constexpr (FACE) {  // x/y face unknowns (BC_FD): the wall nodes beyond either end are 0
        if ((gout && a.bcx == BC_FD) || (hout && a.bcy == BC_FD)) ok = false;
      }
      off[h] = ok ? gj * nx + gi : 0;
      okm |= (ok ? 1u : 0u) << h;
      negm |= (neg ? 1u : 0u) << h;
    }
  }
  auto issue = [&](int q, int slot) {  // raw copies of logical plane q (wrap or clamp in z)
    const int pq = q < 0 ? (perz ? q + nz : 0) : (q >= nz ? (perz ? q - nz : nz - 1) : q);
    const UT* src = P + (size_t)pq * sxy;
    UT* dst = raw + slot * CELLS;
#pragma unroll
    for (int h = 0; h < CPT; ++h) {
      const int e = tid + h * RTHREADS;
      if (h < CPT - 1 || e < CELLS) cp_async<sizeof(UT)>(dst + e, src + off[h], (okm >> h) & 1u);
    }
    cp_commit();
  };
  auto convert = [&](int q, int slot, int fslot) {  // split logical plane q
    const uint32_t zs = q < 0 ? zsg_lo : (q >= nz ? zsg_hi : 0u);
    const UT* src = raw + slot * CELLS;
    CT* dst = fx + fslot * CELLS;
    auto one = [&](UT x, int e) {
      if constexpr (SPLIT3 && U32) dst[e] = to_fxp3(x, C, C2);
      else if constexpr (SPLIT3) dst[e] = to_fxp3(x, sc, iS, iS2);
      else if constexpr (U32) dst[e] = to_fxp(x, C);
      else dst[e] = to_fxp(x, S, iS);
    };
    if ((negm | zs) == 0u) {  // no Dirichlet ghost among this thread's cells
#pragma unroll
      for (int h = 0; h < CPT; ++h) {
        const int e = tid + h * RTHREADS;
        if (h < CPT - 1 || e < CELLS) one(src[e], e);
      }
    } else {
#pragma unroll
      for (int h = 0; h < CPT; ++h) {
        const int e = tid + h * RTHREADS;
        if (h < CPT - 1 || e < CELLS) one(flip_sign(src[e], (((negm >> h) & 1u) << 31) ^ zs), e);
      }
    }
  };

  int cidx[RPT];
  bool in[RPT];
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    cidx[m] = (ty * RPT + m + 1) * W + tx + 1;
    in[m] = (i < nx) && (jb + m < ny);
  }
  // Interior tiles (every row and column in the domain, no face-unknown wall row)
  // take a copy of the march without the per-point domain tests.
  const bool interior = (x0 + RTX <= nx) && (y0 + TY <= ny) &&
                        !(FACE && ((a.bcx == BC_FD && x0 == 0) || (a.bcy == BC_FD && y0 == 0)));
  const size_t col = (size_t)jb * nx + i;  // this thread's column, row jb, plane 0
  // the base of each point: f (FP64, split into hi + lo)
  using base_t = double;
  auto load_base = [&](int k, base_t* bv, auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      const size_t g = (size_t)k * sxy + col + (size_t)m * nx;
      const bool ld = FULL || in[m];
      bv[m] = ld ? __ldg(a.f + g) : 0.0;
    }
  };

  // prologue: planes k0−1 … k0+RDEPTH−2 in flight; split k0−1 and k0
#pragma unroll
  for (int q = 0; q < RDEPTH; ++q) {
    if (k0 - 1 + q <= k1) issue(k0 - 1 + q, q);
    else cp_commit();
  }
  base_t bcur[RPT], bnext[RPT];
  if (interior) load_base(k0, bcur, std::true_type{});
  else load_base(k0, bcur, std::false_type{});
  cp_wait<RDEPTH - 2>();
  __syncthreads();
  convert(k0 - 1, 0, 0);
  convert(k0, 1, 1);
  __syncthreads();
  CT zm[RPT], zc[RPT], zp[RPT];
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    zm[m] = fx[cidx[m]];
    zc[m] = fx[CELLS + cidx[m]];
  }

  float rmax = -INFINITY, rmin = INFINITY, fmax_ = -INFINITY, fmin_ = INFINITY;
  float wr = 0.f;
  // Σ Δz^f·f (pass 0 of a singular problem) in FP64: one FMA per point on the FP64
  // pipe, which nothing else in this kernel uses, instead of ~12 FP32 operations
  // of a double-float product and sum on the issue-bound FP32 path
  double wfd = 0.0;
  const df mu = SUBMU ? df{a.mu[0], a.mu[1]} : df{0.f, 0.f};
  const bool store_r = a.rh_out != nullptr;
  int islot = 0;                 // raw slot of plane k + RDEPTH − 1 (≡ k − k0 mod RDEPTH)
  int cslot = 2 % RDEPTH;        // raw slot of plane k + 1
  auto march = [&](auto full_tag) {
  constexpr bool FULL = decltype(full_tag)::value;
  for (int k = k0; k < k1; ++k) {
    const int par = (k - k0) & 1;  // split slot of plane k+1; plane k is in 1 − par
    if (k + 1 < k1) load_base(k + 1, bnext, full_tag);
    // keep the ring full (an empty group keeps the wait count uniform)
    if (k + RDEPTH - 1 <= k1) issue(k + RDEPTH - 1, islot);
    else cp_commit();
    cp_wait<RDEPTH - 2>();  // plane k+1 has landed
    __syncthreads();
    convert(k + 1, cslot, par);
    __syncthreads();
    islot = (islot + 1 == RDEPTH) ? 0 : islot + 1;
    cslot = (cslot + 1 == RDEPTH) ? 0 : cslot + 1;
    const CT* Fc = fx + (1 - par) * CELLS;
    const CT* Fn = fx + par * CELLS;
#pragma unroll
    for (int m = 0; m < RPT; ++m) zp[m] = Fn[cidx[m]];
    const float2 cl = __ldg(a.zlo + k), ch = __ldg(a.zhi + k);
    const float w = SING ? __ldg(a.wz + k) : 0.f;
    const double wd = (SING && FIRST) ? (double)w : 0.0;
    const size_t gk = (size_t)k * sxy + col;
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      const CT pc = zc[m];
      CT xm = Fc[cidx[m] - 1], xp = Fc[cidx[m] + 1];
      CT ym = (m == 0) ? Fc[cidx[0] - W] : zc[m > 0 ? m - 1 : 0];
      CT yp = (m == RPT - 1) ? Fc[cidx[RPT - 1] + W] : zc[m + 1 < RPT ? m + 1 : 0];
      if constexpr (FACE && !FULL) face_rows(a, i, jb + m, pc, xm, xp, ym, yp);
      const CT zmv = zm[m], zpv = zp[m];
      const df bv = df_from_f64(bcur[m]);
      // exact high-part stencil sums (fixed-point grid), FP32 low parts
      const float sx = (xm.h + xp.h) - 2.f * pc.h, sy = (ym.h + yp.h) - 2.f * pc.h;
      const float dm = zmv.h - pc.h, dpz = zpv.h - pc.h;
      const float lx = (xm.l + xp.l) - 2.f * pc.l, ly = (ym.l + yp.l) - 2.f * pc.l;
      const float lo_terms = lx * a.idx2.h + ly * a.idy2.h + cl.x * (zmv.l - pc.l) + ch.x * (zpv.l - pc.l);
      const df t1 = prod(sx, a.idx2), t2 = prod(sy, a.idy2);
      const df t3 = prod(dm, df{cl.x, cl.y}), t4 = prod(dpz, df{ch.x, ch.y});
      const df s12 = two_sum(t1.h, t2.h);
      const df s123 = two_sum(s12.h, t3.h);
      df s1234 = two_sum(s123.h, t4.h);
      float ap_lo = ((s12.l + s123.l) + (s1234.l + t1.l)) + ((t2.l + t3.l) + (t4.l + lo_terms));
      if constexpr (SHIFT) {  // −α·U: the high level's product exact, the low level in FP32
        const df t5 = prod(pc.h, a.nalpha);
        const df s5 = two_sum(s1234.h, t5.h);
        s1234 = {s5.h, 0.f};
        ap_lo += (s5.l + t5.l) + a.nalpha.h * pc.l;
      }
      if constexpr (SPLIT3) {
        // the middle level: exact sums on its grid, exact products, double-float sums
        const float mx = (xm.m + xp.m) - 2.f * pc.m, my = (ym.m + yp.m) - 2.f * pc.m;
        const df u1 = prod(mx, a.idx2), u2 = prod(my, a.idy2);
        const df u3 = prod(zmv.m - pc.m, df{cl.x, cl.y}), u4 = prod(zpv.m - pc.m, df{ch.x, ch.y});
        const df m12 = two_sum(u1.h, u2.h);
        const df m123 = two_sum(m12.h, u3.h);
        df m1234 = two_sum(m123.h, u4.h);
        if constexpr (SHIFT) {
          const df u5 = prod(pc.m, a.nalpha);
          const df m5 = two_sum(m1234.h, u5.h);
          ap_lo += m1234.l + u5.l;
          m1234 = {m5.h, m5.l};
        }
        const df hm = two_sum(s1234.h, m1234.h);
        s1234 = {hm.h, 0.f};
        ap_lo += ((m12.l + m123.l) + (m1234.l + u1.l)) + ((u2.l + u3.l) + (u4.l + hm.l));
      }
      df r;
      if constexpr (SUBMU) {
        const df d1 = two_sum(bv.h, -mu.h);
        const df d2 = two_sum(d1.h, -s1234.h);
        r = {d2.h, ((d1.l + d2.l) + (bv.l - mu.l)) - ap_lo};
      } else {
        const df d2 = two_sum(bv.h, -s1234.h);
        r = {d2.h, (d2.l + bv.l) - ap_lo};
      }
      const float rf = r.h + r.l;
      if (FULL || in[m]) {
        const size_t g = gk + (size_t)m * nx;
        if constexpr (U32) {
          if (store_r) {
            a.rh_out[g] = rf;
            a.rl_out[g] = r.l - (rf - r.h);
          }
        } else {
          a.r[g] = rf;
        }
        rmax = fmaxf(rmax, rf);
        rmin = fminf(rmin, rf);
        if constexpr (FIRST) {
          const float ff = bv.h + bv.l;
          fmax_ = fmaxf(fmax_, ff);
          fmin_ = fminf(fmin_, ff);
        }
        if constexpr (SING) {
          wr = fmaf(w, rf, wr);
          if constexpr (FIRST) wfd = fma(wd, bcur[m], wfd);  // only pass 0 needs μ_f
        }
      }
    }
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      zm[m] = zc[m];
      zc[m] = zp[m];
      bcur[m] = bnext[m];
    }
  }
  };
  if (interior) march(std::true_type{});
  else march(std::false_type{});
  cp_wait<0>();

  df wf = {0.f, 0.f};
  if constexpr (SING && FIRST) {
    wf.h = (float)wfd;
    wf.l = (float)(wfd - (double)wf.h);
  }
  resid_reduce<FIRST>(a, rmax, rmin, fmax_, fmin_, wr, wf);
}

// ---------------------------------------------------------------------------
// Passes m ≥ 1 in one accumulator word.
//
// The operand is the last correction e (FP32), about 10^-7 of Φ, so A·e needs
// absolute accuracy ~2^-39·‖A‖∞·max|e| only (that error enters the drift bound
// and is far below the FP64 rounding of Φ). The stencil is taken in sum form,
//   A·e = Σ_j w_j·e_j over the cells x±1, y±1, z±1 and the centre,
// with double-float coefficients (the centre's w_c = −(2/Δx² + 2/Δy² + a_k + c_k))
// and accumulated in ONE FP32 word offset by σ = 1.5·2^G, where 2^(G−1) exceeds
// Σ_j |w_j|·max|e| and so every partial sum: the word stays in σ's binade, where
// every FMA acc' = fma(e_j, w_j.h, acc) rounds onto the fixed grid 2^(G−23), the
// difference acc − acc' is exact, and fma(e_j, w_j.h, acc − acc') is the rounding
// error itself (to 2^-24 of it). Those errors and the e_j·w_j.l terms go into a
// second word. Five FP32 operations per term instead of the split, the exact
// products and the TwoSum chain of the general kernel; the evaluation error is at
// most ~2^(G−41) ≤ 2^-39·Σ_j|w_j|·max|e|.
//
// The raw planes of e stream into a shared ring with cp.async (16-byte copies of
// each row's 32 interior cells when n_x is a multiple of 4) and are read in
// place: no split pass, one barrier per plane. The ghost rules of Table 1 are the
// general kernel's, with two changes: a Dirichlet z end keeps the clamped copy of
// the boundary plane and carries the sign in its coefficient (the per-plane table
// zres holds a_k, c_k and w_c with that sign folded in), and Dirichlet x/y halo
// cells are negated in shared memory by the thread that copied them, after the
// copy lands and before the barrier that publishes the plane.
enum : int {
  AK_SING = 1,   // singular problem: weighted sum of r
  AK_SUBMU = 2,  // subtract μ_f from the base (pass 1 of a singular problem)
  AK_OUT = 4,    // store r_m = hi + lo (else norms only)
  AK_VEC = 8     // n_x % 4 == 0: 16-byte row copies
};
constexpr int AW = 40;     // shared row pitch: halo at column 3, interior 4 … 35, halo at 36
constexpr int ADEPTH = 5;  // raw-plane ring: k, k+1 read; k+2 … k+4 in flight
__host__ __device__ constexpr int acc_cells(int rpt) { return AW * (RWARPS * rpt + 2); }

template <int RPT, int KIND>
__global__ void __launch_bounds__(RTHREADS, RPT >= 8 ? 2 : 3) residual_acc_kernel(ResidArgs a) {
  constexpr bool SING = KIND & AK_SING, SUBMU = KIND & AK_SUBMU, OUT = KIND & AK_OUT, VEC = KIND & AK_VEC;
  constexpr int TY = RWARPS * RPT, ROWS = TY + 2, CELLS = acc_cells(RPT);
  constexpr int NC16 = VEC ? (8 * ROWS + RTHREADS - 1) / RTHREADS : 1;           // 16-byte copies
  constexpr int NC4 = VEC ? 1 : ((RTX + 2) * ROWS + RTHREADS - 1) / RTHREADS;    // 4-byte copies
  if (a.skip && *a.skip) return;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t sxy = (size_t)nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RTX + tx;
  const int x0 = blockIdx.x * RTX, y0 = blockIdx.y * TY;
  const int i = x0 + tx, jb = y0 + ty * RPT;
  const int k0 = blockIdx.z * a.zchunk, k1 = min(nz, k0 + a.zchunk);
  const bool perz = (a.bcz == BC_P);
  float sig;  // σ = 1.5·2^G, 2^(G−2) ≤ 1.001·Σ|w|·max|e| < 2^(G−1)
  {
    const double B = 1.001 * a.asum * __longlong_as_double((long long)*a.pmax_bits);
    const int eb = (int)(((unsigned long long)__double_as_longlong(B) >> 52) & 0x7FF);
    const int G = max(-100, min(120, eb == 0 ? -100 : eb - 1023 + 2));
    sig = 1.5f * __uint_as_float((uint32_t)(G + 127) << 23);
  }
  extern __shared__ __align__(16) float ring[];  // [ADEPTH][ROWS][AW]

  // Copies of this thread: shared offset, in-plane source offset, and bits
  // "exists", "source valid" (else zero fill) and "negate" (Dirichlet ghost).
  int s16[NC16], g16[NC16], s4[NC4], g4[NC4];
  uint32_t has16 = 0, ok16 = 0, neg16 = 0, has4 = 0, ok4 = 0, neg4 = 0;
  {
    const int xl = end_lo(a.bcx), xh = end_hi(a.bcx), yl = end_lo(a.bcy), yh = end_hi(a.bcy);
    // row rr of the tile → source row (wrap or clamp), validity, sign
    auto map_y = [&](int rr, int& gj, bool& ok, bool& neg) {
      gj = y0 - 1 + rr;
      ok = true;
      neg = false;
      if (gj < 0) {
        if (a.bcy == BC_P) gj = ny - 1; else if (a.bcy == BC_FD) { gj = 0; ok = false; } else { gj = 0; neg = (yl == END_D); }
      } else if (gj == ny) {
        if (a.bcy == BC_P) gj = 0; else if (a.bcy == BC_FD) { gj = 0; ok = false; } else { gj = ny - 1; neg = (yh == END_D); }
      } else if (gj > ny) {
        ok = false;
      }
    };
    // column cc ∈ [0, 34) of the tile (cc = 0 and 33 are the halo) → source column
    auto map_x = [&](int cc, int& gi, bool& ok, bool& neg) {
      gi = x0 - 1 + cc;
      ok = true;
      neg = false;
      if (gi < 0) {
        if (a.bcx == BC_P) gi = nx - 1; else if (a.bcx == BC_FD) { gi = 0; ok = false; } else { gi = 0; neg = (xl == END_D); }
      } else if (gi == nx) {
        if (a.bcx == BC_P) gi = 0; else if (a.bcx == BC_FD) { gi = 0; ok = false; } else { gi = nx - 1; neg = (xh == END_D); }
      } else if (gi > nx) {
        ok = false;
      }
    };
    auto cell = [&](int rr, int cc, int& so, int& go, bool& ok, bool& neg) {
      int gj, gi;
      bool oky, negy, okx, negx;
      map_y(rr, gj, oky, negy);
      map_x(cc, gi, okx, negx);
      const int oj = y0 - 1 + rr, oi = x0 - 1 + cc;
      ok = oky && okx && !((oi < 0 || oi >= nx) && (oj < 0 || oj >= ny));  // corners unused
      neg = negx ^ negy;
      so = rr * AW + 3 + cc;
      go = ok ? gj * nx + gi : 0;
    };
    if constexpr (VEC) {
#pragma unroll
      for (int h = 0; h < NC16; ++h) {
        const int e = tid + h * RTHREADS;
        const int rr = e >> 3, q = e & 7;
        int gj;
        bool oky, negy;
        map_y(rr < ROWS ? rr : 0, gj, oky, negy);
        // chunks wholly beyond n_x are not copied (their cells are never read;
        // the right ghost of a ragged tile sits in the first of them)
        const bool ex = e < 8 * ROWS && x0 + 4 * q < nx;
        s16[h] = rr * AW + 4 + 4 * q;
        g16[h] = (ex && oky) ? gj * nx + x0 + 4 * q : 0;
        has16 |= (ex ? 1u : 0u) << h;
        ok16 |= (ex && oky ? 1u : 0u) << h;
        neg16 |= (ex && negy ? 1u : 0u) << h;
      }
      {  // the two x-halo cells of each row: x0 − 1 and min(x0 + 32, n_x)
        const int e = tid;
        const int rr = e >> 1, cc = (e & 1) ? min(RTX, nx - x0) + 1 : 0;
        bool ok, neg;
        cell(rr < ROWS ? rr : 0, cc, s4[0], g4[0], ok, neg);
        has4 = (e < 2 * ROWS) ? 1u : 0u;
        ok4 = (ok && has4) ? 1u : 0u;
        neg4 = (neg && has4) ? 1u : 0u;
      }
    } else {
      s16[0] = g16[0] = 0;
#pragma unroll
      for (int h = 0; h < NC4; ++h) {
        const int e = tid + h * RTHREADS;
        const int rr = e / (RTX + 2), cc = e - rr * (RTX + 2);
        bool ok, neg;
        cell(rr < ROWS ? rr : 0, cc, s4[h], g4[h], ok, neg);
        const bool ex = e < (RTX + 2) * ROWS;
        has4 |= (ex ? 1u : 0u) << h;
        ok4 |= (ok && ex ? 1u : 0u) << h;
        neg4 |= (neg && ex ? 1u : 0u) << h;
      }
    }
  }
  const bool doneg = (neg16 | neg4) != 0;
  const float* __restrict__ U = a.u;
  auto issue = [&](int q, int slot) {  // raw copies of logical plane q (wrap or clamp in z)
    const int pq = q < 0 ? (perz ? q + nz : 0) : (q >= nz ? (perz ? q - nz : nz - 1) : q);
    const float* src = U + (size_t)pq * sxy;
    float* dst = ring + slot * CELLS;
    if constexpr (VEC) {
#pragma unroll
      for (int h = 0; h < NC16; ++h)
        if ((has16 >> h) & 1u) {
          const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + s16[h]);
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src + g16[h]),
                       "r"(((ok16 >> h) & 1u) ? 16 : 0));
        }
    }
#pragma unroll
    for (int h = 0; h < NC4; ++h)
      if ((has4 >> h) & 1u) cp_async<4>(dst + s4[h], src + g4[h], (ok4 >> h) & 1u);
    cp_commit();
  };
  auto negate = [&](int slot) {  // Dirichlet ghosts of a landed plane (own copies only)
    float* dst = ring + slot * CELLS;
    if constexpr (VEC) {
#pragma unroll
      for (int h = 0; h < NC16; ++h)
        if ((neg16 >> h) & 1u) {
          float4* c4 = reinterpret_cast<float4*>(dst + s16[h]);
          float4 v = *c4;
          v.x = -v.x; v.y = -v.y; v.z = -v.z; v.w = -v.w;
          *c4 = v;
        }
    }
#pragma unroll
    for (int h = 0; h < NC4; ++h)
      if ((neg4 >> h) & 1u) dst[s4[h]] = -dst[s4[h]];
  };

  int cidx[RPT];
  bool in[RPT];
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    cidx[m] = (ty * RPT + m + 1) * AW + 4 + tx;
    in[m] = (i < nx) && (jb + m < ny);
  }
  const bool interior = (x0 + RTX <= nx) && (y0 + TY <= ny) && !(a.bcx == BC_FD && x0 == 0) &&
                        !(a.bcy == BC_FD && y0 == 0);
  const size_t col = (size_t)jb * nx + i;
  auto load_base = [&](int k, float2* bv, auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      const size_t g = (size_t)k * sxy + col + (size_t)m * nx;
      const bool ld = FULL || in[m];
      bv[m].x = ld ? __ldg(a.rh_in + g) : 0.f;
      bv[m].y = ld ? __ldg(a.rl_in + g) : 0.f;
    }
  };

  // prologue: planes k0−1 … k0+ADEPTH−2 in flight; wait for k0−1 and k0
#pragma unroll
  for (int q = 0; q < ADEPTH; ++q) {
    if (k0 - 1 + q <= k1) issue(k0 - 1 + q, q);
    else cp_commit();
  }
  float2 bcur[RPT], bnext[RPT];
  if (interior) load_base(k0, bcur, std::true_type{});
  else load_base(k0, bcur, std::false_type{});
  cp_wait<ADEPTH - 2>();
  if (doneg) negate(1);
  __syncthreads();
  float zm[RPT], zc[RPT], zp[RPT];
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    zm[m] = ring[cidx[m]];
    zc[m] = ring[CELLS + cidx[m]];
  }
  float rmax = -INFINITY, rmin = INFINITY, wr = 0.f;
  const df mu = SUBMU ? df{a.mu[0], a.mu[1]} : df{0.f, 0.f};
  const df wx = a.idx2, wy = a.idy2;
  int islot = 0;  // slot of plane k−1 (refilled with plane k+ADEPTH−1)
  int cslot = 1;  // plane k
  int nslot = 2;  // plane k+1
  auto march = [&](auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
    for (int k = k0; k < k1; ++k) {
      if (k + 1 < k1) load_base(k + 1, bnext, full_tag);
      cp_wait<ADEPTH - 3>();  // plane k+1 has landed
      if (doneg) negate(nslot);
      __syncthreads();        // … for every thread; plane k−1 is no longer read
      if (k + ADEPTH - 1 <= k1) issue(k + ADEPTH - 1, islot);
      else cp_commit();
      const float* Rc = ring + cslot * CELLS;
      const float* Rn = ring + nslot * CELLS;
      islot = cslot;  // plane k's slot is the free one next time
      cslot = nslot;
      nslot = (nslot + 1 == ADEPTH) ? 0 : nslot + 1;
#pragma unroll
      for (int m = 0; m < RPT; ++m) zp[m] = Rn[cidx[m]];
      const float2 c0 = __ldg(a.zres + 3 * k), c1 = __ldg(a.zres + 3 * k + 1), c2 = __ldg(a.zres + 3 * k + 2);
      const df cl = {c0.x, c0.y}, ch = {c1.x, c1.y}, cd = {c2.x, c2.y};
      const float w = SING ? __ldg(a.wz + k) : 0.f;
      const size_t gk = (size_t)k * sxy + col;
#pragma unroll
      for (int m = 0; m < RPT; ++m) {
        const int ci = cidx[m];
        float xm = Rc[ci - 1], xp = Rc[ci + 1];
        float ym = (m == 0) ? Rc[ci - AW] : zc[m > 0 ? m - 1 : 0];
        float yp = (m == RPT - 1) ? Rc[ci + AW] : zc[m + 1 < RPT ? m + 1 : 0];
        if (!FULL) face_rows(a, i, jb + m, zc[m], xm, xp, ym, yp);
        float acc = sig, lo = 0.f;
        auto term = [&](float u, df wt) {
          const float a2 = __fmaf_rn(u, wt.h, acc);
          lo = __fadd_rn(lo, __fmaf_rn(u, wt.h, __fsub_rn(acc, a2)));
          lo = __fmaf_rn(u, wt.l, lo);
          acc = a2;
        };
        term(zc[m], cd);
        term(zm[m], cl);
        term(zp[m], ch);
        term(xm, wx);
        term(xp, wx);
        term(ym, wy);
        term(yp, wy);
        const float H = __fsub_rn(acc, sig);  // exact: Σ_j w_j·e_j − lo
        df bv = {bcur[m].x, bcur[m].y};
        if constexpr (SUBMU) {
          const df d1 = two_sum(bv.h, -mu.h);
          bv = {d1.h, __fadd_rn(d1.l, __fsub_rn(bv.l, mu.l))};
        }
        const df d2 = two_sum(bv.h, -H);
        const float rl = __fsub_rn(__fadd_rn(d2.l, bv.l), lo);
        const float rf = __fadd_rn(d2.h, rl);
        if (FULL || in[m]) {
          if constexpr (OUT) {
            const size_t g = gk + (size_t)m * nx;
            a.rh_out[g] = rf;
            a.rl_out[g] = __fsub_rn(rl, __fsub_rn(rf, d2.h));
          }
          rmax = fmaxf(rmax, rf);
          rmin = fminf(rmin, rf);
          if constexpr (SING) wr = fmaf(w, rf, wr);
        }
      }
#pragma unroll
      for (int m = 0; m < RPT; ++m) {
        zm[m] = zc[m];
        zc[m] = zp[m];
        bcur[m] = bnext[m];
      }
    }
  };
  if (interior) march(std::true_type{});
  else march(std::false_type{});
  cp_wait<0>();
  resid_reduce<false>(a, rmax, rmin, -INFINITY, INFINITY, wr, df{0.f, 0.f});
}

// Resets the reduction words of r (and of f in pass 0) before a residual pass.
__global__ void reset_red_kernel(int* red, const int* skip, int with_f) {
  if (skip && *skip) return;
  red[0] = f32_key(-INFINITY);
  red[1] = f32_key(INFINITY);
  if (with_f) {
    red[2] = f32_key(-INFINITY);
    red[3] = f32_key(INFINITY);
  }
}

namespace {
// Launch shape of one residual pass: rows per thread, planes per CTA, grid.
struct ResidShape {
  int rpt, zchunk;
  dim3 grid;
};
// which: RS_PASS0 (two-level split), RS_SPLIT3 (three-level), RS_ACC (passes m ≥ 1)
enum { RS_PASS0 = 0, RS_SPLIT3 = 1, RS_ACC = 2 };
ResidShape resid_shape(int nx, int ny, int nz, int which) {
  ResidShape s;
  // rows per thread: more rows share the per-plane work (ring, barriers, addressing);
  // the single-word passes take eight (two CTAs per SM, no spills; measured at 1024³:
  // 3.29 against 3.47 ms with four), the two-level split four (with eight it spills
  // and ran 7.5 against 6.1 ms), three-level cells need the registers of two rows
  s.rpt = which == RS_SPLIT3 ? 2
        : (which == RS_ACC && ny >= 8 * RWARPS) ? 8 : (ny >= 4 * RWARPS ? 4 : 2);
  const int tiles = ((nx + RTX - 1) / RTX) * ((ny + RWARPS * s.rpt - 1) / (RWARPS * s.rpt));
  // about four waves of three CTAs per SM, 8 … 64 planes per CTA
  const long long want = 152LL * (s.rpt >= 8 ? 2 : 3) * 4;
  long long zc = ((long long)nz * tiles) / want;
  zc = zc < 8 ? 8 : (zc > 64 ? 64 : zc);
  s.zchunk = (int)(zc < nz ? zc : nz);
  s.grid = dim3((nx + RTX - 1) / RTX, (ny + RWARPS * s.rpt - 1) / (RWARPS * s.rpt),
                (nz + s.zchunk - 1) / s.zchunk);
  return s;
}
template <int RPT, int KIND>
cudaError_t launch_kind(const ResidArgs& b, dim3 grid, cudaStream_t st) {
  constexpr size_t smem = resid_smem(RPT, (KIND & RK_U32) ? 4 : 8, (KIND & RK_SPLIT3) ? 16 : 8);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(residual_kernel<RPT, KIND>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  residual_kernel<RPT, KIND><<<grid, dim3(RTX, RWARPS), smem, st>>>(b);
  return cudaGetLastError();
}
template <int RPT>
cudaError_t launch_rpt(const ResidArgs& b, int kind, dim3 grid, cudaStream_t st) {
  if (kind & RK_FACE) {  // plans with x or y face unknowns (never singular)
    if constexpr (RPT == 2) {
      switch (kind & ~RK_FACE) {
        case RK_SPLIT3: return launch_kind<RPT, RK_SPLIT3 | RK_FACE>(b, grid, st);
        case RK_SPLIT3 | RK_SHIFT: return launch_kind<RPT, RK_SPLIT3 | RK_SHIFT | RK_FACE>(b, grid, st);
        case RK_SPLIT3 | RK_U32 | RK_FIRST: return launch_kind<RPT, RK_SPLIT3 | RK_U32 | RK_FIRST | RK_FACE>(b, grid, st);
        case RK_SPLIT3 | RK_U32 | RK_FIRST | RK_SHIFT:
          return launch_kind<RPT, RK_SPLIT3 | RK_U32 | RK_FIRST | RK_SHIFT | RK_FACE>(b, grid, st);
        default: break;
      }
    }
    switch (kind & ~RK_FACE) {
      case RK_U32 | RK_FIRST: return launch_kind<RPT, RK_U32 | RK_FIRST | RK_FACE>(b, grid, st);
      case RK_U32 | RK_FIRST | RK_SHIFT: return launch_kind<RPT, RK_U32 | RK_FIRST | RK_SHIFT | RK_FACE>(b, grid, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if constexpr (RPT == 2) {  // the three-level passes run with two rows per thread only
    switch (kind) {
      case RK_SPLIT3: return launch_kind<RPT, RK_SPLIT3>(b, grid, st);
      case RK_SPLIT3 | RK_SHIFT: return launch_kind<RPT, RK_SPLIT3 | RK_SHIFT>(b, grid, st);
      case RK_SPLIT3 | RK_U32 | RK_FIRST | RK_SHIFT:
        return launch_kind<RPT, RK_SPLIT3 | RK_U32 | RK_FIRST | RK_SHIFT>(b, grid, st);
      case RK_SPLIT3 | RK_SING | RK_SUBMU: return launch_kind<RPT, RK_SPLIT3 | RK_SING | RK_SUBMU>(b, grid, st);
      case RK_SPLIT3 | RK_U32 | RK_FIRST: return launch_kind<RPT, RK_SPLIT3 | RK_U32 | RK_FIRST>(b, grid, st);
      case RK_SPLIT3 | RK_U32 | RK_FIRST | RK_SING:
        return launch_kind<RPT, RK_SPLIT3 | RK_U32 | RK_FIRST | RK_SING>(b, grid, st);
      default: break;
    }
  }
  switch (kind) {
    case RK_U32 | RK_FIRST: return launch_kind<RPT, RK_U32 | RK_FIRST>(b, grid, st);
    case RK_U32 | RK_FIRST | RK_SHIFT: return launch_kind<RPT, RK_U32 | RK_FIRST | RK_SHIFT>(b, grid, st);
    case RK_U32 | RK_FIRST | RK_SING: return launch_kind<RPT, RK_U32 | RK_FIRST | RK_SING>(b, grid, st);
    default: return cudaErrorInvalidValue;
  }
}
template <int RPT, int KIND>
cudaError_t launch_acc_kind(const ResidArgs& b, dim3 grid, cudaStream_t st) {
  constexpr size_t smem = (size_t)ADEPTH * acc_cells(RPT) * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(residual_acc_kernel<RPT, KIND>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  residual_acc_kernel<RPT, KIND><<<grid, dim3(RTX, RWARPS), smem, st>>>(b);
  return cudaGetLastError();
}
template <int RPT, int K>
cudaError_t launch_acc_out(const ResidArgs& b, bool out, bool vec, dim3 grid, cudaStream_t st) {
  if (out) return vec ? launch_acc_kind<RPT, K | AK_OUT | AK_VEC>(b, grid, st) : launch_acc_kind<RPT, K | AK_OUT>(b, grid, st);
  return vec ? launch_acc_kind<RPT, K | AK_VEC>(b, grid, st) : launch_acc_kind<RPT, K>(b, grid, st);
}
template <int RPT>
cudaError_t launch_acc_rpt(const ResidArgs& b, int kind, bool out, bool vec, dim3 grid, cudaStream_t st) {
  switch (kind) {
    case 0: return launch_acc_out<RPT, 0>(b, out, vec, grid, st);
    case AK_SING: return launch_acc_out<RPT, AK_SING>(b, out, vec, grid, st);
    case AK_SING | AK_SUBMU: return launch_acc_out<RPT, AK_SING | AK_SUBMU>(b, out, vec, grid, st);
    default: return cudaErrorInvalidValue;
  }
}
// Passes m ≥ 1: same grid as the two-level passes (the finalize sums that many partials).
cudaError_t launch_resid_acc(const ResidArgs& b0, int pass, cudaStream_t st) {
  reset_red_kernel<<<1, 1, 0, st>>>(b0.red, b0.skip, 0);
  const ResidShape s = resid_shape(b0.nx, b0.ny, b0.nz, RS_ACC);
  ResidArgs b = b0;
  b.zchunk = s.zchunk;
  const int kind = b.singular ? (AK_SING | (pass == 1 ? AK_SUBMU : 0)) : 0;
  const bool out = b.rh_out != nullptr, vec = (b.nx % 4) == 0;
  return s.rpt == 8 ? launch_acc_rpt<8>(b, kind, out, vec, s.grid, st)
       : s.rpt == 4 ? launch_acc_rpt<4>(b, kind, out, vec, s.grid, st)
                    : launch_acc_rpt<2>(b, kind, out, vec, s.grid, st);
}
cudaError_t launch_resid(const ResidArgs& b0, int kind, int reset_f, cudaStream_t st) {
  reset_red_kernel<<<1, 1, 0, st>>>(b0.red, b0.skip, reset_f);
  if (b0.bcx == BC_FD || b0.bcy == BC_FD) kind |= RK_FACE;
  const ResidShape s = resid_shape(b0.nx, b0.ny, b0.nz, (kind & RK_SPLIT3) ? RS_SPLIT3 : RS_PASS0);
  ResidArgs b = b0;
  b.zchunk = s.zchunk;
  return s.rpt == 4 ? launch_rpt<4>(b, kind, s.grid, st) : launch_rpt<2>(b, kind, s.grid, st);
}
}  // namespace

int residual_blocks(int nx, int ny, int nz, int which) {
  const ResidShape s = resid_shape(nx, ny, nz, which);
  return (int)(s.grid.x * s.grid.y * s.grid.z);
}

cudaError_t launch_residual_inc(const ResidArgs& a, int pass, int split3, cudaStream_t st) {
  if (!a.u || (pass > 0 && (!a.rh_in || !a.rl_in)) || (!a.rh_out != !a.rl_out) || (split3 && pass))
    return cudaErrorInvalidValue;
  if (pass > 0) {
    if (!a.zres) return cudaErrorInvalidValue;
    return launch_resid_acc(a, pass, st);
  }
  int kind = RK_U32 | RK_FIRST | (split3 ? RK_SPLIT3 : 0) | (a.nalpha.h != 0.f ? RK_SHIFT : 0);
  if (a.singular) kind |= RK_SING;
  if (a.singular && pass == 1) kind |= RK_SUBMU;
  return launch_resid(a, kind, pass == 0, st);
}

cudaError_t launch_residual_exact(const ResidArgs& a, cudaStream_t st) {
  if (!a.p || !a.r) return cudaErrorInvalidValue;
  return launch_resid(a, RK_SPLIT3 | (a.singular ? (RK_SING | RK_SUBMU) : 0) | (a.nalpha.h != 0.f ? RK_SHIFT : 0),
                      0, st);
}

namespace {
// Σ over the per-block partials of (Δz^f·r, Δz^f·f) in double-float, one CTA;
// thread 0 gets them in FP64.
__device__ void sum_partials(const float* partial, int nblocks, double& sr_out, double& sf_out) {
  __shared__ df sr[32], sf[32];
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
  __syncthreads();
  double s1 = 0.0, s2 = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s1 += (double)sr[w].h + (double)sr[w].l;
      s2 += (double)sf[w].h + (double)sf[w].l;
    }
  sr_out = s1;
  sf_out = s2;
}
__device__ double bits_f64(unsigned long long b) { return __longlong_as_double((long long)b); }
}  // namespace

// One CTA after each pass of the refinement loop: weighted means (singular),
// norms, the drift bound, the convergence test, the confirmation decision and
// the info record.
//
// Pass 0 first runs with the two-level split, whose evaluation error is about
// 2^-44·‖A‖∞·max|Φ_0| (bounded here by 2^-43·…). Every later residual inherits it,
// so if that bound exceeds 5 % of rtol·‖f_c‖∞ this finalize (attempt 0) decides
// nothing and asks for pass 0 again with the three-level split (attempt 1).
//
// Drift bound: pass m ≥ 1 evaluates r_{m−1} − A·e_{m−1} instead of f − A·Φ_m. It
// differs from a fresh evaluation from the stored Φ_m by the evaluation error of
// A·e_{m−1} (≤ 2^-39·‖A‖∞·max|e|, the single-word accumulation) and by the FP64 rounding of Φ += e
// (≤ 2^-52·‖A‖∞·max|Φ|). If the accumulated bound exceeds 5 % of rtol·‖f_c‖∞ when
// the loop ends (converged or not), the exact pass at the end re-evaluates the
// residual from the stored Φ and decides.
__global__ void __launch_bounds__(1024) finalize_kernel(Ctrl* c, const float* partial, int nblocks,
                                                        double wsum_total, int singular, double rtol,
                                                        int iteration, int attempt, int last,
                                                        double anorm, const int* skip, ps_info* info) {
  if ((skip && *skip) || c->converged) return;
  double s1 = 0.0, s2 = 0.0;
  if (singular) sum_partials(partial, nblocks, s1, s2);
  if (threadIdx.x != 0) return;
  double mr = 0.0, mf = 0.0;
  if (singular) {
    mr = s1 / wsum_total;
    if (iteration == 0) {  // μ_f is measured once, in pass 0
      mf = s2 / wsum_total;
      c->mf = mf;
      const float h = (float)mf;
      c->mu[0] = h;
      c->mu[1] = (float)(mf - (double)h);
    } else {
      mf = c->mf;
    }
  }
  if (iteration > 0)
    c->bnd += anorm * (ldexp(bits_f64(c->dmax), -39) + ldexp(bits_f64(c->pmax), -52));
  c->dmax_prev = c->dmax;  // the scale of the output repeat of this pass
  c->dmax = 0;             // the next correction's x backward records max|e| here
  const double rmax = key_f32(c->red[0]), rmin = key_f32(c->red[1]);
  const double vfmax = key_f32(c->red[2]), vfmin = key_f32(c->red[3]);
  const double rn = fmax(rmax - mr, mr - rmin);
  const double fn = fmax(vfmax - mf, mf - vfmin);
  const double rel = fn > 0 ? rn / fn : (rn > 0 ? INFINITY : 0.0);
  if (iteration == 0 && attempt == 0) {
    const bool redo = ldexp(anorm * bits_f64(c->pmax), -43) > 0.05 * rtol * fn;
    c->skip_redo = redo ? 0 : 1;
    c->nomat0 = 1;
    if (redo) return;
  }
  c->rnorm = rn;
  c->fnorm = fn;
  c->rel = rel;
  c->iterations = iteration;
  const bool ok = rel <= rtol;
  if (ok) c->converged = 1;
  if (ok || last) c->vskip = (c->bnd <= 0.05 * rtol * fn) ? 1 : 0;
  if (iteration == 0) c->nomat0 = (ok || last) ? 0 : 1;
  c->skip_out = (ok || last) ? 1 : 0;
  if (info && (ok || last)) {
    info->status = ok ? PS_OK : PS_NOT_CONVERGED;
    info->iterations = iteration;
    info->rel_residual = rel;
    info->r_norm = rn;
    info->f_norm = fn;
  }
}

// One CTA after the exact confirmation pass (which runs only when the drift
// bound was not small): its residual decides the status.
__global__ void __launch_bounds__(1024) finalize_exact_kernel(Ctrl* c, const float* partial, int nblocks,
                                                              double wsum_total, int singular,
                                                              double rtol, ps_info* info) {
  if (c->vskip) return;
  double s1 = 0.0, s2 = 0.0;
  if (singular) sum_partials(partial, nblocks, s1, s2);
  if (threadIdx.x != 0) return;
  const double mr = singular ? s1 / wsum_total : 0.0, mf = singular ? c->mf : 0.0;
  const double rmax = key_f32(c->red[0]), rmin = key_f32(c->red[1]);
  const double vfmax = key_f32(c->red[2]), vfmin = key_f32(c->red[3]);
  const double rn = fmax(rmax - mr, mr - rmin);
  const double fn = fmax(vfmax - mf, mf - vfmin);
  const double rel = fn > 0 ? rn / fn : (rn > 0 ? INFINITY : 0.0);
  const bool ok = rel <= rtol;
  c->rnorm = rn;
  c->rel = rel;
  if (info) {
    info->status = ok ? PS_OK : PS_NOT_CONVERGED;
    info->iterations = c->iterations;
    info->rel_residual = rel;
    info->r_norm = rn;
    info->f_norm = fn;
  }
}

cudaError_t launch_finalize(Ctrl* ctrl, const float* partial, int nblocks, double wsum_total,
                            int singular, double rtol, int iteration, int attempt, int last,
                            double anorm, const int* skip, ps_info* info, cudaStream_t st) {
  finalize_kernel<<<1, 1024, 0, st>>>(ctrl, partial, nblocks, wsum_total, singular, rtol, iteration,
                                      attempt, last, anorm, skip, info);
  return cudaGetLastError();
}

cudaError_t launch_finalize_exact(Ctrl* ctrl, const float* partial, int nblocks, double wsum_total,
                                  int singular, double rtol, ps_info* info, cudaStream_t st) {
  finalize_exact_kernel<<<1, 1024, 0, st>>>(ctrl, partial, nblocks, wsum_total, singular, rtol, info);
  return cudaGetLastError();
}

__global__ void widen_kernel(const float* __restrict__ u, double* __restrict__ p, size_t n, const int* skip) {
  if (*skip) return;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < n; g += (size_t)gridDim.x * blockDim.x)
    p[g] = widen_f32(u[g]);
}

cudaError_t launch_widen(const float* u, double* p, size_t n, const int* skip, cudaStream_t st) {
  widen_kernel<<<152 * 8, 256, 0, st>>>(u, p, n, skip);
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
