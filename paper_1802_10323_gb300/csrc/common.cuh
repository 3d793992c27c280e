// common.cuh — device helpers shared by the solver's kernels.
//
// * cplx<T>: a plain complex pair for the shared-memory FFTs.
// * Integer-only FP64 <-> FP32 conversions. On this part both F2F directions
//   and every FP64 add/multiply issue at the FP64 rate (~2 per clock per SM,
//   1/64 of FP32), so the FP32 paths never use `cvt` or FP64 arithmetic on the
//   bulk data: widening and narrowing are done on the IEEE bit patterns.
// * Double-float ("df") arithmetic: an unevaluated sum hi + lo of two floats
//   with ~48 significant bits, built from Knuth's TwoSum and the FMA-based
//   exact product (Dekker/Ogita–Rump–Oishi). Used for the refinement residual.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

template <class T>
struct cplx {
  T x, y;
};

template <class T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <class T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T>
__device__ __forceinline__ cplx<T> conj_(cplx<T> a) { return {a.x, -a.y}; }
template <class T>
__device__ __forceinline__ cplx<T> mul_i(cplx<T> a) { return {-a.y, a.x}; }       // i·a
template <class T>
__device__ __forceinline__ cplx<T> mul_mi(cplx<T> a) { return {a.y, -a.x}; }      // −i·a
template <class T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return {a.x * s, a.y * s}; }

// ---- FP64 <-> FP32 on bit patterns ---------------------------------------

// Exact widening. Subnormal floats flush to signed zero; inf/nan map to inf/nan.
__device__ __forceinline__ double widen_f32(float f) {
  uint32_t b = __float_as_uint(f);
  uint32_t s = b & 0x80000000u;
  uint32_t e = (b >> 23) & 0xFFu;
  uint32_t m = b & 0x7FFFFFu;
  uint32_t hi = s | ((e + 896u) << 20) | (m >> 3);
  uint32_t lo = m << 29;
  hi = (e == 0u) ? s : hi;
  lo = (e == 0u) ? 0u : lo;
  hi = (e == 0xFFu) ? (s | 0x7FF00000u | (m >> 3)) : hi;
  return __hiloint2double((int)hi, (int)lo);
}

// Narrowing with round-half-away-from-zero on the 24th bit. Values below the
// float normal range flush to signed zero; values above it give infinity.
__device__ __forceinline__ float narrow_f64(double d) {
  uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  uint32_t s = hi & 0x80000000u;
  int e = (int)((hi >> 20) & 0x7FFu) - 896;
  uint32_t mag = ((uint32_t)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  mag += (lo >> 28) & 1u;  // carry may ripple into the exponent, as it should
  mag = (e <= 0) ? 0u : mag;
  mag = (e >= 255 || mag >= 0x7F800000u) ? 0x7F800000u : mag;
  return __uint_as_float(s | mag);
}

// Split d into hi + lo: hi = d truncated to 24 significant bits, lo = the
// remainder (same sign) rounded toward zero to 24 bits. |d − hi − lo| ≤ 2^-47 |d|
// for |d| ≥ 2^-74; smaller magnitudes are flushed (absolute error < 2^-74).
// hi: the exponent rebiased (1023 → 127) and the top 23 fraction bits taken with
// one 64-bit funnel shift; zero below the float normal range. lo: the remaining 29
// fraction bits, whose unit is 2^(E−52) for the exponent E of d (and of hi), i.e.
// hi's exponent field minus 52 (zero when that is below the float normal range).
__device__ __forceinline__ void split_f64(double d, float& h, float& l) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t s = hi & 0x80000000u;
  const uint32_t mag = __funnelshift_l(lo, hi - (896u << 20), 3) & 0x7FFFFFFFu;
  const bool normal = (hi & 0x7FF00000u) > (896u << 20);
  const uint32_t hb = normal ? (s | mag) : s;
  h = __uint_as_float(hb);
  const int eb = (int)(hb & 0x7F800000u) - (52 << 23);
  const float scale = __int_as_float(eb > 0 ? eb : 0);
  const float lf = __uint2float_rz(lo & 0x1FFFFFFFu) * scale;
  l = __uint_as_float(__float_as_uint(lf) | s);
}

// ---- double-float arithmetic ------------------------------------------------

struct df {
  float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {  // needs |a| ≥ |b| or a == 0
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.h, b.h);
  float t = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return quick_two_sum(s.h, t);
}
__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_from_f64(double d) {
  df r;
  split_f64(d, r.h, r.l);
  return r;
}
__device__ __forceinline__ float df_to_f32(df a) { return __fadd_rn(a.h, a.l); }

// Wall clock (ns) and an acquire load at GPU scope, for the bounded waits of the
// persistent kernels (a consumer waits on a completion counter of earlier tasks).
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Order-preserving int key of a float (for atomicMax/atomicMin on signed values).
__device__ __forceinline__ int f32_key(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : (i ^ 0x7FFFFFFF);
}
__host__ __device__ inline float key_f32(int k) {
  int i = k >= 0 ? k : (k ^ 0x7FFFFFFF);
  float f;
#ifdef __CUDA_ARCH__
  f = __int_as_float(i);
#else
  union { int i; float f; } u;
  u.i = i;
  f = u.f;
#endif
  return f;
}

// ---- type-directed load/store conversions -------------------------------------

template <class TC, class TI>
struct ld_cvt;
template <>
struct ld_cvt<float, float> {
  static __device__ __forceinline__ float f(float v) { return v; }
};
template <>
struct ld_cvt<double, double> {
  static __device__ __forceinline__ double f(double v) { return v; }
};
template <>
struct ld_cvt<float, double> {
  static __device__ __forceinline__ float f(double v) { return narrow_f64(v); }
};

template <class TO, class TC>
struct st_cvt;
template <>
struct st_cvt<float, float> {
  static __device__ __forceinline__ float f(float v) { return v; }
};
template <>
struct st_cvt<double, double> {
  static __device__ __forceinline__ double f(double v) { return v; }
};
template <>
struct st_cvt<double, float> {
  static __device__ __forceinline__ double f(float v) { return widen_f32(v); }
};
