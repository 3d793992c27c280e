// xform_long.cu — line transforms of n = 2M reals with M ∈ {1024, 2048, 4096}
// (lines of 2048, 4096 and 8192 cells), and the plane transpose that turns
// y lines of those lengths into x lines.
//
// Same mathematics as every other transform unit (one M-point complex FFT per
// line with the Table 2 pre/post processing per BC; see xform_dev.cuh), laid out
// for lines too long for the register-resident kernels:
//   * one CTA of M/16 threads per line, persistent over lines; the line is
//     loaded and stored with coalesced accesses through a shared real buffer;
//   * the M-point FFT in three Stockham stages of radix 16, 16 and M/256, each
//     thread holding 16 complex points in registers; between stages the points
//     pass through a shared complex buffer (one pad slot per 16 entries);
//   * the twiddles come from small shared tables laid out so that the 32 lanes of
//     a warp read consecutive entries or one broadcast entry (no bank conflicts):
//     stage 1 a [r][k] table, stage 2 the product of [r][k mod 16] and
//     [r][k div 16] tables, the pre/post-processing factors e^{−2πi·ck/(8n)}
//     (c = 2, 4, 8) products of [k mod 64] and [k div 64] tables; the real line
//     is padded by one float per 32 so that stride-2 and stride-4 accesses are
//     conflict-free too;
//   * the forward pre-processing gathers the first stage's operands straight from
//     the real buffer, and the backward post-processing writes the last stage's
//     outputs straight to it.
// y lines (strided by n_x) are transposed plane by plane into a scratch array,
// transformed as x lines there and transposed back: the x↔y transposes of the
// pencil algorithm (§3) as in-HBM tiled transposes, two extra passes over the
// data, instead of strided loads that would fetch one 32-byte sector per value.
#include "xform_units.cuh"

// threads per SM the FP32 kernels are compiled for (their register cap)
#ifndef PS_LONG_THREADS
#define PS_LONG_THREADS 1024
#endif

namespace ps {
namespace lng {

template <int M>
struct LShape {
  static constexpr int E = 16;       // complex points per thread
  static constexpr int NT = M / E;   // threads per line (= per CTA)
  static constexpr int NST = 3;
  __host__ __device__ static constexpr int radix(int s) { return s < 2 ? 16 : M / 256; }
};

__host__ __device__ constexpr int lpad(int i) { return i + (i >> 4); }   // complex buffer

// Twiddle tables of one CTA (every entry a value of the 8n-entry table
// e^{−2πi t/(8n)}, so exact up to one complex product where two are combined):
// in shared memory, and the coarse factors of the pre/post-processing straight
// from the global table (at most two distinct entries per warp, L1-resident).
template <class T, int M>
struct LTab {
  static constexpr int R2 = M / 256;        // radix of the last stage
  static constexpr int ENTRIES = 256 + 2 * 16 * R2 + 3 * 64;
  cplx<T>* s1;   // [16][16]: ω_M^(r·k·M/256), stage 1 (k < 16)
  cplx<T>* s2a;  // [R2][16]: ω_M^(r·(k mod 16)), stage 2 (k < 256)
  cplx<T>* s2b;  // [R2][16]: ω_M^(16·r·(k div 16))
  cplx<T>* lo;   // [3][64]: e^{−2πi·c·(k mod 64)/(8n)}, c = 2, 4, 8
  const cplx<T>* tw;  // the global table (8n = 16M entries; ω_M^t = tw[16t])
  __device__ void carve(cplx<T>* base, const cplx<T>* tw_) {
    s1 = base;
    s2a = s1 + 256;
    s2b = s2a + 16 * R2;
    lo = s2b + 16 * R2;
    tw = tw_;
  }
  __device__ void fill(int tid, int nt) {  // all threads of the CTA
    for (int i = tid; i < 256; i += nt) s1[i] = tw[16 * (((i >> 4) * (i & 15) * (M / 256)) & (M - 1))];
    for (int i = tid; i < 16 * R2; i += nt) {
      const int r = i >> 4, j = i & 15;
      s2a[i] = tw[16 * ((r * j) & (M - 1))];
      s2b[i] = tw[16 * ((16 * r * j) & (M - 1))];
    }
    for (int i = tid; i < 3 * 64; i += nt) lo[i] = tw[(2 << (i >> 6)) * (i & 63)];
  }
  // e^{−2πi·c·k/(8n)} for c = 2 (ci 0), 4 (ci 1), 8 (ci 2); 0 ≤ k ≤ M
  __device__ __forceinline__ cplx<T> pp(int ci, int k) const {
    const int c = 2 << ci;
    const cplx<T>* h = tw + ((c * 64 * (k >> 6)) & (16 * M - 1));
    cplx<T> hv;
    if constexpr (sizeof(T) == 4) {
      const float2 t2 = __ldg(reinterpret_cast<const float2*>(h));
      hv = {t2.x, t2.y};
    } else {
      const double2 t2 = __ldg(reinterpret_cast<const double2*>(h));
      hv = {t2.x, t2.y};
    }
    return cmul(lo[64 * ci + (k & 63)], hv);
  }
};

// Stages STAGE… of the M-point FFT of this thread's line (the Stockham indexing of
// the column unit, one line per CTA). On entry v[q·R + r] = x[b_q + r·M/R] with
// b_q = b + q·NT; on return v[q·R + r] holds the output at b_q + r·(M/R_last).
// ω_M^t = e^{−2πi·16t/(8n)}.
template <class T, int M, bool INV, int STAGE, int NS>
__device__ __forceinline__ void fft_line(cplx<T> (&v)[16], cplx<T>* buf, const LTab<T, M>& tb, int b) {
  using S = LShape<M>;
  constexpr int E = S::E, NT = S::NT;
  constexpr int R = S::radix(STAGE);
  static_assert(STAGE == 0 || (STAGE == 1 && NS == 16 && R == 16) || (STAGE == 2 && NS == 256), "stage tables");
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
    const int bq = b + q * NT;
    if constexpr (STAGE > 0) {
      const int k = bq & (NS - 1);  // twiddle ω_M^(r·k·M/(NS·R))
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w;
        if constexpr (STAGE == 1) w = tb.s1[16 * r + k];
        else w = cmul(tb.s2a[16 * r + (k & 15)], tb.s2b[16 * r + (k >> 4)]);
        if (INV) w.y = -w.y;
        v[q * R + r] = cmul(v[q * R + r], w);
      }
    }
    col::dft<T, R, INV>(&v[q * R]);
  }
  if constexpr (STAGE + 1 < S::NST) {
    constexpr int R2 = S::radix(STAGE + 1);
    __syncthreads();  // earlier readers of buf are done
#pragma unroll
    for (int q = 0; q < E / R; ++q) {
      const int bq = b + q * NT;
      const int o = (bq / NS) * NS * R + (bq & (NS - 1));
#pragma unroll
      for (int r = 0; r < R; ++r) buf[lpad(o + r * NS)] = v[q * R + r];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E / R2; ++q) {
      const int bq = b + q * NT;
#pragma unroll
      for (int r = 0; r < R2; ++r) v[q * R2 + r] = buf[lpad(bq + r * (M / R2))];
    }
    fft_line<T, M, INV, STAGE + 1, NS * R>(v, buf, tb, b);
  }
}

template <class T, int M>
__host__ __device__ constexpr size_t long_smem() {
  // twiddle tables and the complex exchange buffer (padded)
  return (size_t)LTab<T, M>::ENTRIES * sizeof(cplx<T>) + (size_t)(lpad(M) + 1) * sizeof(cplx<T>);
}

// Makhoul index map (as xform_dev.cuh): position j of v ↔ position of a.
__device__ __forceinline__ int mk(int j, int n, int m) { return j < m ? 2 * j : 2 * n - 1 - 2 * j; }

// a.nlines lines of n = 2M contiguous reals; line ln belongs to plane ln / a.ny
// (for the per-plane scale). Output modes as the row kernels (FastArgs). The first
// stage's operands are read straight from the line in global memory (each lane a
// consecutive pair or a mirrored position, so a warp's loads cover contiguous
// 256-byte spans), and the post-processing writes each output value straight to
// global memory: the only shared buffer is the complex exchange of the FFT. All
// reads of a line happen before the first stage's barrier and all writes after
// the last, so in == out is safe.
template <class T, class TI, class TO, int M, bool FWD, int OM>
__global__ void __launch_bounds__(LShape<M>::NT, (sizeof(T) == 8 ? 256 : PS_LONG_THREADS) / LShape<M>::NT)
    xform_long_kernel(FastArgs<T> a) {
  using S = LShape<M>;
  constexpr int N = 2 * M, NT = S::NT, E = S::E, RL = S::radix(S::NST - 1);
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LTab<T, M> tb;
  tb.carve(reinterpret_cast<cplx<T>*>(smem_raw), a.tw);
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw) + LTab<T, M>::ENTRIES;  // [lpad(M) + 1]
  const int b = threadIdx.x;
  tb.fill(b, NT);
  __syncthreads();  // the tables are complete before the first line's gather reads them
  const cplx<T> tw1 = a.tw[1];  // e^{−2πi/(8n)}: the ND post-twiddle is tw(4k)·tw1
  const int bc = a.bc;
  // no __restrict__: in and out may be the same array
  const TI* in = static_cast<const TI*>(a.in);
  TO* out = static_cast<TO*>(a.out);
  T tmax = (T)0;  // max |new value| before widening (the bits of its widening order as the values)
  for (int ln = blockIdx.x; ln < a.nlines; ln += gridDim.x) {
    const size_t g0 = (size_t)ln * N;
    const int z = ln / a.ny;
    {  // ask L2 for this CTA's next line, so that its loads do not wait on HBM
      const int nl = ln + gridDim.x;
      if (nl < a.nlines) {
        const char* nb = reinterpret_cast<const char*>(in + (size_t)nl * N);
        for (int o = b * 128; o < N * (int)sizeof(TI); o += NT * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(nb + o));
      }
    }
    if constexpr (!FWD && sizeof(TO) == 8 && (OM == row::OM_BASE || OM == row::OM_ACC)) {
      // the operand of the output stage (the FP32 base, or the FP64 output accumulated
      // into) is read only after the transform: ask L2 for it now
      const char* ob = (OM == row::OM_BASE) ? reinterpret_cast<const char*>(a.base32 + g0)
                                            : reinterpret_cast<const char*>(out + g0);
      const int obytes = N * ((OM == row::OM_BASE) ? 4 : 8);
      for (int o = b * 128; o < obytes; o += NT * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(ob + o));
    }
    const TI* src = in + g0;
    const T sci = (FWD && a.plane_scale) ? a.plane_scale[z] : (T)1;
    const T sco = (!FWD && a.plane_scale) ? a.plane_scale[z] : (T)1;
    // the line is read once: evict-first loads, so that the twiddle table stays in L1
    auto X = [&](int e) -> T { return ld_cvt<T, TI>::f(__ldcs(src + e)) * sci; };
    // a consecutive pair (e even): one 8- or 16-byte load
    auto X2 = [&](int e) -> cplx<T> {
      if constexpr (sizeof(TI) == 4) {
        const float2 q = __ldcs(reinterpret_cast<const float2*>(src + e));
        return {ld_cvt<T, TI>::f(q.x) * sci, ld_cvt<T, TI>::f(q.y) * sci};
      } else {
        const double2 q = __ldcs(reinterpret_cast<const double2*>(src + e));
        return {ld_cvt<T, TI>::f(q.x) * sci, ld_cvt<T, TI>::f(q.y) * sci};
      }
    };
    // one output value at position e of the line, in the output mode OM of the row
    // kernels (plane scale; FP64 out: stored, accumulated, or a widened FP32 base plus
    // the value, or none, with the FP32 copy and the max-abs of the new values; T out:
    // stored or accumulated). The mode is a template argument, so each instance
    // carries only its own store path.
    auto emit = [&](int e, T val) {
      const size_t g = g0 + e;
      const T vs = val * sco;
      if constexpr (sizeof(TO) == 8) {
        const TO d = st_cvt<TO, T>::f(vs);
        tmax = fmax(tmax, fabs(vs));
        if constexpr (OM == row::OM_BASE && sizeof(T) == 4) out[g] = widen_f32(a.base32[g]) + d;
        else if constexpr (OM == row::OM_ACC) out[g] = out[g] + d;
        else if constexpr (OM == row::OM_STORE) out[g] = d;
        if constexpr (sizeof(T) == 4)
          if (a.out2) a.out2[g] = vs;
      } else {
        TO x = st_cvt<TO, T>::f(vs);
        if constexpr (OM == row::OM_ACC) x = out[g] + x;
        __stcs(out + g, x);
      }
    };
    // two consecutive output values (e even): the same with 8- and 16-byte accesses
    auto emit2 = [&](int e, T val0, T val1) {
      const size_t g = g0 + e;
      const T s0 = val0 * sco, s1 = val1 * sco;
      if constexpr (sizeof(TO) == 8) {
        const TO d0 = st_cvt<TO, T>::f(s0), d1 = st_cvt<TO, T>::f(s1);
        tmax = fmax(tmax, fmax(fabs(s0), fabs(s1)));
        if constexpr (OM == row::OM_BASE && sizeof(T) == 4) {
          const float2 q = *reinterpret_cast<const float2*>(a.base32 + g);
          *reinterpret_cast<double2*>(out + g) = make_double2(widen_f32(q.x) + d0, widen_f32(q.y) + d1);
        } else if constexpr (OM == row::OM_ACC) {
          const double2 q = *reinterpret_cast<const double2*>(out + g);
          *reinterpret_cast<double2*>(out + g) = make_double2(q.x + d0, q.y + d1);
        } else if constexpr (OM == row::OM_STORE) {
          *reinterpret_cast<double2*>(out + g) = make_double2(d0, d1);
        }
        if constexpr (sizeof(T) == 4)
          if (a.out2) *reinterpret_cast<float2*>(a.out2 + g) = make_float2(s0, s1);
      } else {
        TO x0 = st_cvt<TO, T>::f(s0), x1 = st_cvt<TO, T>::f(s1);
        if constexpr (OM == row::OM_ACC) {
          x0 = out[g] + x0;
          x1 = out[g + 1] + x1;
        }
        if constexpr (sizeof(TO) == 4) __stcs(reinterpret_cast<float2*>(out + g), make_float2(x0, x1));
        else __stcs(reinterpret_cast<double2*>(out + g), make_double2(x0, x1));
      }
    };
    cplx<T> v[E];
    if (FWD) {
      // ---- pre-processing gathered into the first stage's operands z_p, p = b + r·NT ----
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int p = b + r * NT;
        cplx<T> zz;
        if (bc == BC_P) {
          zz = X2(2 * p);
        } else if (bc_iv(bc)) {  // DN: the reversed line, the two reals swap
          const T e0 = X(2 * p), e1 = X(N - 1 - 2 * p);
          zz = cmul(bc == BC_DN ? cplx<T>{e1, e0} : cplx<T>{e0, e1}, tb.pp(1, p));
        } else {
          const int j0 = 2 * p, j1 = 2 * p + 1;
          T v0 = X(mk(j0, N, M)), v1 = X(mk(j1, N, M));
          if (bc == BC_DD) {
            if (j0 >= M) v0 = -v0;
            if (j1 >= M) v1 = -v1;
          }
          zz = {v0, v1};
        }
        v[r] = zz;
      }
      __syncthreads();  // the previous line's buffer reads are done
      fft_line<T, M, false, 0, 1>(v, buf, tb, b);
      // ---- post-processing: pair k with M − k through the complex buffer ----
      __syncthreads();
#pragma unroll
      for (int q = 0; q < E / RL; ++q)
#pragma unroll
        for (int r = 0; r < RL; ++r) buf[lpad(b + q * NT + r * (M / RL))] = v[q * RL + r];
      __syncthreads();
      if (bc_iv(bc)) {
#pragma unroll 4
        for (int k = b; k < M; k += NT) {
          const cplx<T> c = cmul(cmul(tb.pp(1, k), tw1), buf[lpad(k)]);
          emit(2 * k, (T)2 * c.x);
          emit(N - 1 - 2 * k, (T)-2 * c.y);
        }
      } else {
#pragma unroll 4
        for (int k = b; k <= M / 2; k += NT) {
          const cplx<T> Zk = buf[lpad(k)], Zmk = buf[lpad(k == 0 ? 0 : M - k)];
          const cplx<T> Ek = cscale(cadd(Zk, conj_(Zmk)), (T)0.5);
          const cplx<T> Ok = cscale(mul_mi(csub(Zk, conj_(Zmk))), (T)0.5);
          const cplx<T> B = cmul(tb.pp(2, k), Ok);
          const cplx<T> Vk = cadd(Ek, B), Vmk = conj_(csub(Ek, B));  // k = 0: Vmk is V_M
          if (bc == BC_P) {
            if (k == 0) {
              emit(0, Vk.x);
              emit(N - 1, Vmk.x);
            } else {
              emit(2 * k - 1, Vk.x);
              emit(2 * k, -Vk.y);
              if (2 * k != M) {
                emit(2 * (M - k) - 1, Vmk.x);
                emit(2 * (M - k), -Vmk.y);
              }
            }
          } else {
            const bool rev = (bc == BC_DD);
            auto put = [&](int qq, T val) { emit(rev ? (N - 1 - qq) : qq, val); };
            if (k == 0) {
              put(0, (T)2 * Vk.x);
              put(M, (T)1.41421356237309504880 * Vmk.x);
            } else {
              const cplx<T> c1 = cmul(tb.pp(0, k), Vk);
              put(k, (T)2 * c1.x);
              put(N - k, (T)-2 * c1.y);
              if (2 * k != M) {
                const cplx<T> c2 = cmul(tb.pp(0, M - k), Vmk);
                put(M - k, (T)2 * c2.x);
                put(M + k, (T)-2 * c2.y);
              }
            }
          }
        }
      }
    } else {
      // ---- backward pre-processing: reals → the M complex points (pairs k, M − k) ----
      __syncthreads();  // the previous line's buffer reads are done
      if (bc_iv(bc)) {
#pragma unroll 4
        for (int k = b; k < M; k += NT) buf[lpad(k)] = cmul(cplx<T>{X(2 * k), X(N - 1 - 2 * k)}, tb.pp(1, k));
      } else {
#pragma unroll 4
        for (int k = b; k <= M / 2; k += NT) {
          cplx<T> Vk, Vmk;
          if (bc == BC_P) {
            if (k == 0) {
              Vk = {X(0), (T)0};
              Vmk = {X(N - 1), (T)0};
            } else {
              Vk = {X(2 * k - 1), -X(2 * k)};
              Vmk = {X(2 * (M - k) - 1), -X(2 * (M - k))};
            }
          } else {
            // DCT-III via Makhoul: V_q = e^{+iπq/2n} (X_q − i X_{n−q}) / 2, X_n = 0;
            // DST-III: the same on Y_q = X_{n−1−q}
            const bool rev = (bc == BC_DD);
            auto XQ = [&](int qq) { return qq >= N ? (T)0 : X(rev ? (N - 1 - qq) : qq); };
            cplx<T> w = tb.pp(0, k);
            w.y = -w.y;
            Vk = cscale(cmul(w, cplx<T>{XQ(k), -XQ(N - k)}), (T)0.5);
            cplx<T> w2 = tb.pp(0, M - k);
            w2.y = -w2.y;
            Vmk = cscale(cmul(w2, cplx<T>{XQ(M - k), -XQ(N - (M - k))}), (T)0.5);
          }
          // E_k = (V_k + conj V_{M−k})/2, O_k = (V_k − conj V_{M−k}) e^{+2πik/n}/2
          const cplx<T> Ek = cscale(cadd(Vk, conj_(Vmk)), (T)0.5);
          cplx<T> wn = tb.pp(2, k);
          wn.y = -wn.y;
          const cplx<T> Ok = cscale(cmul(csub(Vk, conj_(Vmk)), wn), (T)0.5);
          if (k < M) buf[lpad(k)] = cadd(Ek, mul_i(Ok));
          if (k != 0 && 2 * k != M) buf[lpad(M - k)] = cadd(conj_(Ek), mul_i(conj_(Ok)));
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < E; ++r) v[r] = buf[lpad(b + r * NT)];
      if (bc_iv(bc)) fft_line<T, M, false, 0, 1>(v, buf, tb, b);  // DCT-IV is its own inverse
      else fft_line<T, M, true, 0, 1>(v, buf, tb, b);
      // ---- backward post-processing straight from the last stage to the line ----
      const T inv_m = (T)1 / (T)M;
#pragma unroll
      for (int q = 0; q < E / RL; ++q) {
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int k = b + q * NT + r * (M / RL);
          const cplx<T> zk = v[q * RL + r];
          if (bc_iv(bc)) {
            const T s = (T)1 / (T)N;  // 2·(1/2n)
            const cplx<T> c = cmul(cmul(tb.pp(1, k), tw1), zk);
            const T A = s * c.x, B = -s * c.y;  // DN: the two outputs trade places
            emit(2 * k, (bc == BC_DN) ? B : A);
            emit(N - 1 - 2 * k, (bc == BC_DN) ? A : B);
          } else if (bc == BC_P) {
            emit2(2 * k, zk.x * inv_m, zk.y * inv_m);
          } else {
            const int i0 = mk(2 * k, N, M), i1 = mk(2 * k + 1, N, M);
            T v0 = zk.x * inv_m, v1 = zk.y * inv_m;
            if (bc == BC_DD) {
              if (i0 & 1) v0 = -v0;
              if (i1 & 1) v1 = -v1;
            }
            emit(i0, v0);
            emit(i1, v1);
          }
        }
      }
    }
  }
  if constexpr (sizeof(TO) == 8) {
    if (a.amax) {
      for (int o = 16; o > 0; o >>= 1) tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
      const unsigned long long amax = (unsigned long long)__double_as_longlong(st_cvt<double, T>::f(tmax));
      if ((threadIdx.x & 31) == 0 && amax) atomicMax(a.amax, amax);
    }
  }
}

// Transpose of every z plane: src [n_z][rows][cols] → dst [n_z][cols][rows], tiles of
// 64 × 64 through shared memory (one pad column), 32 × 8 threads, each moving pairs of
// consecutive values (8- or 16-byte accesses: rows and cols are even) in eight rows.
template <class T>
__global__ void __launch_bounds__(256) transpose_kernel(const T* __restrict__ src, T* __restrict__ dst, int rows,
                                                        int cols, const int* skip) {
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char tsm[];
  T(*tile)[65] = reinterpret_cast<T(*)[65]>(tsm);  // [64][65]
  const int c0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
  const size_t plane = (size_t)rows * cols;
  const T* s = src + (size_t)blockIdx.z * plane;
  T* d = dst + (size_t)blockIdx.z * plane;
  const int tx = threadIdx.x, ty = threadIdx.y;
  T2 q[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int r = r0 + ty + 8 * j, c = c0 + 2 * tx;
    if (r < rows && c < cols) q[j] = __ldcs(reinterpret_cast<const T2*>(s + (size_t)r * cols + c));
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    tile[ty + 8 * j][2 * tx] = q[j].x;
    tile[ty + 8 * j][2 * tx + 1] = q[j].y;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = c0 + ty + 8 * j, r = r0 + 2 * tx;
    if (r < rows && c < cols) {
      T2 o;
      o.x = tile[2 * tx][ty + 8 * j];
      o.y = tile[2 * tx + 1][ty + 8 * j];
      __stcs(reinterpret_cast<T2*>(d + (size_t)c * rows + r), o);
    }
  }
}

}  // namespace lng

namespace {
template <class T, class TI, class TO, int M, bool FWD, int OM>
cudaError_t launch_long_mode(FastArgs<T> a, cudaStream_t st) {
  using S = lng::LShape<M>;
  auto k = lng::xform_long_kernel<T, TI, TO, M, FWD, OM>;
  constexpr size_t smem = lng::long_smem<T, M>();
  static int bps = 0;
  if (bps == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, S::NT, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = a.nlines < sms * bps ? a.nlines : sms * bps;
  if (grid <= 0) return cudaSuccess;
  k<<<grid, S::NT, smem, st>>>(a);
  return cudaGetLastError();
}
}  // namespace

// the output mode from the arguments, as for the row kernels
template <class T, class TI, class TO, int M, bool FWD>
cudaError_t launch_xform_long(FastArgs<T> a, cudaStream_t st) {
  if constexpr (!FWD && sizeof(TO) == 8 && sizeof(T) == 4) {
    if (a.base32) return launch_long_mode<T, TI, TO, M, FWD, row::OM_BASE>(a, st);
    if (!a.out) return launch_long_mode<T, TI, TO, M, FWD, row::OM_NONE>(a, st);
  }
  if (a.accumulate) return launch_long_mode<T, TI, TO, M, FWD, row::OM_ACC>(a, st);
  return launch_long_mode<T, TI, TO, M, FWD, row::OM_STORE>(a, st);
}

template <class T>
cudaError_t launch_plane_transpose(const T* src, T* dst, int rows, int cols, int nz, const int* skip,
                                   cudaStream_t st) {
  if (nz <= 0 || rows <= 0 || cols <= 0) return cudaSuccess;
  if ((rows | cols) & 1) return cudaErrorInvalidValue;  // pairs of consecutive values
  const dim3 grid((cols + 63) / 64, (rows + 63) / 64, nz);
  const size_t smem = 64 * 65 * sizeof(T);  // ≤ 33 KB: no opt-in needed
  lng::transpose_kernel<T><<<grid, dim3(32, 8), smem, st>>>(src, dst, rows, cols, skip);
  return cudaGetLastError();
}

#define PS_LONG_INST(M)                                                                                   \
  template cudaError_t launch_xform_long<double, double, double, M, true>(FastArgs<double>, cudaStream_t); \
  template cudaError_t launch_xform_long<double, double, double, M, false>(FastArgs<double>, cudaStream_t); \
  template cudaError_t launch_xform_long<float, float, float, M, true>(FastArgs<float>, cudaStream_t);     \
  template cudaError_t launch_xform_long<float, float, float, M, false>(FastArgs<float>, cudaStream_t);    \
  template cudaError_t launch_xform_long<float, double, float, M, true>(FastArgs<float>, cudaStream_t);    \
  template cudaError_t launch_xform_long<float, float, double, M, false>(FastArgs<float>, cudaStream_t);

PS_LONG_INST(1024)
PS_LONG_INST(2048)
PS_LONG_INST(4096)

template cudaError_t launch_plane_transpose<float>(const float*, float*, int, int, int, const int*, cudaStream_t);
template cudaError_t launch_plane_transpose<double>(const double*, double*, int, int, int, const int*,
                                                    cudaStream_t);

}  // namespace ps
