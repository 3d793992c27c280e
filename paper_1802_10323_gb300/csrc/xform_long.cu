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
__host__ __device__ constexpr int rpad(int e) { return e + (e >> 5); }   // real line

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
  // twiddle tables, the complex buffer (padded), the real line (padded)
  return (size_t)LTab<T, M>::ENTRIES * sizeof(cplx<T>) + (size_t)(lpad(M) + 1) * sizeof(cplx<T>) +
         (size_t)(rpad(2 * M) + 2) * sizeof(T);
}

// Makhoul index map (as xform_dev.cuh): position j of v ↔ position of a.
__device__ __forceinline__ int mk(int j, int n, int m) { return j < m ? 2 * j : 2 * n - 1 - 2 * j; }

// a.nlines lines of n = 2M contiguous reals; line ln belongs to plane ln / a.ny
// (for the per-plane scale). Output modes as the row kernels (FastArgs).
template <class T, class TI, class TO, int M, bool FWD>
__global__ void __launch_bounds__(LShape<M>::NT, (sizeof(T) == 8 ? 256 : 768) / LShape<M>::NT)
    xform_long_kernel(FastArgs<T> a) {
  using S = LShape<M>;
  constexpr int N = 2 * M, NT = S::NT, E = S::E, RL = S::radix(S::NST - 1);
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LTab<T, M> tb;
  tb.carve(reinterpret_cast<cplx<T>*>(smem_raw), a.tw);
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw) + LTab<T, M>::ENTRIES;  // [lpad(M) + 1]
  T* rbuf = reinterpret_cast<T*>(buf + lpad(M) + 1);                           // [rpad(N) + 1]
  const int b = threadIdx.x;
  tb.fill(b, NT);
  const cplx<T> tw1 = a.tw[1];  // e^{−2πi/(8n)}: the ND post-twiddle is tw(4k)·tw1
  auto RB = [&](int e) -> T& { return rbuf[rpad(e)]; };
  const int bc = a.bc;
  // no __restrict__: in and out may be the same array
  const TI* in = static_cast<const TI*>(a.in);
  TO* out = static_cast<TO*>(a.out);
  unsigned long long amax = 0;
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
    __syncthreads();  // tables ready; the previous line's buffers are no longer read
    {  // 16-byte loads, 128 bytes of each thread in flight at once
      const T sc = (FWD && a.plane_scale) ? a.plane_scale[z] : (T)1;
      constexpr int V = 16 / sizeof(TI);   // values per vector
      constexpr int NV = N / (V * NT);     // vectors per thread
      constexpr int KV = NV < 8 ? NV : 8;  // vectors per round
      static_assert(N % (V * NT) == 0 && NV % KV == 0, "whole vectors per thread");
#pragma unroll
      for (int i0 = 0; i0 < NV; i0 += KV) {
        TI val[KV * V];
#pragma unroll
        for (int i = 0; i < KV; ++i) {
          const int e = V * (b + (i0 + i) * NT);
          if constexpr (V == 4) {
            const float4 q = *reinterpret_cast<const float4*>(in + g0 + e);
            val[V * i] = q.x; val[V * i + 1] = q.y; val[V * i + 2] = q.z; val[V * i + 3] = q.w;
          } else {
            const double2 q = *reinterpret_cast<const double2*>(in + g0 + e);
            val[V * i] = q.x; val[V * i + 1] = q.y;
          }
        }
#pragma unroll
        for (int i = 0; i < KV; ++i)
#pragma unroll
          for (int u = 0; u < V; ++u) RB(V * (b + (i0 + i) * NT) + u) = ld_cvt<T, TI>::f(val[V * i + u]) * sc;
      }
    }
    __syncthreads();
    cplx<T> v[E];
    if (FWD) {
      // ---- pre-processing gathered into the first stage's operands z_p, p = b + r·NT ----
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int p = b + r * NT;
        cplx<T> zz;
        if (bc == BC_P) {
          zz = {RB(2 * p), RB(2 * p + 1)};
        } else if (bc_iv(bc)) {  // DN: the reversed line, the two reals swap
          const T e0 = RB(2 * p), e1 = RB(N - 1 - 2 * p);
          zz = cmul(bc == BC_DN ? cplx<T>{e1, e0} : cplx<T>{e0, e1}, tb.pp(1, p));
        } else {
          const int j0 = 2 * p, j1 = 2 * p + 1;
          T v0 = RB(mk(j0, N, M)), v1 = RB(mk(j1, N, M));
          if (bc == BC_DD) {
            if (j0 >= M) v0 = -v0;
            if (j1 >= M) v1 = -v1;
          }
          zz = {v0, v1};
        }
        v[r] = zz;
      }
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
          RB(2 * k) = (T)2 * c.x;
          RB(N - 1 - 2 * k) = (T)-2 * c.y;
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
              RB(0) = Vk.x;
              RB(N - 1) = Vmk.x;
            } else {
              RB(2 * k - 1) = Vk.x;
              RB(2 * k) = -Vk.y;
              if (2 * k != M) {
                RB(2 * (M - k) - 1) = Vmk.x;
                RB(2 * (M - k)) = -Vmk.y;
              }
            }
          } else {
            const bool rev = (bc == BC_DD);
            auto put = [&](int qq, T val) { RB(rev ? (N - 1 - qq) : qq) = val; };
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
      if (bc_iv(bc)) {
#pragma unroll 4
        for (int k = b; k < M; k += NT) buf[lpad(k)] = cmul(cplx<T>{RB(2 * k), RB(N - 1 - 2 * k)}, tb.pp(1, k));
      } else {
#pragma unroll 4
        for (int k = b; k <= M / 2; k += NT) {
          cplx<T> Vk, Vmk;
          if (bc == BC_P) {
            if (k == 0) {
              Vk = {RB(0), (T)0};
              Vmk = {RB(N - 1), (T)0};
            } else {
              Vk = {RB(2 * k - 1), -RB(2 * k)};
              Vmk = {RB(2 * (M - k) - 1), -RB(2 * (M - k))};
            }
          } else {
            // DCT-III via Makhoul: V_q = e^{+iπq/2n} (X_q − i X_{n−q}) / 2, X_n = 0;
            // DST-III: the same on Y_q = X_{n−1−q}
            const bool rev = (bc == BC_DD);
            auto XQ = [&](int qq) { return qq >= N ? (T)0 : RB(rev ? (N - 1 - qq) : qq); };
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
      // ---- backward post-processing straight from the last stage to the real line ----
      __syncthreads();  // (the real buffer was last read by the pre-processing)
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
            RB(2 * k) = (bc == BC_DN) ? B : A;
            RB(N - 1 - 2 * k) = (bc == BC_DN) ? A : B;
          } else if (bc == BC_P) {
            RB(2 * k) = zk.x * inv_m;
            RB(2 * k + 1) = zk.y * inv_m;
          } else {
            const int i0 = mk(2 * k, N, M), i1 = mk(2 * k + 1, N, M);
            T v0 = zk.x * inv_m, v1 = zk.y * inv_m;
            if (bc == BC_DD) {
              if (i0 & 1) v0 = -v0;
              if (i1 & 1) v1 = -v1;
            }
            RB(i0) = v0;
            RB(i1) = v1;
          }
        }
      }
    }
    __syncthreads();
    // ---- store, with the output modes of the row kernels: V consecutive values per
    // thread and vector access (16 bytes of the output), the reads of a round first ----
    {
      const T sc = (!FWD && a.plane_scale) ? a.plane_scale[z] : (T)1;
      constexpr int V = 16 / sizeof(TO);
      constexpr int NV = N / (V * NT);
      constexpr int KV = NV < 8 ? NV : 8;
      static_assert(N % (V * NT) == 0 && NV % KV == 0, "whole vectors per thread");
#pragma unroll
      for (int i0 = 0; i0 < NV; i0 += KV) {
        T vv[KV * V];
        TO old[KV * V];  // the base (FP64 output: widened base32 or the accumulated out)
#pragma unroll
        for (int i = 0; i < KV; ++i) {
          const int e = V * (b + (i0 + i) * NT);
#pragma unroll
          for (int u = 0; u < V; ++u) {
            vv[V * i + u] = RB(e + u) * sc;
            old[V * i + u] = (TO)0;
          }
          if constexpr (sizeof(TO) == 8 && sizeof(T) == 4) {
            if (a.base32) {
              const float2 q = *reinterpret_cast<const float2*>(a.base32 + g0 + e);
              old[V * i] = widen_f32(q.x);
              old[V * i + 1] = widen_f32(q.y);
            } else if (out && a.accumulate) {
              const double2 q = *reinterpret_cast<const double2*>(out + g0 + e);
              old[V * i] = q.x;
              old[V * i + 1] = q.y;
            }
          } else if (a.accumulate) {
#pragma unroll
            for (int u = 0; u < V; ++u) old[V * i + u] = out[g0 + e + u];
          }
        }
#pragma unroll
        for (int i = 0; i < KV; ++i) {
          const int e = V * (b + (i0 + i) * NT);
          TO x[V];
#pragma unroll
          for (int u = 0; u < V; ++u) {
            x[u] = st_cvt<TO, T>::f(vv[V * i + u]);
            const bool add = (sizeof(TO) == 8 && sizeof(T) == 4) ? (a.base32 != nullptr || a.accumulate != 0)
                                                                   : (a.accumulate != 0);
            if (add) x[u] = old[V * i + u] + x[u];
          }
          if constexpr (sizeof(TO) == 8) {
#pragma unroll
            for (int u = 0; u < V; ++u)
              amax = max(amax, (unsigned long long)__double_as_longlong(st_cvt<TO, T>::f(vv[V * i + u])) &
                                   0x7FFFFFFFFFFFFFFFull);
            if (out) *reinterpret_cast<double2*>(out + g0 + e) = make_double2(x[0], x[1]);
            if constexpr (sizeof(T) == 4)
              if (a.out2) *reinterpret_cast<float2*>(a.out2 + g0 + e) = make_float2(vv[V * i], vv[V * i + 1]);
          } else {
            *reinterpret_cast<float4*>(out + g0 + e) = make_float4(x[0], x[1], x[2], x[3]);
          }
        }
      }
    }
  }
  if constexpr (sizeof(TO) == 8) {
    if (a.amax) {
      for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if ((threadIdx.x & 31) == 0 && amax) atomicMax(a.amax, amax);
    }
  }
}

// Transpose of every z plane: src [n_z][rows][cols] → dst [n_z][cols][rows], tiles of
// 32 × 32 through shared memory (one pad column), 32 × 8 threads, four rows each.
template <class T>
__global__ void __launch_bounds__(256) transpose_kernel(const T* __restrict__ src, T* __restrict__ dst, int rows,
                                                        int cols, const int* skip) {
  if (skip && *skip) return;
  __shared__ T tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const size_t plane = (size_t)rows * cols;
  const T* s = src + (size_t)blockIdx.z * plane;
  T* d = dst + (size_t)blockIdx.z * plane;
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int j = 0; j < 32; j += 8) {
    const int r = r0 + ty + j, c = c0 + tx;
    if (r < rows && c < cols) tile[ty + j][tx] = s[(size_t)r * cols + c];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 32; j += 8) {
    const int c = c0 + ty + j, r = r0 + tx;
    if (r < rows && c < cols) d[(size_t)c * rows + r] = tile[tx][ty + j];
  }
}

}  // namespace lng

template <class T, class TI, class TO, int M, bool FWD>
cudaError_t launch_xform_long(FastArgs<T> a, cudaStream_t st) {
  using S = lng::LShape<M>;
  auto k = lng::xform_long_kernel<T, TI, TO, M, FWD>;
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

template <class T>
cudaError_t launch_plane_transpose(const T* src, T* dst, int rows, int cols, int nz, const int* skip,
                                   cudaStream_t st) {
  if (nz <= 0 || rows <= 0 || cols <= 0) return cudaSuccess;
  const dim3 grid((cols + 31) / 32, (rows + 31) / 32, nz);
  lng::transpose_kernel<T><<<grid, dim3(32, 8), 0, st>>>(src, dst, rows, cols, skip);
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
