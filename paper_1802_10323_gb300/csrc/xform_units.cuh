// xform_units.cuh — the units of work of the register-resident line transforms:
// one x line per warp (row_line) and one tile of CW y columns per CTA (col_tile),
// called by the per-axis kernels (xform_row.cu, xform_col.cu). The mathematics is
// the same in every unit: an M-point complex FFT per line of n = 2M reals with the
// Table 2 pre/post processing per BC; the layouts are described in the two kernel
// files.
#pragma once
#include <type_traits>

#include "xform_fast.cuh"

namespace ps {

// Twiddle tables of one axis into shared memory at stw: ω_M^t (t < M), the
// real-FFT split factors (M + 1) and the BC factors (NN/DD: n; ND: 2·M).
template <class T, int M>
__device__ __forceinline__ void load_line_tables(const cplx<T>* tw, int bc, cplx<T>* stw) {
  constexpr int N = 2 * M;
  cplx<T>* ptw = stw + M;
  cplx<T>* xtw = ptw + (M + 1);
  for (int i = threadIdx.x; i < M; i += blockDim.x) stw[i] = tw[16 * i];
  for (int i = threadIdx.x; i <= M; i += blockDim.x) ptw[i] = tw[8 * i];
  if (bc == BC_NN || bc == BC_DD) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) xtw[i] = tw[2 * i];
  } else if (bc_iv(bc)) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      xtw[i] = tw[4 * i];
      xtw[M + i] = tw[4 * i + 1];
    }
  }
}

namespace row {

using fast::Shape;
using fast::cpad;

template <class T, int N>
struct alignas(sizeof(T) * N) vec {
  T v[N];
};

constexpr int WARPS = 8;  // warps per CTA

template <class TC, class TI>
__device__ __forceinline__ TC in_cvt(TI x) { return ld_cvt<TC, TI>::f(x); }

// Output modes of the backward transform (compile-time, so that no mode pays for
// another's registers): store; accumulate (out += v); base (out = widen(base32) + v);
// none (no FP64 output: only the FP32 copy and the max).
enum { OM_STORE = 0, OM_ACC = 1, OM_BASE = 2, OM_NONE = 3 };

// Slots of a 32-lane line (M ≥ 128): lane t holds wavenumbers k = t + 32·j, j < E.
// After the last FFT stage slot si holds j = jout(si); the first stage takes slot si
// at j = jin(si). The partner M − k of k is held by lane (32 − t) mod 32 at
// j' = E − 1 − j (lane 0: j' = E − j, and k = 0 pairs with itself).
template <int M>
struct LaneSlots {
  static constexpr int E = Shape<M>::E, R0 = Shape<M>::radix(0), RL = Shape<M>::radix(Shape<M>::NST - 1);
  __host__ __device__ static constexpr int jin(int si) { return si / R0 + (si % R0) * (M / R0 / 32); }
  __host__ __device__ static constexpr int jout(int si) { return si / RL + (si % RL) * (M / RL / 32); }
  __host__ __device__ static constexpr int sin_(int j) {
    int r = 0;
    for (int s = 0; s < E; ++s)
      if (jin(s) == j) r = s;
    return r;
  }
  __host__ __device__ static constexpr int sout(int j) {
    int r = 0;
    for (int s = 0; s < E; ++s)
      if (jout(s) == j) r = s;
    return r;
  }
};

// One line (two for M = 64, half a warp each) of the x transform: the warp's
// exchange buffers at bufs, tables in shared memory, the first line index l0.
// tmax accumulates max |FP64 output| (before widening) for the caller's reduction.
template <class T, class TI, class TO, int M, bool FWD, int OM>
__device__ __forceinline__ void row_line(const FastArgs<T>& a, const cplx<T>* stw, const cplx<T>* ptw,
                                         const cplx<T>* xtw, cplx<T>* bufs, int l0, T& tmax) {
  using S = Shape<M>;
  constexpr int N = 2 * M, E = S::E, TPL = S::TPL;
  constexpr int R0 = S::radix(0), RL = S::radix(S::NST - 1);
  constexpr int LB = M + M / 8;  // complex slots of a line's exchange buffer (skewed)
  const int bc = a.bc;
  const int lane = threadIdx.x & 31;
  const int t = lane % TPL, half = lane / TPL;
  const int mate = lane ^ (TPL - 1);  // lane of the mirrored points M−1−p
  cplx<T>* lc = bufs + half * LB;
  const TI* in = static_cast<const TI*>(a.in);  // may equal out (in-place passes)
  TO* out = static_cast<TO*>(a.out);
  const int ny = a.ny, nlines = a.nlines;
  const unsigned full = 0xffffffffu;
  const int line = l0 + half;
  const bool live = line < nlines;  // the other half-warp line may be past the end
  const size_t base = (size_t)(live ? line : l0) * N;
  const TI* src = in + base;
  TO* dst = out + base;
  const T s = a.plane_scale ? a.plane_scale[(live ? line : l0) / ny] : (T)1;
  cplx<T> v[E];
  if (FWD) {
    // ---- gather the first-stage operands from the line ----
    // slot si = q·R0 + r holds point p = t + q·TPL + r·(M/R0); p < M/2 iff r < R0/2
    if (bc == BC_P) {
#pragma unroll
      for (int si = 0; si < E; ++si) {
        const int p = t + (si / R0) * TPL + (si % R0) * (M / R0);
        const vec<TI, 2> x = *reinterpret_cast<const vec<TI, 2>*>(src + 2 * p);
        v[si] = {in_cvt<T>(x.v[0]) * s, in_cvt<T>(x.v[1]) * s};
      }
    } else if (bc_iv(bc)) {
      // z_p = (x_{2p}, x_{n−1−2p})·e^{−iπp/n}; x_{n−1−2p} = x_{2p'+1} of p' = M−1−p
      // (DN, the reversed line: z_p = (x_{n−1−2p}, x_{2p}), the two parts trade places)
#pragma unroll
      for (int si = 0; si < E; ++si) {
        const int p = t + (si / R0) * TPL + (si % R0) * (M / R0);
        const vec<TI, 2> x = *reinterpret_cast<const vec<TI, 2>*>(src + 2 * p);
        v[si].x = in_cvt<T>(x.v[0]) * s;
        const T odd = in_cvt<T>(x.v[1]) * s;
        v[E - 1 - si].y = __shfl_sync(full, odd, mate);
      }
      if (bc == BC_DN) {
#pragma unroll
        for (int si = 0; si < E; ++si) v[si] = {v[si].y, v[si].x};
      }
#pragma unroll
      for (int si = 0; si < E; ++si) {
        const int p = t + (si / R0) * TPL + (si % R0) * (M / R0);
        v[si] = cmul(v[si], xtw[p]);
      }
    } else {
      // z_p = (v_{2p}, v_{2p+1}) with v_j = x_{2j} (j < M), ±x_{2n−1−2j} (j ≥ M, − for DD);
      // the 4-vector at 4p (p < M/2) is (z_p.x, z_{p'}.y, z_p.y, z_{p'}.x), p' = M−1−p
      const T sg = (bc == BC_DD) ? (T)-1 : (T)1;
#pragma unroll
      for (int si = 0; si < E; ++si) {
        if ((si % R0) >= R0 / 2) continue;
        const int p = t + (si / R0) * TPL + (si % R0) * (M / R0);
        T x[4];
        if constexpr (sizeof(TI) == 4) {
          const vec<TI, 4> q = *reinterpret_cast<const vec<TI, 4>*>(src + 4 * p);
#pragma unroll
          for (int u = 0; u < 4; ++u) x[u] = in_cvt<T>(q.v[u]) * s;
        } else {
          const vec<TI, 2> q0 = *reinterpret_cast<const vec<TI, 2>*>(src + 4 * p);
          const vec<TI, 2> q1 = *reinterpret_cast<const vec<TI, 2>*>(src + 4 * p + 2);
          x[0] = in_cvt<T>(q0.v[0]) * s;
          x[1] = in_cvt<T>(q0.v[1]) * s;
          x[2] = in_cvt<T>(q1.v[0]) * s;
          x[3] = in_cvt<T>(q1.v[1]) * s;
        }
        v[si] = {x[0], x[2]};
        const T ry = __shfl_sync(full, x[1], mate), rx = __shfl_sync(full, x[3], mate);
        v[E - 1 - si] = {sg * rx, sg * ry};
      }
    }
    fast::fft_stages<T, M, false, 0, 1>(v, lc, stw, t);
    if constexpr (TPL == 32) {
      // ---- post-processing in registers: pairs (k, M−k), Z_{M−k} from the partner lane ----
      // Lane t takes its slots j < E/2 (k = t + 32j) and writes the outputs of k and of
      // M − k, whose Z arrives by shuffle from slot E−1−j of lane (32 − t) mod 32; every
      // slot is read once. Lane 0's partners are its own slots E − j: the value it
      // shuffled to itself one iteration earlier (k = 0 pairs with itself), and after the
      // loop, the one of k = M/2.
      using LS = LaneSlots<M>;
      auto Y = [&](int i, T val) {
        if (live) dst[i] = st_cvt<TO, T>::f(val);
      };
      if (bc_iv(bc)) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int k = t + 32 * j;
          const cplx<T> c = cmul(xtw[M + k], v[LS::sout(j)]);
          Y(2 * k, (T)2 * c.x);
          Y(N - 1 - 2 * k, (T)-2 * c.y);
        }
      } else {
        const int pl = (32 - t) & 31;
        const bool rev = (bc == BC_DD);
        auto OUTQ = [&](int q, T val) { Y(rev ? (N - 1 - q) : q, val); };
        // outputs of k (and of M − k unless k = 0 or 2k = M) from Z_k and Z_{M−k}
        auto pair_out = [&](int k, cplx<T> Zk, cplx<T> Zmk) {
          const cplx<T> Ek = cscale(cadd(Zk, conj_(Zmk)), (T)0.5);
          const cplx<T> Ok = cscale(mul_mi(csub(Zk, conj_(Zmk))), (T)0.5);
          const cplx<T> B = cmul(ptw[k], Ok);
          const cplx<T> Vk = cadd(Ek, B), Vmk = conj_(csub(Ek, B));
          if (bc == BC_P) {
            if (k == 0) {
              Y(0, Vk.x);
              Y(N - 1, Vmk.x);
            } else {
              Y(2 * k - 1, Vk.x);
              Y(2 * k, -Vk.y);
              if (2 * k != M) {
                Y(2 * (M - k) - 1, Vmk.x);
                Y(2 * (M - k), -Vmk.y);
              }
            }
          } else if (k == 0) {
            OUTQ(0, (T)2 * Vk.x);
            OUTQ(M, (T)1.41421356237309504880 * Vmk.x);
          } else {
            const cplx<T> c1 = cmul(xtw[k], Vk);
            OUTQ(k, (T)2 * c1.x);
            OUTQ(N - k, (T)-2 * c1.y);
            if (2 * k != M) {
              const cplx<T> c2 = cmul(xtw[M - k], Vmk);
              OUTQ(M - k, (T)2 * c2.x);
              OUTQ(M + k, (T)-2 * c2.y);
            }
          }
        };
        cplx<T> prev = {(T)0, (T)0};
#pragma unroll
        for (int j = 0; j < E / 2; ++j) {
          const cplx<T> Zk = v[LS::sout(j)];
          const cplx<T> recv = {__shfl_sync(full, v[LS::sout(E - 1 - j)].x, pl),
                                __shfl_sync(full, v[LS::sout(E - 1 - j)].y, pl)};
          const cplx<T> Zmk = (t != 0) ? recv : (j == 0 ? Zk : prev);
          prev = recv;
          pair_out(t + 32 * j, Zk, Zmk);
        }
        if (t == 0) pair_out(M / 2, prev, prev);  // k = M/2 pairs with itself
      }
    } else {
      // ---- post-processing: pairs (k, M−k) through the exchange buffer, scalar stores ----
      __syncwarp();
  #pragma unroll
      for (int q = 0; q < E / RL; ++q)
  #pragma unroll
        for (int r = 0; r < RL; ++r) lc[cpad(t + q * TPL + r * (M / RL))] = v[q * RL + r];
      __syncwarp();
      auto Y = [&](int i, T val) {
        if (live) dst[i] = st_cvt<TO, T>::f(val);
      };
      if (bc_iv(bc)) {
  #pragma unroll
        for (int i = 0; i < E; ++i) {
          const int k = t + i * TPL;
          const cplx<T> c = cmul(xtw[M + k], lc[cpad(k)]);
          Y(2 * k, (T)2 * c.x);
          Y(N - 1 - 2 * k, (T)-2 * c.y);
        }
      } else {
        constexpr int NP = (M / 2) / TPL + 1;
  #pragma unroll
        for (int i = 0; i < NP; ++i) {
          const int k = t + i * TPL;
          if (k > M / 2) break;
          const cplx<T> Zk = lc[cpad(k)], Zmk = lc[cpad(k == 0 ? 0 : M - k)];
          const cplx<T> Ek = cscale(cadd(Zk, conj_(Zmk)), (T)0.5);
          const cplx<T> Ok = cscale(mul_mi(csub(Zk, conj_(Zmk))), (T)0.5);
          const cplx<T> B = cmul(ptw[k], Ok);
          const cplx<T> Vk = cadd(Ek, B), Vmk = conj_(csub(Ek, B));
          if (bc == BC_P) {
            if (k == 0) {
              Y(0, Vk.x);
              Y(N - 1, Vmk.x);
            } else {
              Y(2 * k - 1, Vk.x);
              Y(2 * k, -Vk.y);
              if (2 * k != M) {
                Y(2 * (M - k) - 1, Vmk.x);
                Y(2 * (M - k), -Vmk.y);
              }
            }
          } else {
            const bool rev = (bc == BC_DD);
            auto OUTQ = [&](int q, T val) { Y(rev ? (N - 1 - q) : q, val); };
            if (k == 0) {
              OUTQ(0, (T)2 * Vk.x);
              OUTQ(M, (T)1.41421356237309504880 * Vmk.x);
            } else {
              const cplx<T> c1 = cmul(xtw[k], Vk);
              OUTQ(k, (T)2 * c1.x);
              OUTQ(N - k, (T)-2 * c1.y);
              if (2 * k != M) {
                const cplx<T> c2 = cmul(xtw[M - k], Vmk);
                OUTQ(M - k, (T)2 * c2.x);
                OUTQ(M + k, (T)-2 * c2.y);
              }
            }
          }
        }
      }
      __syncwarp();  // buffer reads done before the next line overwrites it
    }
  } else {
    // The FP64 output modes read the line's base (FP32 Φ_0) or its accumulator (FP64
    // p) only when the outputs are written; ask L2 for them now, one 128-byte
    // segment per lane, so that those loads do not wait on HBM after the transform.
    if constexpr (sizeof(TO) == 8 && sizeof(T) == 4 && (OM == OM_BASE || OM == OM_ACC)) {
      if (live) {
        const char* pf = (OM == OM_BASE) ? reinterpret_cast<const char*>(a.base32 + base)
                                         : reinterpret_cast<const char*>(dst);
        constexpr int SEG = (OM == OM_BASE ? N * 4 : N * 8) / 128;  // 128-byte segments of the line
#pragma unroll
        for (int j = t; j < SEG; j += TPL) asm volatile("prefetch.global.L2 [%0];" ::"l"(pf + 128 * j));
      }
    }
    auto X = [&](int i) { return in_cvt<T>(src[i]); };
    if constexpr (TPL == 32) {
      // ---- backward pre-processing in registers: own V_k, V_{M−k} from the partner lane,
      // Z_k straight into its first-stage slot ----
      using LS = LaneSlots<M>;
      if (bc_iv(bc)) {
        // (x_{2k}, x_{n−1−2k})·e^{−iπk/n}; x_{n−1−2k} = x_{2k'+1} of k' = M−1−k (mirrored lane)
        cplx<T> z[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int k = t + i * TPL;
          const vec<TI, 2> x = *reinterpret_cast<const vec<TI, 2>*>(src + 2 * k);
          z[i].x = in_cvt<T>(x.v[0]);
          z[E - 1 - i].y = __shfl_sync(full, in_cvt<T>(x.v[1]), mate);
        }
#pragma unroll
        for (int j = 0; j < E; ++j) v[LS::sin_(j)] = cmul(z[j], xtw[t + 32 * j]);
      } else {
        const bool rev = (bc == BC_DD);
        auto qx = [&](int q) { return rev ? (N - 1 - q) : q; };
        cplx<T> Vv[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int k = t + 32 * j;
          if (bc == BC_P) {
            Vv[j] = (k == 0) ? cplx<T>{X(0), (T)0} : cplx<T>{X(2 * k - 1), -X(2 * k)};
          } else {
            const T x0 = X(qx(k)), x1 = (k == 0) ? (T)0 : X(qx(N - k));
            cplx<T> w = xtw[k];
            w.y = -w.y;
            Vv[j] = cscale(cmul(w, cplx<T>{x0, -x1}), (T)0.5);
          }
        }
        // V_M, the partner of k = 0 (lane 0)
        cplx<T> VM;
        if (bc == BC_P) {
          VM = {X(N - 1), (T)0};
        } else {
          const T xm = X(qx(M));
          cplx<T> w = xtw[M];
          w.y = -w.y;
          VM = cscale(cmul(w, cplx<T>{xm, -xm}), (T)0.5);
        }
        const int pl = (32 - t) & 31;
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int k = t + 32 * j;
          cplx<T> Vm = {__shfl_sync(full, Vv[E - 1 - j].x, pl), __shfl_sync(full, Vv[E - 1 - j].y, pl)};
          if (t == 0) Vm = (j == 0) ? VM : Vv[(E - j) % E];
          const cplx<T> Ek = cscale(cadd(Vv[j], conj_(Vm)), (T)0.5);
          cplx<T> wn = ptw[k];
          wn.y = -wn.y;
          const cplx<T> Ok = cscale(cmul(csub(Vv[j], conj_(Vm)), wn), (T)0.5);
          v[LS::sin_(j)] = cadd(Ek, mul_i(Ok));
        }
      }
    } else {
      // ---- backward pre-processing: pairs (k, M−k) from the line into the buffer ----
      if (bc_iv(bc)) {
        // (x_{2k}, x_{n−1−2k})·e^{−iπk/n}; x_{n−1−2k} = x_{2k'+1} of k' = M−1−k
  #pragma unroll
        for (int i = 0; i < E; ++i) {
          const int k = t + i * TPL;
          const vec<TI, 2> x = *reinterpret_cast<const vec<TI, 2>*>(src + 2 * k);
          v[i].x = in_cvt<T>(x.v[0]);
          v[E - 1 - i].y = __shfl_sync(full, in_cvt<T>(x.v[1]), mate);
        }
  #pragma unroll
        for (int i = 0; i < E; ++i) {
          const int k = t + i * TPL;
          lc[cpad(k)] = cmul(v[i], xtw[k]);
        }
      } else {
        constexpr int NP = (M / 2) / TPL + 1;
        T xv[NP][4];
  #pragma unroll
        for (int i = 0; i < NP; ++i) {
          const int k = t + i * TPL;
          const bool ok = (i < NP - 1) || (k <= M / 2);
          int q[4];
          bool use[4] = {ok, ok, ok, ok};
          if (bc == BC_P) {
            q[0] = k == 0 ? 0 : 2 * k - 1;
            q[1] = 2 * k;
            q[2] = k == 0 ? N - 1 : 2 * (M - k) - 1;
            q[3] = 2 * (M - k);
            use[1] = use[3] = ok && k != 0;
          } else {
            const bool rev = (bc == BC_DD);
            const int qq[4] = {k, N - k, M - k, N - M + k};
  #pragma unroll
            for (int u = 0; u < 4; ++u) {
              q[u] = rev ? (N - 1 - qq[u]) : qq[u];
              use[u] = ok && qq[u] < N;
            }
          }
  #pragma unroll
          for (int u = 0; u < 4; ++u) xv[i][u] = use[u] ? X(q[u]) : (T)0;
        }
  #pragma unroll
        for (int i = 0; i < NP; ++i) {
          const int k = t + i * TPL;
          if (i == NP - 1 && k > M / 2) break;
          cplx<T> Vk, Vm;
          if (bc == BC_P) {
            Vk = {xv[i][0], -xv[i][1]};
            Vm = {xv[i][2], -xv[i][3]};
          } else {
            cplx<T> w = xtw[k];
            w.y = -w.y;
            Vk = cscale(cmul(w, cplx<T>{xv[i][0], -xv[i][1]}), (T)0.5);
            cplx<T> w2 = xtw[M - k];
            w2.y = -w2.y;
            Vm = cscale(cmul(w2, cplx<T>{xv[i][2], -xv[i][3]}), (T)0.5);
          }
          const cplx<T> Ek = cscale(cadd(Vk, conj_(Vm)), (T)0.5);
          cplx<T> wn = ptw[k];
          wn.y = -wn.y;
          const cplx<T> Ok = cscale(cmul(csub(Vk, conj_(Vm)), wn), (T)0.5);
          if (k < M) lc[cpad(k)] = cadd(Ek, mul_i(Ok));
          if (k != 0 && 2 * k != M) lc[cpad(M - k)] = cadd(conj_(Ek), mul_i(conj_(Ok)));
        }
      }
      __syncwarp();
  #pragma unroll
      for (int q = 0; q < E / R0; ++q)
  #pragma unroll
        for (int r = 0; r < R0; ++r) v[q * R0 + r] = lc[cpad(t + q * TPL + r * (M / R0))];
    }
    if (bc_iv(bc)) fast::fft_stages<T, M, false, 0, 1>(v, lc, stw, t);
    else fast::fft_stages<T, M, true, 0, 1>(v, lc, stw, t);
    __syncwarp();  // the last stage's buffer reads are done before the next line
    // ---- backward outputs straight from the last stage, as vectors ----
    // slot si = q·RL + r holds wavenumber k = t + q·TPL + r·(M/RL); k < M/2 iff r < RL/2
    // n consecutive outputs at i0; an FP64 output may also keep its FP32 value in out2
    // (the line's own input array: every input of the line is already in registers)
    auto put = [&](int i0, const T* val, auto n_tag) {
      constexpr int NV = decltype(n_tag)::value;
      constexpr bool F64OUT = sizeof(TO) == 8 && sizeof(T) == 4;
      vec<TO, NV> o;
      vec<T, NV> o2;
      if constexpr (OM == OM_ACC) o = *reinterpret_cast<const vec<TO, NV>*>(dst + i0);
      if constexpr (F64OUT && OM == OM_BASE) {
        const vec<float, NV> b32 = *reinterpret_cast<const vec<float, NV>*>(a.base32 + base + i0);
#pragma unroll
        for (int u = 0; u < NV; ++u) o.v[u] = widen_f32(b32.v[u]);
      }
#pragma unroll
      for (int u = 0; u < NV; ++u) {
        o2.v[u] = val[u] * s;
        const TO x = st_cvt<TO, T>::f(o2.v[u]);
        if constexpr (OM == OM_ACC || (F64OUT && OM == OM_BASE)) o.v[u] = o.v[u] + x;
        else o.v[u] = x;
        if constexpr (sizeof(TO) == 8)
          if (live) tmax = fmax(tmax, fabs(o2.v[u]));
      }
      if (live) {
        if constexpr (OM != OM_NONE) *reinterpret_cast<vec<TO, NV>*>(dst + i0) = o;
        if constexpr (F64OUT)
          if (a.out2) *reinterpret_cast<vec<T, NV>*>(a.out2 + base + i0) = o2;
      }
    };
    using two = std::integral_constant<int, 2>;
    using four = std::integral_constant<int, 4>;
    const T inv_m = (T)1 / (T)M;
    if (bc == BC_P) {
#pragma unroll
      for (int si = 0; si < E; ++si) {
        const int k = t + (si / RL) * TPL + (si % RL) * (M / RL);
        const T val[2] = {v[si].x * inv_m, v[si].y * inv_m};
        put(2 * k, val, two{});
      }
    } else if (bc_iv(bc)) {
      // output 2k = Re(c_k)/n, output n−1−2k = −Im(c_k)/n with c_k = e^{...}·z_k;
      // the pair (2k, 2k+1) takes −Im(c_{k'})/n of k' = M−1−k from the mirrored slot
      // (DN, the reversed line: the two outputs of each k trade places)
      const T inv_n = (T)1 / (T)N;
      T re[E], im[E];
#pragma unroll
      for (int si = 0; si < E; ++si) {
        const int k = t + (si / RL) * TPL + (si % RL) * (M / RL);
        const cplx<T> c = cmul(xtw[M + k], v[si]);
        const T A = c.x * inv_n, B = -c.y * inv_n;
        re[si] = (bc == BC_DN) ? B : A;
        im[si] = (bc == BC_DN) ? A : B;
      }
#pragma unroll
      for (int si = 0; si < E; ++si) {
        const int k = t + (si / RL) * TPL + (si % RL) * (M / RL);
        const T val[2] = {re[si], __shfl_sync(full, im[E - 1 - si], mate)};
        put(2 * k, val, two{});
      }
    } else {
      // z_k → outputs (i0, i1) = (4k, 4k+2) for k < M/2 and the odd (2n−1−4k, 2n−3−4k)
      // for k ≥ M/2 (negated for DD): the 4-vector at 4k (k < M/2) is
      // (z_k.x, ±z_{k'}.y, z_k.y, ±z_{k'}.x), k' = M−1−k
      const T sg = (bc == BC_DD) ? (T)-1 : (T)1;
#pragma unroll
      for (int si = 0; si < E; ++si) {
        const int j = E - 1 - si;  // every lane hands its mirrored slot to its mate
        const T hy = __shfl_sync(full, v[j].y, mate), hx = __shfl_sync(full, v[j].x, mate);
        if ((si % RL) >= RL / 2) continue;
        const int k = t + (si / RL) * TPL + (si % RL) * (M / RL);
        const T val[4] = {v[si].x * inv_m, sg * hy * inv_m, v[si].y * inv_m, sg * hx * inv_m};
        put(4 * k, val, four{});
      }
    }
  }
}

}  // namespace row

namespace col {

template <int M, int CW>  // CW: x columns per CTA (16 or 8)
struct CShape {
  static constexpr int TPL = (M >= 128) ? 32 : 16;  // threads per column
  static constexpr int E = M / TPL;                 // complex points per thread
  static constexpr int NT = CW * TPL;               // threads per CTA
  static constexpr int NST = (M == 128) ? 4 : 3;
  // radix of stage s; the first equals E (one butterfly per thread), all divide E
  __host__ __device__ static constexpr int radix(int s) {
    return (M == 512) ? (s == 0 ? 16 : (s == 1 ? 8 : 4))
         : (M == 256) ? (s < 2 ? 8 : 4)
         : (M == 128) ? (s < 3 ? 4 : 2)
         : 4;
  }
};

// 16-point DFT in natural order, as 4 × 4: X[k1 + 4k2] =
// Σ_{n2} W4^{n2·k2} · W16^{n2·k1} · Σ_{n1} x[n2 + 4n1] · W4^{n1·k1}.
template <class T, bool INV>
__device__ __forceinline__ void dft16(cplx<T>* v) {
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // cos, sin of π/8
  const T h = (T)0.70710678118654752440;
  cplx<T> a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) a[n2][n1] = v[n2 + 4 * n1];
    fast::dft4<T, INV>(a[n2]);
  }
  // W16^m = (cos 2πm/16, −sin 2πm/16) for the forward transform, conjugate for the inverse
  auto tw = [&](cplx<T> z, T wr, T wi) {
    if (INV) wi = -wi;
    return cplx<T>{z.x * wr - z.y * wi, z.x * wi + z.y * wr};
  };
  a[1][1] = tw(a[1][1], c1, -s1);  // m = 1
  a[1][2] = tw(a[1][2], h, -h);    // m = 2
  a[1][3] = tw(a[1][3], s1, -c1);  // m = 3
  a[2][1] = tw(a[2][1], h, -h);    // m = 2
  a[2][2] = INV ? mul_i(a[2][2]) : mul_mi(a[2][2]);  // m = 4
  a[2][3] = tw(a[2][3], -h, -h);   // m = 6
  a[3][1] = tw(a[3][1], s1, -c1);  // m = 3
  a[3][2] = tw(a[3][2], -h, -h);   // m = 6
  a[3][3] = tw(a[3][3], -c1, s1);  // m = 9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cplx<T> b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    fast::dft4<T, INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
  }
}

template <class T, int R, bool INV>
__device__ __forceinline__ void dft(cplx<T>* v) {
  if constexpr (R == 16) dft16<T, INV>(v);
  else fast::dftR<T, R, INV>(v);
}

// Stages STAGE… of the M-point FFT of this thread's column. On entry
// v[q·R + r] = x[b_q + r·M/R] with b_q = b + q·TPL; on return v holds the last
// stage's outputs, v[q·R + r] at position b_q + r·(M/R_last).
template <class T, int M, int CW, bool INV, int STAGE, int NS>
__device__ __forceinline__ void fft_col(cplx<T> (&v)[CShape<M, CW>::E], cplx<T>* buf, const cplx<T>* stw,
                                        int b, int c) {
  using S = CShape<M, CW>;
  constexpr int E = S::E, TPL = S::TPL;
  constexpr int R = S::radix(STAGE);
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
    const int bq = b + q * TPL;
    if constexpr (STAGE > 0) {
      const int k = bq & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = stw[(r * k * (M / (NS * R))) & (M - 1)];
        if (INV) w.y = -w.y;
        v[q * R + r] = cmul(v[q * R + r], w);
      }
    }
    dft<T, R, INV>(&v[q * R]);
  }
  if constexpr (STAGE + 1 < S::NST) {
    constexpr int R2 = S::radix(STAGE + 1);
    __syncthreads();  // earlier readers of buf are done
#pragma unroll
    for (int q = 0; q < E / R; ++q) {
      const int bq = b + q * TPL;
      const int o = (bq / NS) * NS * R + (bq & (NS - 1));
#pragma unroll
      for (int r = 0; r < R; ++r) buf[(o + r * NS) * CW + c] = v[q * R + r];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E / R2; ++q) {
      const int bq = b + q * TPL;
#pragma unroll
      for (int r = 0; r < R2; ++r) v[q * R2 + r] = buf[(bq + r * (M / R2)) * CW + c];
    }
    fft_col<T, M, CW, INV, STAGE + 1, NS * R>(v, buf, stw, b, c);
  }
}

template <class T, int M, int CW>
__host__ __device__ constexpr size_t col_smem(int bc) {
  return fast_table_bytes<T, M>(bc) + (size_t)M * CW * sizeof(cplx<T>);
}

// One tile of the y transform: CW consecutive x columns of one z plane (tile g
// of the n_z·n_x/CW tiles, x fastest); tables and the exchange buffer in shared
// memory. Starts with a block barrier (tables ready, earlier buffer reads done).
template <class T, int M, bool FWD, int CW>
__device__ __forceinline__ void col_tile(const FastArgs<T>& a, const cplx<T>* stw, const cplx<T>* ptw,
                                         const cplx<T>* xtw, cplx<T>* buf, int g) {
  using S = CShape<M, CW>;
  constexpr int N = 2 * M, E = S::E, TPL = S::TPL;
  constexpr int RL = S::radix(S::NST - 1);
  const int bc = a.bc;
  const int c = threadIdx.x % CW, b = threadIdx.x / CW;
  const T* in = static_cast<const T*>(a.in);  // may equal out (in-place y passes)
  T* out = static_cast<T*>(a.out);
  const int nx = a.nx, ny = a.ny;
  const int tpz = nx / CW;
  const int zb = g / tpz, x0 = (g - zb * tpz) * CW;
  // DN is the ND problem on the reversed line: the forward transform reads its input
  // rows from row n−1 downwards and runs the ND code unchanged; the backward one swaps
  // the two outputs of each wavenumber
  const bool rv = FWD && (bc == BC_DN);
  const int sstr = rv ? -nx : nx;
  const T* src = in + (size_t)zb * ny * nx + x0 + c + (rv ? (size_t)(N - 1) * nx : 0);
  T* dst = out + (size_t)zb * ny * nx + x0 + c;
  // row offsets fit in 32 bits (n_y·n_x ≤ 2^20)
  auto X = [&](int q) { return src[q * sstr]; };
  auto Y = [&](int q, T val) { dst[q * nx] = val; };
  const T s = a.plane_scale ? a.plane_scale[zb] : (T)1;
  cplx<T> v[E];
  __syncthreads();  // tables ready; the previous tile's buffer reads are done
  if (FWD) {
    // ---- pre-processing gathered from the rows into the first-stage operands ----
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int p = b + r * TPL;
      cplx<T> z;
      if (bc == BC_P) {
        z = {X(2 * p), X(2 * p + 1)};
      } else if (bc_iv(bc)) {  // (DN: rows addressed in reverse, see above)
        z = cmul(cplx<T>{X(2 * p), X(N - 1 - 2 * p)}, xtw[p]);
      } else {
        const int j0 = 2 * p, j1 = 2 * p + 1;
        T v0 = X(j0 < M ? 2 * j0 : 2 * N - 1 - 2 * j0);
        T v1 = X(j1 < M ? 2 * j1 : 2 * N - 1 - 2 * j1);
        if (bc == BC_DD) {
          if (j0 >= M) v0 = -v0;
          if (j1 >= M) v1 = -v1;
        }
        z = {v0, v1};
      }
      v[r] = cscale(z, s);
    }
    fft_col<T, M, CW, false, 0, 1>(v, buf, stw, b, c);
    // ---- post-processing: pair k with M − k through the buffer, rows out ----
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E / RL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) buf[(b + q * TPL + r * (M / RL)) * CW + c] = v[q * RL + r];
    __syncthreads();
    if (bc_iv(bc)) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int k = b + i * TPL;
        const cplx<T> cc = cmul(xtw[M + k], buf[k * CW + c]);
        Y(2 * k, (T)2 * cc.x);
        Y(N - 1 - 2 * k, (T)-2 * cc.y);
      }
    } else {
      constexpr int NP = (M / 2) / TPL + 1;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const int k = b + i * TPL;
        if (k > M / 2) break;
        const cplx<T> Zk = buf[k * CW + c], Zmk = buf[(k == 0 ? 0 : M - k) * CW + c];
        const cplx<T> Ek = cscale(cadd(Zk, conj_(Zmk)), (T)0.5);
        const cplx<T> Ok = cscale(mul_mi(csub(Zk, conj_(Zmk))), (T)0.5);
        const cplx<T> B = cmul(ptw[k], Ok);
        const cplx<T> Vk = cadd(Ek, B), Vmk = conj_(csub(Ek, B));
        if (bc == BC_P) {
          if (k == 0) {
            Y(0, Vk.x);
            Y(N - 1, Vmk.x);
          } else {
            Y(2 * k - 1, Vk.x);
            Y(2 * k, -Vk.y);
            if (2 * k != M) {
              Y(2 * (M - k) - 1, Vmk.x);
              Y(2 * (M - k), -Vmk.y);
            }
          }
        } else {
          const bool rev = (bc == BC_DD);
          auto OUTQ = [&](int q, T val) { Y(rev ? (N - 1 - q) : q, val); };
          if (k == 0) {
            OUTQ(0, (T)2 * Vk.x);
            OUTQ(M, (T)1.41421356237309504880 * Vmk.x);
          } else {
            const cplx<T> c1 = cmul(xtw[k], Vk);
            OUTQ(k, (T)2 * c1.x);
            OUTQ(N - k, (T)-2 * c1.y);
            if (2 * k != M) {
              const cplx<T> c2 = cmul(xtw[M - k], Vmk);
              OUTQ(M - k, (T)2 * c2.x);
              OUTQ(M + k, (T)-2 * c2.y);
            }
          }
        }
      }
    }
  } else {
    // ---- backward pre-processing from the rows into the buffer ----
    if (bc_iv(bc)) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int k = b + i * TPL;
        buf[k * CW + c] = cmul(cplx<T>{X(2 * k), X(N - 1 - 2 * k)}, xtw[k]);
      }
    } else {
      // all row loads of the pairs first (they are independent), then the arithmetic
      constexpr int NP = (M / 2) / TPL + 1;  // pairs per thread; only b = 0 has k = M/2 in the last
      T xv[NP][4];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const int k = b + i * TPL;
        const bool ok = (i < NP - 1) || (k <= M / 2);
        int q[4];
        bool use[4] = {ok, ok, ok, ok};
        if (bc == BC_P) {
          q[0] = k == 0 ? 0 : 2 * k - 1;
          q[1] = 2 * k;
          q[2] = k == 0 ? N - 1 : 2 * (M - k) - 1;
          q[3] = 2 * (M - k);
          use[1] = use[3] = ok && k != 0;
        } else {
          const bool rev = (bc == BC_DD);
          const int qq[4] = {k, N - k, M - k, N - M + k};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            q[u] = rev ? (N - 1 - qq[u]) : qq[u];
            use[u] = ok && qq[u] < N;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[i][u] = use[u] ? X(q[u]) : (T)0;
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const int k = b + i * TPL;
        if (i == NP - 1 && k > M / 2) break;
        cplx<T> Vk, Vm;
        if (bc == BC_P) {
          Vk = {xv[i][0], -xv[i][1]};
          Vm = {xv[i][2], -xv[i][3]};
        } else {
          cplx<T> w = xtw[k];
          w.y = -w.y;
          Vk = cscale(cmul(w, cplx<T>{xv[i][0], -xv[i][1]}), (T)0.5);
          cplx<T> w2 = xtw[M - k];
          w2.y = -w2.y;
          Vm = cscale(cmul(w2, cplx<T>{xv[i][2], -xv[i][3]}), (T)0.5);
        }
        const cplx<T> Ek = cscale(cadd(Vk, conj_(Vm)), (T)0.5);
        cplx<T> wn = ptw[k];
        wn.y = -wn.y;
        const cplx<T> Ok = cscale(cmul(csub(Vk, conj_(Vm)), wn), (T)0.5);
        if (k < M) buf[k * CW + c] = cadd(Ek, mul_i(Ok));
        if (k != 0 && 2 * k != M) buf[(M - k) * CW + c] = cadd(conj_(Ek), mul_i(conj_(Ok)));
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < E; ++r) v[r] = buf[(b + r * TPL) * CW + c];
    if (bc_iv(bc)) fft_col<T, M, CW, false, 0, 1>(v, buf, stw, b, c);
    else fft_col<T, M, CW, true, 0, 1>(v, buf, stw, b, c);
    // ---- backward post-processing straight from the last stage to the rows ----
    const T inv_m = (T)1 / (T)M;
#pragma unroll
    for (int q = 0; q < E / RL; ++q) {
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int k = b + q * TPL + r * (M / RL);
        const cplx<T> zk = v[q * RL + r];
        if (bc_iv(bc)) {
          const cplx<T> cc = cmul(xtw[M + k], zk);
          const T A = cc.x * ((T)1 / (T)N) * s, B = -cc.y * ((T)1 / (T)N) * s;
          if (bc == BC_DN) {
            Y(2 * k, B);
            Y(N - 1 - 2 * k, A);
          } else {
            Y(2 * k, A);
            Y(N - 1 - 2 * k, B);
          }
        } else if (bc == BC_P) {
          Y(2 * k, zk.x * inv_m * s);
          Y(2 * k + 1, zk.y * inv_m * s);
        } else {
          const int j0 = 2 * k, j1 = 2 * k + 1;
          const int i0 = j0 < M ? 2 * j0 : 2 * N - 1 - 2 * j0;
          const int i1 = j1 < M ? 2 * j1 : 2 * N - 1 - 2 * j1;
          T v0 = zk.x * inv_m * s, v1 = zk.y * inv_m * s;
          if (bc == BC_DD) {
            if (i0 & 1) v0 = -v0;
            if (i1 & 1) v1 = -v1;
          }
          Y(i0, v0);
          Y(i1, v1);
        }
      }
    }
  }
}

}  // namespace col

}  // namespace ps
