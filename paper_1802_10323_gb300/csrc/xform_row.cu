// xform_row.cu — x-axis line transforms read and written by the warp that owns the line.
//
// Same mathematics as the other line transforms (one M-point complex FFT per
// line of n = 2M contiguous reals, with the Table 2 pre/post processing per BC).
// TPL = M/E lanes own a line (a warp, or half of one for M = 64), E complex
// points each, and nothing but the FFT exchanges goes through shared memory:
//   * Lane t's first-stage operands are the points t + TPL·j, so for each j the
//     lanes of a line touch consecutive memory. The forward gather loads its
//     operands straight from the line: P reads pairs (x_{2p}, x_{2p+1}); the
//     cosine/sine orderings read one 4-vector (x_{4p} … x_{4p+3}) that holds two
//     values of point p and two of point M−1−p, and point M−1−p is the mirrored
//     slot E−1−s of the mirrored lane t ^ (TPL−1): one shuffle hands them over.
//     The backward outputs are assembled into the same vectors the same way.
//   * The other side of each transform (forward outputs, backward inputs) pairs
//     wavenumbers k and M−k; those go through the line's exchange buffer and
//     touch memory with scalar accesses at consecutive or every-other address.
//   * A line never leaves its warp: exchanges synchronise with __syncwarp, and
//     warps stride over the lines independently (persistent grid).
#include <type_traits>

#include "xform_fast.cuh"

namespace ps {
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

template <class T, class TI, class TO, int M, bool FWD, int OM>
__global__ void __launch_bounds__(32 * WARPS, sizeof(T) == 4 ? (M >= 512 ? 3 : 4) : 2)
    xform_row_kernel(FastArgs<T> a) {
  if (a.skip && *a.skip) return;
  using S = Shape<M>;
  constexpr int N = 2 * M, E = S::E, TPL = S::TPL, LPW = 32 / TPL;
  constexpr int R0 = S::radix(0), RL = S::radix(S::NST - 1);
  constexpr int LB = M + M / 8;  // complex slots of a line's exchange buffer (skewed)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int bc = a.bc;
  cplx<T>* stw = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* ptw = stw + M;
  cplx<T>* xtw = ptw + (M + 1);
  cplx<T>* bufs = reinterpret_cast<cplx<T>*>(smem_raw + fast_table_bytes<T, M>(bc));
  for (int i = threadIdx.x; i < M; i += blockDim.x) stw[i] = a.tw[16 * i];
  for (int i = threadIdx.x; i <= M; i += blockDim.x) ptw[i] = a.tw[8 * i];
  if (bc == BC_NN || bc == BC_DD) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) xtw[i] = a.tw[2 * i];
  } else if (bc == BC_ND) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      xtw[i] = a.tw[4 * i];
      xtw[M + i] = a.tw[4 * i + 1];
    }
  }
  __syncthreads();  // the only block-wide barrier: tables ready

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane % TPL, half = lane / TPL;
  const int mate = lane ^ (TPL - 1);  // lane of the mirrored points M−1−p
  cplx<T>* lc = bufs + (warp * LPW + half) * LB;
  T* lr = reinterpret_cast<T*>(lc);
  const TI* in = static_cast<const TI*>(a.in);  // may equal out (in-place passes)
  TO* out = static_cast<TO*>(a.out);
  const int ny = a.ny, nlines = a.nlines;
  const unsigned full = 0xffffffffu;
  // max |transform output| of FP64 outputs, tracked on the values before widening
  // (exact) so that no 64-bit work per value reaches the FP64 pipe
  T tmax = (T)0;

  const int wstride = gridDim.x * WARPS * LPW;
  for (int l0 = (blockIdx.x * WARPS + warp) * LPW; l0 < nlines; l0 += wstride) {
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
      } else if (bc == BC_ND) {
        // z_p = (x_{2p}, x_{n−1−2p})·e^{−iπp/n}; x_{n−1−2p} = x_{2p'+1} of p' = M−1−p
#pragma unroll
        for (int si = 0; si < E; ++si) {
          const int p = t + (si / R0) * TPL + (si % R0) * (M / R0);
          const vec<TI, 2> x = *reinterpret_cast<const vec<TI, 2>*>(src + 2 * p);
          v[si].x = in_cvt<T>(x.v[0]) * s;
          const T odd = in_cvt<T>(x.v[1]) * s;
          v[E - 1 - si].y = __shfl_sync(full, odd, mate);
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
      if (bc == BC_ND) {
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
    } else {
      // ---- backward pre-processing: pairs (k, M−k) from the line into the buffer ----
      auto X = [&](int i) { return in_cvt<T>(src[i]); };
      if (bc == BC_ND) {
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
      if (bc == BC_ND) fast::fft_stages<T, M, false, 0, 1>(v, lc, stw, t);
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
      } else if (bc == BC_ND) {
        // output 2k = Re(c_k)/n, output n−1−2k = −Im(c_k)/n with c_k = e^{...}·z_k;
        // the pair (2k, 2k+1) takes −Im(c_{k'})/n of k' = M−1−k from the mirrored slot
        const T inv_n = (T)1 / (T)N;
        T re[E], im[E];
#pragma unroll
        for (int si = 0; si < E; ++si) {
          const int k = t + (si / RL) * TPL + (si % RL) * (M / RL);
          const cplx<T> c = cmul(xtw[M + k], v[si]);
          re[si] = c.x * inv_n;
          im[si] = -c.y * inv_n;
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
  if constexpr (sizeof(TO) == 8) {
    if (a.amax) {
      for (int o = 16; o > 0; o >>= 1) tmax = fmax(tmax, __shfl_xor_sync(full, tmax, o));
      const unsigned long long amax =
          (unsigned long long)__double_as_longlong(st_cvt<double, T>::f(tmax));  // ≥ 0: the bits order as the values
      if (lane == 0 && amax) atomicMax(a.amax, amax);
    }
  }
}

}  // namespace row

namespace {
template <class T, class TI, class TO, int M, bool FWD, int OM>
cudaError_t launch_row_mode(FastArgs<T> a, cudaStream_t st) {
  using S = fast::Shape<M>;
  constexpr int LPW = 32 / S::TPL;
  constexpr size_t LB = M + M / 8;
  auto k = row::xform_row_kernel<T, TI, TO, M, FWD, OM>;
  const size_t smem = fast_table_bytes<T, M>(a.bc) + (size_t)row::WARPS * LPW * LB * sizeof(cplx<T>);
  static int smem_set = 0;
  static int blocks_per_sm[2] = {};
  if (!smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(fast_table_bytes<T, M>(1) + row::WARPS * LPW * LB * sizeof(cplx<T>)));
    if (e != cudaSuccess) return e;
    smem_set = 1;
  }
  int& bps = blocks_per_sm[a.bc != 0];
  if (bps == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, 32 * row::WARPS, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_cta = row::WARPS * LPW;
  const int ctas = (a.nlines + per_cta - 1) / per_cta;
  const int grid = ctas < sms * bps ? ctas : sms * bps;
  (void)cudaGetLastError();  // a stale error from elsewhere must not be blamed here
  k<<<grid, 32 * row::WARPS, smem, st>>>(a);
  return cudaGetLastError();
}
}  // namespace

template <class T, class TI, class TO, int M, bool FWD>
cudaError_t launch_xform_row(FastArgs<T> a, cudaStream_t st) {
  if (a.axis != 0 || a.nx != 2 * M) return cudaErrorInvalidValue;
  if constexpr (!FWD && sizeof(TO) == 8 && sizeof(T) == 4) {
    if (a.base32) return launch_row_mode<T, TI, TO, M, FWD, row::OM_BASE>(a, st);
    if (!a.out) return launch_row_mode<T, TI, TO, M, FWD, row::OM_NONE>(a, st);
  }
  if (a.accumulate) return launch_row_mode<T, TI, TO, M, FWD, row::OM_ACC>(a, st);
  return launch_row_mode<T, TI, TO, M, FWD, row::OM_STORE>(a, st);
}

#define PS_ROW_INST(M)                                                                                   \
  template cudaError_t launch_xform_row<double, double, double, M, true>(FastArgs<double>, cudaStream_t); \
  template cudaError_t launch_xform_row<double, double, double, M, false>(FastArgs<double>, cudaStream_t); \
  template cudaError_t launch_xform_row<float, float, float, M, true>(FastArgs<float>, cudaStream_t);     \
  template cudaError_t launch_xform_row<float, float, float, M, false>(FastArgs<float>, cudaStream_t);    \
  template cudaError_t launch_xform_row<float, double, float, M, true>(FastArgs<float>, cudaStream_t);    \
  template cudaError_t launch_xform_row<float, float, double, M, false>(FastArgs<float>, cudaStream_t);

PS_ROW_INST(64)
PS_ROW_INST(128)
PS_ROW_INST(256)
PS_ROW_INST(512)

}  // namespace ps
