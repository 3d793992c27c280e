// xform_fast.cu — kernel body of the register-resident line transforms (see xform_fast.cuh).
#include "xform_fast.cuh"

#include <stdio.h>

namespace ps {

thread_local char g_launch_diag[256] = "";

// Asynchronous global→shared copies (cp.async): 16-byte and element-sized.
__device__ __forceinline__ void cpa16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
template <int B>
__device__ __forceinline__ void cpa_elem(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(B));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cpa_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Vector of N elements of T for one shared-memory access.
template <class T, int N>
struct alignas(sizeof(T) * N) svec {
  T v[N];
};

using fast::Shape;
using fast::cpad;

template <class T, class TI, class TO, int M, bool FWD>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) xform_fast_kernel(FastArgs<T> a) {
  if (a.skip && *a.skip) return;
  constexpr int N = 2 * M;
  constexpr int E = Shape<M>::E, TPL = Shape<M>::TPL;
  constexpr int LD = N + N / 8 + (sizeof(T) == 4 ? 4 : 2);  // reals per line buffer (16-byte rows; room for the skewed complex view)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int bc = a.bc;
  const int lpc = a.lpc;
  // ---- tables ----
  cplx<T>* stw = reinterpret_cast<cplx<T>*>(smem_raw);  // ω_M^t, t < M
  cplx<T>* ptw = stw + M;                               // e^{−2πik/n}, k ≤ M  (P, NN, DD)
  cplx<T>* xtw = ptw + (M + 1);                         // NN/DD: e^{−iπq/2n}, q < n; ND: pre, post
  T* lines = reinterpret_cast<T*>(smem_raw + fast_table_bytes<T, M>(bc));
  // FP32 passes whose input is FP32 stream the next group into a second buffer
  constexpr bool kAsyncType = (sizeof(T) == 4) && (sizeof(TI) == sizeof(T));
  const bool async_in = kAsyncType && a.axis == 0 && !(FWD && a.plane_scale);
  T* lines_alt = lines + lpc * LD;
  for (int i = threadIdx.x; i < M; i += blockDim.x) stw[i] = a.tw[16 * i];
  for (int i = threadIdx.x; i <= M; i += blockDim.x) ptw[i] = a.tw[8 * i];
  if (bc == BC_NN || bc == BC_DD) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) xtw[i] = a.tw[2 * i];
  } else if (bc_iv(bc)) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      xtw[i] = a.tw[4 * i];          // e^{−iπr/n}
      xtw[M + i] = a.tw[4 * i + 1];  // e^{−iπ(4k+1)/4n}
    }
  }
  const int li = threadIdx.x / TPL;  // line within the CTA
  const int t = threadIdx.x % TPL;
  const TI* __restrict__ in = static_cast<const TI*>(a.in);
  TO* __restrict__ out = static_cast<TO*>(a.out);
  const int nx = a.nx, ny = a.ny;
  const int ngroups = (a.axis == 0) ? (a.nlines + lpc - 1) / lpc : a.nz * (nx / lpc);
  constexpr int VI = 16 / sizeof(TI);  // input elements per 16-byte load
  constexpr int VO = 16 / sizeof(TO);
  unsigned long long amax = 0;  // max |value| bits of FP64 outputs (when requested)

  // issue the asynchronous load of group gg into buffer dst
  auto issue = [&](int gg, T* dst) {
    if (a.axis == 0) {
      const int nlg = min(lpc, a.nlines - gg * lpc);
      const T* src = reinterpret_cast<const T*>(in) + (size_t)gg * lpc * N;
      constexpr int V = 16 / sizeof(T);
      for (int v = threadIdx.x; v < nlg * N / V; v += blockDim.x) {
        const int l = v / (N / V), e = (v % (N / V)) * V;
        cpa16(dst + l * LD + e, src + (size_t)v * V);
      }
    } else {
      const int gpz = nx / lpc;
      const int zz = gg / gpz, xx = (gg - zz * gpz) * lpc;
      const T* src = reinterpret_cast<const T*>(in) + (size_t)zz * ny * nx + xx;
      for (int v = threadIdx.x; v < N * lpc; v += blockDim.x) {
        const int e = v / lpc, c = v - e * lpc;
        cpa_elem<sizeof(T)>(dst + c * LD + e, src + (size_t)e * nx + c);
      }
    }
    cpa_commit();
  };
  if (async_in && (int)blockIdx.x < ngroups) issue(blockIdx.x, lines);

  int it = 0;
  for (int g = blockIdx.x; g < ngroups; g += gridDim.x, ++it) {
    T* cur = (async_in && (it & 1)) ? lines_alt : lines;
    T* lr = cur + li * LD;                          // this line's reals
    cplx<T>* lc = reinterpret_cast<cplx<T>*>(lr);  // same buffer as M complex
    __syncthreads();  // tables ready / previous group's store done
    // ---- stage in ----
    int zb = 0, x0 = 0;
    int nl = lpc;
    if (a.axis == 1) {
      const int gpz = nx / lpc;
      zb = g / gpz;
      x0 = (g - zb * gpz) * lpc;
    } else {
      nl = min(lpc, a.nlines - g * lpc);
    }
    if (async_in) {
      const int gn = g + gridDim.x;
      if (gn < ngroups) issue(gn, (it & 1) ? lines : lines_alt);
      else cpa_commit();  // empty group keeps the wait count uniform
      cpa_wait1();
    } else if (a.axis == 0) {
      const size_t base = (size_t)g * lpc * N;
      const int nvec = nl * N / VI;
      for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
        const int l = v / (N / VI), e = (v % (N / VI)) * VI;
        TI buf[VI];
        *reinterpret_cast<uint4*>(buf) = *reinterpret_cast<const uint4*>(in + base + (size_t)v * VI);
        T s = (T)1;
        if (FWD && a.plane_scale) s = a.plane_scale[(g * lpc + l) / ny];
        svec<T, VI> sv;
#pragma unroll
        for (int u = 0; u < VI; ++u) sv.v[u] = ld_cvt<T, TI>::f(buf[u]) * s;
        *reinterpret_cast<svec<T, VI>*>(&cur[l * LD + e]) = sv;
      }
    } else {
      const size_t base = (size_t)zb * ny * nx + x0;
      const int vpr = lpc / VI;  // vectors per row
      T s = (T)1;
      if (FWD && a.plane_scale) s = a.plane_scale[zb];
      for (int v = threadIdx.x; v < N * vpr; v += blockDim.x) {
        const int e = v / vpr, c = (v % vpr) * VI;
        TI buf[VI];
        *reinterpret_cast<uint4*>(buf) = *reinterpret_cast<const uint4*>(in + base + (size_t)e * nx + c);
#pragma unroll
        for (int u = 0; u < VI; ++u) cur[(c + u) * LD + e] = ld_cvt<T, TI>::f(buf[u]) * s;
      }
    }
    __syncthreads();

    // every lane runs the line code (lines past the end compute on stale data and
    // are not stored), so __syncwarp always sees the full warp
    {
      cplx<T> v[E];
      if (FWD) {
        // ---- pre-processing gathered straight into the stage-1 operands ----
        constexpr int R0 = Shape<M>::radix(0);
#pragma unroll
        for (int q = 0; q < E / R0; ++q) {
#pragma unroll
          for (int r = 0; r < R0; ++r) {
            const int p = t + q * TPL + r * (M / R0);
            cplx<T> z;
            if (bc == BC_P) {
              z = *reinterpret_cast<const cplx<T>*>(&lr[2 * p]);
            } else if (bc_iv(bc)) {  // DN: the reversed line, the two reals swap
              const T e0 = lr[2 * p], e1 = lr[N - 1 - 2 * p];
              z = cmul(bc == BC_DN ? cplx<T>{e1, e0} : cplx<T>{e0, e1}, xtw[p]);
            } else {
              const int j0 = 2 * p, j1 = 2 * p + 1;
              T v0 = lr[j0 < M ? 2 * j0 : 2 * N - 1 - 2 * j0];
              T v1 = lr[j1 < M ? 2 * j1 : 2 * N - 1 - 2 * j1];
              if (bc == BC_DD) {
                if (j0 >= M) v0 = -v0;
                if (j1 >= M) v1 = -v1;
              }
              z = {v0, v1};
            }
            v[q * R0 + r] = z;
          }
        }
        fast::fft_stages<T, M, false, 0, 1>(v, lc, stw, t);
        // ---- post-processing ----
        constexpr int RL = Shape<M>::radix(Shape<M>::NST - 1);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < E / RL; ++q)
#pragma unroll
          for (int r = 0; r < RL; ++r) lc[cpad(t + q * TPL + r * (M / RL))] = v[q * RL + r];
        __syncwarp();
        if (bc_iv(bc)) {
          cplx<T> c[E];
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const int k = t + i * TPL;
            c[i] = cmul(xtw[M + k], lc[cpad(k)]);
          }
          __syncwarp();
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const int k = t + i * TPL;
            lr[2 * k] = (T)2 * c[i].x;
            lr[N - 1 - 2 * k] = (T)-2 * c[i].y;
          }
        } else {
          // pairs (k, M−k), k = 0 … M/2: V_k = A + B, V_{M−k} = conj(A − B)
          constexpr int NP = (M / 2) / TPL + 1;
          cplx<T> Vk[NP], Vmk[NP];
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            const int k = t + i * TPL;
            if (k > M / 2) break;
            const cplx<T> Zk = lc[cpad(k)], Zmk = lc[cpad(k == 0 ? 0 : M - k)];
            const cplx<T> Ek = cscale(cadd(Zk, conj_(Zmk)), (T)0.5);
            const cplx<T> Ok = cscale(mul_mi(csub(Zk, conj_(Zmk))), (T)0.5);
            const cplx<T> B = cmul(ptw[k], Ok);
            Vk[i] = cadd(Ek, B);
            Vmk[i] = conj_(csub(Ek, B));
          }
          __syncwarp();
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            const int k = t + i * TPL;
            if (k > M / 2) break;
            if (bc == BC_P) {
              if (k == 0) {
                lr[0] = Vk[i].x;
                lr[N - 1] = Vmk[i].x;
              } else {
                lr[2 * k - 1] = Vk[i].x;
                lr[2 * k] = -Vk[i].y;
                if (2 * k != M) {
                  lr[2 * (M - k) - 1] = Vmk[i].x;
                  lr[2 * (M - k)] = -Vmk[i].y;
                }
              }
            } else {
              const bool rev = (bc == BC_DD);
#define OUTQ(q, val) lr[rev ? (N - 1 - (q)) : (q)] = (val)
              if (k == 0) {
                OUTQ(0, (T)2 * Vk[i].x);
                OUTQ(M, (T)1.41421356237309504880 * Vmk[i].x);
              } else {
                const cplx<T> c1 = cmul(xtw[k], Vk[i]);
                OUTQ(k, (T)2 * c1.x);
                OUTQ(N - k, (T)-2 * c1.y);
                if (2 * k != M) {
                  const cplx<T> c2 = cmul(xtw[M - k], Vmk[i]);
                  OUTQ(M - k, (T)2 * c2.x);
                  OUTQ(M + k, (T)-2 * c2.y);
                }
              }
#undef OUTQ
            }
          }
        }
      } else {
        // ---- backward pre-processing into the complex buffer ----
        if (bc_iv(bc)) {
          cplx<T> z[E];
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const int k = t + i * TPL;
            z[i] = cmul(cplx<T>{lr[2 * k], lr[N - 1 - 2 * k]}, xtw[k]);
          }
          __syncwarp();
#pragma unroll
          for (int i = 0; i < E; ++i) lc[cpad(t + i * TPL)] = z[i];
        } else {
          constexpr int NP = (M / 2) / TPL + 1;
          cplx<T> Zk[NP], Zmk[NP];
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            const int k = t + i * TPL;
            if (k > M / 2) break;
            cplx<T> Vk, Vm;
            if (bc == BC_P) {
              if (k == 0) {
                Vk = {lr[0], (T)0};
                Vm = {lr[N - 1], (T)0};
              } else {
                Vk = {lr[2 * k - 1], -lr[2 * k]};
                Vm = {lr[2 * (M - k) - 1], -lr[2 * (M - k)]};
              }
            } else {
              const bool rev = (bc == BC_DD);
#define XQ(q) ((q) >= N ? (T)0 : lr[rev ? (N - 1 - (q)) : (q)])
              cplx<T> w = xtw[k];
              w.y = -w.y;
              Vk = cscale(cmul(w, cplx<T>{XQ(k), -XQ(N - k)}), (T)0.5);
              cplx<T> w2 = xtw[M - k];
              w2.y = -w2.y;
              Vm = cscale(cmul(w2, cplx<T>{XQ(M - k), -XQ(N - M + k)}), (T)0.5);
#undef XQ
            }
            const cplx<T> Ek = cscale(cadd(Vk, conj_(Vm)), (T)0.5);
            cplx<T> wn = ptw[k];
            wn.y = -wn.y;
            const cplx<T> Ok = cscale(cmul(csub(Vk, conj_(Vm)), wn), (T)0.5);
            Zk[i] = cadd(Ek, mul_i(Ok));
            Zmk[i] = cadd(conj_(Ek), mul_i(conj_(Ok)));
          }
          __syncwarp();
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            const int k = t + i * TPL;
            if (k > M / 2) break;
            if (k < M) lc[cpad(k)] = Zk[i];
            if (k != 0 && 2 * k != M) lc[cpad(M - k)] = Zmk[i];
          }
        }
        __syncwarp();
        constexpr int R0 = Shape<M>::radix(0);
#pragma unroll
        for (int q = 0; q < E / R0; ++q)
#pragma unroll
          for (int r = 0; r < R0; ++r) v[q * R0 + r] = lc[cpad(t + q * TPL + r * (M / R0))];
        if (bc_iv(bc)) fast::fft_stages<T, M, false, 0, 1>(v, lc, stw, t);
        else fast::fft_stages<T, M, true, 0, 1>(v, lc, stw, t);
        // ---- backward post-processing straight from the last stage's outputs ----
        constexpr int RL = Shape<M>::radix(Shape<M>::NST - 1);
        __syncwarp();
        const T inv_m = (T)1 / (T)M;
#pragma unroll
        for (int q = 0; q < E / RL; ++q) {
#pragma unroll
          for (int r = 0; r < RL; ++r) {
            const int k = t + q * TPL + r * (M / RL);
            const cplx<T> zk = v[q * RL + r];
            if (bc_iv(bc)) {
              const cplx<T> c = cmul(xtw[M + k], zk);
              const T A = c.x * ((T)1 / (T)N), B = -c.y * ((T)1 / (T)N);  // DN: trade places
              lr[2 * k] = (bc == BC_DN) ? B : A;
              lr[N - 1 - 2 * k] = (bc == BC_DN) ? A : B;
            } else if (bc == BC_P) {
              lr[2 * k] = zk.x * inv_m;
              lr[2 * k + 1] = zk.y * inv_m;
            } else {
              const int j0 = 2 * k, j1 = 2 * k + 1;
              const int i0 = j0 < M ? 2 * j0 : 2 * N - 1 - 2 * j0;
              const int i1 = j1 < M ? 2 * j1 : 2 * N - 1 - 2 * j1;
              T v0 = zk.x * inv_m, v1 = zk.y * inv_m;
              if (bc == BC_DD) {
                if (i0 & 1) v0 = -v0;
                if (i1 & 1) v1 = -v1;
              }
              lr[i0] = v0;
              lr[i1] = v1;
            }
          }
        }
      }
    }
    __syncthreads();

    // ---- stage out ----
    if (a.axis == 0) {
      const size_t base = (size_t)g * lpc * N;
      const int nvec = nl * N / VO;
      for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
        const int l = v / (N / VO), e = (v % (N / VO)) * VO;
        T s = (T)1;
        if (!FWD && a.plane_scale) s = a.plane_scale[(g * lpc + l) / ny];
        TO ob[VO];
        TO* dst = out + base + (size_t)v * VO;
        if (a.accumulate) *reinterpret_cast<uint4*>(ob) = *reinterpret_cast<const uint4*>(dst);
        const svec<T, VO> sv = *reinterpret_cast<const svec<T, VO>*>(&cur[l * LD + e]);
#pragma unroll
        for (int u = 0; u < VO; ++u) {
          const TO val = st_cvt<TO, T>::f(sv.v[u] * s);
          ob[u] = a.accumulate ? ob[u] + val : val;
          if constexpr (sizeof(TO) == 8)
            amax = max(amax, (unsigned long long)__double_as_longlong(ob[u]) & 0x7FFFFFFFFFFFFFFFull);
        }
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(ob);
      }
    } else {
      const size_t base = (size_t)zb * ny * nx + x0;
      const int vpr = lpc / VO;
      T s = (T)1;
      if (!FWD && a.plane_scale) s = a.plane_scale[zb];
      for (int v = threadIdx.x; v < N * vpr; v += blockDim.x) {
        const int e = v / vpr, c = (v % vpr) * VO;
        TO ob[VO];
        TO* dst = out + base + (size_t)e * nx + c;
        if (a.accumulate) *reinterpret_cast<uint4*>(ob) = *reinterpret_cast<const uint4*>(dst);
#pragma unroll
        for (int u = 0; u < VO; ++u) {
          const TO val = st_cvt<TO, T>::f(cur[(c + u) * LD + e] * s);
          ob[u] = a.accumulate ? ob[u] + val : val;
          if constexpr (sizeof(TO) == 8)
            amax = max(amax, (unsigned long long)__double_as_longlong(ob[u]) & 0x7FFFFFFFFFFFFFFFull);
        }
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(ob);
      }
    }
  }
  if (async_in) asm volatile("cp.async.wait_group 0;\n" ::);
  if constexpr (sizeof(TO) == 8) {
    if (a.amax) {
      for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if ((threadIdx.x & 31) == 0 && amax) atomicMax(a.amax, amax);
    }
  }
}

template <class T, class TI, class TO, int M, bool FWD>
cudaError_t launch_xform_fast(FastArgs<T> a, cudaStream_t st) {
  constexpr int N = 2 * M;
  constexpr int TPL = Shape<M>::TPL;
  constexpr int LD = N + N / 8 + (sizeof(T) == 4 ? 4 : 2);
  if (a.axis == 0) a.lpc = 256 / TPL;
  else a.lpc = (sizeof(T) == 4 && sizeof(TI) == 4 && sizeof(TO) == 4) ? 16 : 8;
  const int threads = a.lpc * TPL;
  constexpr bool kAsyncType = (sizeof(T) == 4) && (sizeof(TI) == sizeof(T));
  const bool async_in = kAsyncType && a.axis == 0 && !(FWD && a.plane_scale);
  const size_t smem = fast_table_bytes<T, M>(a.bc) + (size_t)(async_in ? 2 : 1) * a.lpc * LD * sizeof(T);
  auto k = xform_fast_kernel<T, TI, TO, M, FWD>;
  // One instantiation serves both axes with different tile sizes: the dynamic
  // shared-memory cap is set once, to the larger of the two configurations.
  static int smem_set = 0;
  static int blocks_per_sm[2][2][2] = {};  // [axis][bc != P][async]
  if (!smem_set) {
    const size_t tables = fast_table_bytes<T, M>(1);
    const size_t lx = 256 / TPL, ly = (sizeof(T) == 4 && sizeof(TI) == 4 && sizeof(TO) == 4) ? 16 : 8;
    const size_t sx = (kAsyncType ? 2 : 1) * lx, smax = tables + (sx > ly ? sx : ly) * LD * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    if (e != cudaSuccess) return e;
    smem_set = 1;
  }
  int& bps = blocks_per_sm[a.axis][a.bc != 0][async_in ? 1 : 0];
  if (bps == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, threads, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ngroups = (a.axis == 0) ? (a.nlines + a.lpc - 1) / a.lpc : a.nz * (a.nx / a.lpc);
  const int grid = min(ngroups, sms * bps);
  cudaError_t pre = cudaGetLastError();  // a stale error from elsewhere must not be blamed here
  k<<<grid, threads, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || pre != cudaSuccess) {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, k);
    snprintf(g_launch_diag, sizeof(g_launch_diag),
             "M=%d axis=%d lpc=%d threads=%d smem=%zu grid=%d bps=%d regs=%d maxthr=%d pre=%s",
             M, a.axis, a.lpc, threads, smem, grid, bps, fa.numRegs, fa.maxThreadsPerBlock,
             cudaGetErrorString(pre));
  }
  return e;
}

#define PS_FAST_INST(M)                                                                  \
  template cudaError_t launch_xform_fast<double, double, double, M, true>(FastArgs<double>, cudaStream_t); \
  template cudaError_t launch_xform_fast<double, double, double, M, false>(FastArgs<double>, cudaStream_t); \
  template cudaError_t launch_xform_fast<float, float, float, M, true>(FastArgs<float>, cudaStream_t);     \
  template cudaError_t launch_xform_fast<float, float, float, M, false>(FastArgs<float>, cudaStream_t);    \
  template cudaError_t launch_xform_fast<float, double, float, M, true>(FastArgs<float>, cudaStream_t);    \
  template cudaError_t launch_xform_fast<float, float, double, M, false>(FastArgs<float>, cudaStream_t);

PS_FAST_INST(64)
PS_FAST_INST(128)
PS_FAST_INST(256)
PS_FAST_INST(512)

}  // namespace ps
