// xform_col.cu — y-axis line transforms with the lines spread across lanes.
//
// Same mathematics as the other line transforms (one M-point complex FFT per
// line of n = 2M reals, with the Table 2 pre/post processing per BC), laid out
// for lines that are strided in memory. A CTA owns CW = 16 consecutive x columns
// of one z plane: lane c of each half-warp is column x0 + c, and the TPL threads
// that share a column split its line, E = M/TPL complex points each.
//   * Every global access is a row segment of CW consecutive x values (64 bytes
//     in FP32), and the BC pre/post processing happens at that interface: the
//     forward transform gathers its first-stage operands straight from the
//     permuted rows, and both directions write their outputs straight to rows.
//     No shared-memory transpose of the lines is needed.
//   * Stockham stages of radix R | E with the operands in registers; between
//     stages the line goes through a shared buffer laid out [index][column], so
//     each half-warp reads or writes 16 consecutive complex values: two
//     wavefronts per warp access, whatever the index pattern.
//   * A column's threads span several warps, so the exchanges synchronise the
//     CTA; twiddles come from shared tables loaded once per persistent CTA.
#include "xform_fast.cuh"

namespace ps {
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

template <class T, int M, bool FWD, int CW>
__global__ void __launch_bounds__(CShape<M, CW>::NT, sizeof(T) == 4 ? 1024 / CShape<M, CW>::NT : 1)
    xform_col_kernel(FastArgs<T> a) {
  if (a.skip && *a.skip) return;
  using S = CShape<M, CW>;
  constexpr int N = 2 * M, E = S::E, TPL = S::TPL;
  static_assert(S::radix(0) == E, "the first stage takes all of a thread's points");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int bc = a.bc;
  cplx<T>* stw = reinterpret_cast<cplx<T>*>(smem_raw);  // ω_M^t, t < M
  cplx<T>* ptw = stw + M;                               // e^{−2πik/n}, k ≤ M
  cplx<T>* xtw = ptw + (M + 1);                         // NN/DD: e^{−iπq/2n}, q < n; ND: pre, post
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw + fast_table_bytes<T, M>(bc));  // [M][CW]
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
  const int c = threadIdx.x % CW, b = threadIdx.x / CW;
  const T* in = static_cast<const T*>(a.in);  // may equal out (in-place y passes)
  T* out = static_cast<T*>(a.out);
  const int nx = a.nx, ny = a.ny;
  const int tpz = nx / CW;
  const int ntiles = a.nz * tpz;
  constexpr int RL = S::radix(S::NST - 1);

  for (int g = blockIdx.x; g < ntiles; g += gridDim.x) {
    const int zb = g / tpz, x0 = (g - zb * tpz) * CW;
    const T* src = in + (size_t)zb * ny * nx + x0 + c;  // row q of this column: src[q·nx]
    T* dst = out + (size_t)zb * ny * nx + x0 + c;
    // row offsets fit in 32 bits (n_y·n_x ≤ 2^20)
    auto X = [&](int q) { return src[q * nx]; };
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
        } else if (bc == BC_ND) {
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
      if (bc == BC_ND) {
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
      if (bc == BC_ND) {
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
      if (bc == BC_ND) fft_col<T, M, CW, false, 0, 1>(v, buf, stw, b, c);
      else fft_col<T, M, CW, true, 0, 1>(v, buf, stw, b, c);
      // ---- backward post-processing straight from the last stage to the rows ----
      const T inv_m = (T)1 / (T)M;
#pragma unroll
      for (int q = 0; q < E / RL; ++q) {
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int k = b + q * TPL + r * (M / RL);
          const cplx<T> zk = v[q * RL + r];
          if (bc == BC_ND) {
            const cplx<T> cc = cmul(xtw[M + k], zk);
            Y(2 * k, cc.x * ((T)1 / (T)N) * s);
            Y(N - 1 - 2 * k, -cc.y * ((T)1 / (T)N) * s);
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
}

}  // namespace col

namespace {
template <class T, int M, bool FWD, int CW>
cudaError_t launch_col_cw(FastArgs<T> a, cudaStream_t st) {
  using S = col::CShape<M, CW>;
  auto k = col::xform_col_kernel<T, M, FWD, CW>;
  const size_t smem = col::col_smem<T, M, CW>(a.bc);
  static int smem_set = 0;
  static int blocks_per_sm[2] = {};  // [bc != P]
  if (!smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)col::col_smem<T, M, CW>(1));
    if (e != cudaSuccess) return e;
    smem_set = 1;
  }
  int& bps = blocks_per_sm[a.bc != 0];
  if (bps == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, S::NT, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = a.nz * (a.nx / CW);
  const int grid = ntiles < sms * bps ? ntiles : sms * bps;
  (void)cudaGetLastError();  // a stale error from elsewhere must not be blamed here
  k<<<grid, S::NT, smem, st>>>(a);
  return cudaGetLastError();
}
}  // namespace

// Tiles of 16 columns: 64-byte rows in FP32, 128-byte rows in FP64.
template <class T, int M, bool FWD>
cudaError_t launch_xform_col(FastArgs<T> a, cudaStream_t st) {
  constexpr int CW = 16;  // (measured at 1024^3: 8 and 32 columns are slower)
  if (a.axis != 1 || a.ny != 2 * M || a.nx % CW != 0 || a.accumulate || a.amax)
    return cudaErrorInvalidValue;
  return launch_col_cw<T, M, FWD, CW>(a, st);
}

#define PS_COL_INST(M)                                                                              \
  template cudaError_t launch_xform_col<float, M, true>(FastArgs<float>, cudaStream_t);           \
  template cudaError_t launch_xform_col<float, M, false>(FastArgs<float>, cudaStream_t);          \
  template cudaError_t launch_xform_col<double, M, true>(FastArgs<double>, cudaStream_t);         \
  template cudaError_t launch_xform_col<double, M, false>(FastArgs<double>, cudaStream_t);

PS_COL_INST(64)
PS_COL_INST(128)
PS_COL_INST(256)
PS_COL_INST(512)

}  // namespace ps
