// xform_dev.cuh — device code of the generic line transforms (Table 2) along x or y.
//
// Every transform of length n (even) is reduced to one complex FFT of length
// m = n/2 done in shared memory (Stockham, radix 4/2/3), with BC-specific
// pre- and post-processing:
//   P   (DFT, half-complex layout): z_p = a_2p + i a_2p+1, then the standard
//        even/odd split X_k = E_k + e^{−2πik/n} O_k.
//   NN  (DCT-II / DCT-III): Makhoul's reordering v_j = a_2j, v_{n−1−j} = a_2j+1,
//        a real DFT of v, then X_q = 2 Re(e^{−iπq/2n} V_q).
//   DD  (DST-II / DST-III): DST-II(a)_q = DCT-II((−1)^p a_p)_{n−1−q}.
//   ND  (DCT-IV): u_r = (a_2r + i a_{n−1−2r}) e^{−iπr/n}, U = FFT_m(u),
//        X_2k = 2 Re(c_k), X_{n−1−2k} = −2 Im(c_k), c_k = e^{−iπ(4k+1)/4n} U_k;
//        DCT-IV is its own inverse up to 2n.
//   FD  (x/y face unknowns, DST-I of the interior, the wall entry copied): the odd
//        extension y of length 2n (y_0 = y_n = 0, y_t = a_t, y_{2n−t} = −a_t) is a
//        real sequence whose DFT is Y_k = −2i Σ_t a_t sin(πtk/n); it is done as an
//        FFT of m = n complex points z_j = y_2j + i y_2j+1 and the real-DFT split
//        Y_k = E_k + e^{−iπk/n} O_k, giving X_k = −Im(Y_k). DST-I is its own inverse
//        up to 2n, so the backward transform is the same with the factor 1/(2n).
// Backward transforms include Table 1's normalisation (1/n or 1/2n).
//
// One CTA transforms L lines. x-lines are contiguous rows of the
// [n_z][n_y][n_x] array; y-lines are strided by n_x and a CTA takes L
// consecutive x columns of one z plane, so its global loads and stores are
// coalesced across the L columns (the transposes of the pencil algorithm of
// §3 become this strided tiling).
#pragma once
#include "internal.h"

namespace ps {

template <class T, bool INV>
__device__ __forceinline__ void bfly2(cplx<T>* v) {
  cplx<T> a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <class T, bool INV>
__device__ __forceinline__ void bfly4(cplx<T>* v) {
  cplx<T> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  cplx<T> t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
  t3 = INV ? mul_i(t3) : mul_mi(t3);
  v[0] = cadd(t0, t2);
  v[1] = cadd(t1, t3);
  v[2] = csub(t0, t2);
  v[3] = csub(t1, t3);
}

template <class T, bool INV>
__device__ __forceinline__ void bfly3(cplx<T>* v) {
  const T s3 = (T)0.86602540378443864676;  // sin(π/3)
  cplx<T> t = cadd(v[1], v[2]);
  cplx<T> d = csub(v[1], v[2]);
  cplx<T> x0 = cadd(v[0], t);
  cplx<T> u = {v[0].x - (T)0.5 * t.x, v[0].y - (T)0.5 * t.y};
  cplx<T> w = INV ? mul_i(cscale(d, s3)) : mul_mi(cscale(d, s3));
  v[0] = x0;
  v[1] = cadd(u, w);
  v[2] = csub(u, w);
}

// One Stockham stage of radix R over L lines of m points (row stride ld).
// tw is the 8n-entry table e^{−2πi t/(8n)}; ω_m^x = tw[twm·x] with twm = 8n/m
// (16 for the m = n/2 FFTs, 8 for the m = n FFT of a face-centred line).
template <class T, int R, bool INV>
__device__ __forceinline__ void stage(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst,
                                      int L, int m, int ld, int Ns, const cplx<T>* __restrict__ tw, int twm) {
  const int nb = m / R;
  const int tws = m / (Ns * R);
  for (int idx = threadIdx.x; idx < L * nb; idx += blockDim.x) {
    const int l = idx / nb;
    const int j = idx - l * nb;
    const int k = j % Ns;
    const cplx<T>* s = src + l * ld;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[j + r * nb];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = tw[twm * (r * k * tws)];
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    if constexpr (R == 2) bfly2<T, INV>(v);
    if constexpr (R == 3) bfly3<T, INV>(v);
    if constexpr (R == 4) bfly4<T, INV>(v);
    cplx<T>* d = dst + l * ld + (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[r * Ns] = v[r];
  }
}

// Makhoul index map: position j of v ↔ position of a.
__device__ __forceinline__ int mk_idx(int j, int n, int m) { return j < m ? 2 * j : 2 * n - 1 - 2 * j; }

// Transforms line group `grp` (x: rows grp*L …; y: L columns of one z plane);
// every thread of the CTA takes part; smem_raw holds 2·L·(m+1) complex values.
template <class T, class TI, class TO, bool FWD>
__device__ void xform_group(const XformArgs<T>& a, int grp, unsigned char* smem_raw) {
  const int n = a.n, m = a.m, L = a.L, ld = m + 1, ldr = 2 * ld;
  cplx<T>* bufA = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* bufB = bufA + L * ld;
  // no __restrict__: in and out may be the same array, and in the batched kernel
  // other CTAs rewrite it between tasks (the read-only cache path must not be used)
  const TI* in = static_cast<const TI*>(a.in);
  TO* out = static_cast<TO*>(a.out);
  const cplx<T>* __restrict__ tw = a.tw;
  const int nx = a.nx, ny = a.ny;

  // ---- line addressing -------------------------------------------------------
  // x: line index ln = grp*L + l is the row (z*ny + y); element e at ln*n + e.
  // y: grp = z*(nx/L) + xg; line l is column x = xg*L + l; element e at
  //    z*ny*nx + e*nx + x.
  const int gpz = nx / L;  // y only
  const int zb = (a.axis == 1) ? grp / gpz : 0;
  const int x0 = (a.axis == 1) ? (grp - zb * gpz) * L : 0;
  const size_t ybase = (size_t)zb * ny * nx + x0;
  const int nlines_here = (a.axis == 0) ? min(L, a.nlines - (int)grp * L) : L;

  // ---- 1. load (into bufB as reals) -------------------------------------------
  T* rB = reinterpret_cast<T*>(bufB);
  for (int idx = threadIdx.x; idx < L * n; idx += blockDim.x) {
    int l, e;
    size_t g;
    int z;
    if (a.axis == 0) {
      l = idx / n;
      e = idx - l * n;
      if (l >= nlines_here) continue;
      size_t ln = (size_t)grp * L + l;
      g = ln * n + e;
      z = (int)(ln / ny);
    } else {
      e = idx / L;
      l = idx - e * L;
      g = ybase + (size_t)e * nx + l;
      z = zb;
    }
    T v = ld_cvt<T, TI>::f(in[g]);
    if (FWD && a.plane_scale) v *= a.plane_scale[z];
    rB[l * ldr + e] = v;
  }
  __syncthreads();

  // ---- 2. pre-processing: reals (bufB) -> m complex points (bufA) ---------------
  const int bc = a.bc;
  if (bc == BC_FD) {  // both directions: z_j = (y_2j, y_2j+1) of the odd extension (m = n)
    for (int idx = threadIdx.x; idx < L * m; idx += blockDim.x) {
      const int l = idx / m, j = idx - l * m;
      const T* x = rB + l * ldr;
      auto y = [&](int t) -> T { return (t == 0 || t == n) ? (T)0 : (t < n ? x[t] : -x[2 * n - t]); };
      bufA[l * ld + j] = cplx<T>{y(2 * j), y(2 * j + 1)};
      if (j == 0) bufA[l * ld + m] = cplx<T>{x[0], (T)0};  // the wall entry, in the slot no stage writes
    }
  } else if (FWD) {
    for (int idx = threadIdx.x; idx < L * m; idx += blockDim.x) {
      const int l = idx / m, p = idx - l * m;
      const T* x = rB + l * ldr;
      cplx<T> z;
      if (bc == BC_P) {
        z = {x[2 * p], x[2 * p + 1]};
      } else if (bc == BC_NN || bc == BC_DD) {
        const int j0 = 2 * p, j1 = 2 * p + 1;
        T v0 = x[mk_idx(j0, n, m)], v1 = x[mk_idx(j1, n, m)];
        if (bc == BC_DD) {  // (−1)^index: odd a-indices come from j ≥ m
          if (j0 >= m) v0 = -v0;
          if (j1 >= m) v1 = -v1;
        }
        z = {v0, v1};
      } else {  // ND (DN: the reversed line, the two reals swap)
        const T e0 = x[2 * p], e1 = x[n - 1 - 2 * p];
        z = cmul(bc == BC_DN ? cplx<T>{e1, e0} : cplx<T>{e0, e1}, tw[4 * p]);
      }
      bufA[l * ld + p] = z;
    }
  } else {
    const int np = bc_iv(bc) ? m : (m / 2 + 1);
    for (int idx = threadIdx.x; idx < L * np; idx += blockDim.x) {
      const int l = idx / np, k = idx - l * np;
      const T* X = rB + l * ldr;
      cplx<T>* Z = bufA + l * ld;
      if (bc_iv(bc)) {
        Z[k] = cmul(cplx<T>{X[2 * k], X[n - 1 - 2 * k]}, tw[4 * k]);
        continue;
      }
      // spectrum V_k and V_{m−k} of the real sequence whose half-length FFT we invert
      cplx<T> Vk, Vmk;
      if (bc == BC_P) {
        if (k == 0) {
          Vk = {X[0], (T)0};
          Vmk = {X[n - 1], (T)0};
        } else {
          Vk = {X[2 * k - 1], -X[2 * k]};
          Vmk = {X[2 * (m - k) - 1], -X[2 * (m - k)]};
        }
      } else {
        // DCT-III via Makhoul: V_q = e^{+iπq/2n} (X_q − i X_{n−q}) / 2, X_n = 0.
        // DST-III: the same on Y_q = X_{n−1−q}.
        const bool rev = (bc == BC_DD);
#define XQ(q) ((q) >= n ? (T)0 : X[rev ? (n - 1 - (q)) : (q)])
        {
          const int q = k;
          cplx<T> w = tw[2 * q];
          w.y = -w.y;
          cplx<T> s = {XQ(q), -XQ(n - q)};
          Vk = cscale(cmul(w, s), (T)0.5);
        }
        {
          const int q = m - k;
          cplx<T> w = tw[2 * q];
          w.y = -w.y;
          cplx<T> s = {XQ(q), -XQ(n - q)};
          Vmk = cscale(cmul(w, s), (T)0.5);
        }
#undef XQ
      }
      // E_k = (V_k + conj V_{m−k})/2, O_k = (V_k − conj V_{m−k}) e^{+2πik/n}/2
      cplx<T> E = cscale(cadd(Vk, conj_(Vmk)), (T)0.5);
      cplx<T> wn = tw[8 * k];
      wn.y = -wn.y;
      cplx<T> O = cscale(cmul(csub(Vk, conj_(Vmk)), wn), (T)0.5);
      Z[k] = cadd(E, mul_i(O));
      if (k != 0 && 2 * k != m) Z[m - k] = cadd(conj_(E), mul_i(conj_(O)));
    }
  }
  __syncthreads();

  // ---- 3. complex FFT of length m (forward e^{−2πi/m}; backward e^{+2πi/m}, except
  //         DCT-IV, which is its own inverse and uses the forward FFT both ways) ----------
  cplx<T>* src = bufA;
  cplx<T>* dst = bufB;
  {
    const bool inv = !FWD && !bc_iv(bc) && bc != BC_FD;
    const int twm = (8 * n) / m;
    int Ns = 1;
    for (int s = 0; s < a.nstages; ++s) {
      const int R = a.radix[s];
      if (inv) {
        if (R == 4) stage<T, 4, true>(src, dst, L, m, ld, Ns, tw, twm);
        else if (R == 2) stage<T, 2, true>(src, dst, L, m, ld, Ns, tw, twm);
        else stage<T, 3, true>(src, dst, L, m, ld, Ns, tw, twm);
      } else {
        if (R == 4) stage<T, 4, false>(src, dst, L, m, ld, Ns, tw, twm);
        else if (R == 2) stage<T, 2, false>(src, dst, L, m, ld, Ns, tw, twm);
        else stage<T, 3, false>(src, dst, L, m, ld, Ns, tw, twm);
      }
      __syncthreads();
      cplx<T>* t = src;
      src = dst;
      dst = t;
      Ns *= R;
    }
  }
  // result in src; dst is free for the real output
  T* rO = reinterpret_cast<T*>(dst);

  // ---- 4. post-processing: m complex points -> n reals --------------------------
  if (bc == BC_FD) {  // X_k = −Im(Y_k), k = 1 … n−1 (× 1/2n backward); the wall entry copied
    const T sc = FWD ? (T)1 : (T)1 / (T)(2 * n);
    for (int idx = threadIdx.x; idx < L * n; idx += blockDim.x) {
      const int l = idx / n, k = idx - l * n;
      const cplx<T>* Z = src + l * ld;
      T* o = rO + l * ldr;
      if (k == 0) {  // the wall entry (saved beside the FFT data by the pre-processing)
        o[0] = bufA[l * ld + m].x;
        continue;
      }
      const cplx<T> Zk = Z[k], Zmk = Z[m - k];
      const cplx<T> E = cscale(cadd(Zk, conj_(Zmk)), (T)0.5);
      const cplx<T> O = cscale(mul_mi(csub(Zk, conj_(Zmk))), (T)0.5);
      const cplx<T> Y = cadd(E, cmul(tw[4 * k], O));
      o[k] = -Y.y * sc;
    }
  } else if (FWD) {
    const int np = bc_iv(bc) ? m : (m / 2 + 1);
    for (int idx = threadIdx.x; idx < L * np; idx += blockDim.x) {
      const int l = idx / np, k = idx - l * np;
      const cplx<T>* Z = src + l * ld;
      T* o = rO + l * ldr;
      if (bc_iv(bc)) {
        cplx<T> c = cmul(tw[4 * k + 1], Z[k]);
        o[2 * k] = (T)2 * c.x;
        o[n - 1 - 2 * k] = (T)-2 * c.y;
        continue;
      }
      // real DFT of the packed sequence: V_k = A + B, V_{m−k} = conj(A − B)
      cplx<T> Zk = Z[k], Zmk = Z[k == 0 ? 0 : m - k];
      cplx<T> E = cscale(cadd(Zk, conj_(Zmk)), (T)0.5);
      cplx<T> O = cscale(mul_mi(csub(Zk, conj_(Zmk))), (T)0.5);
      cplx<T> B = cmul(tw[8 * k], O);
      cplx<T> Vk = cadd(E, B);
      cplx<T> Vmk = conj_(csub(E, B));  // for k = 0 this is V_m
      if (bc == BC_P) {
        if (k == 0) {
          o[0] = Vk.x;
          o[n - 1] = Vmk.x;
        } else {
          o[2 * k - 1] = Vk.x;
          o[2 * k] = -Vk.y;
          if (2 * k != m) {
            o[2 * (m - k) - 1] = Vmk.x;
            o[2 * (m - k)] = -Vmk.y;
          }
        }
      } else {
        const bool rev = (bc == BC_DD);
#define OUT(q, val) o[rev ? (n - 1 - (q)) : (q)] = (val)
        if (k == 0) {
          OUT(0, (T)2 * Vk.x);
          OUT(m, (T)1.41421356237309504880 * Vmk.x);
        } else {
          cplx<T> c = cmul(tw[2 * k], Vk);
          OUT(k, (T)2 * c.x);
          OUT(n - k, (T)-2 * c.y);
          if (2 * k != m) {
            cplx<T> c2 = cmul(tw[2 * (m - k)], Vmk);
            OUT(m - k, (T)2 * c2.x);
            OUT(m + k, (T)-2 * c2.y);
          }
        }
#undef OUT
      }
    }
  } else {
    const T inv_m = (T)1 / (T)m;
    for (int idx = threadIdx.x; idx < L * m; idx += blockDim.x) {
      const int l = idx / m, k = idx - l * m;
      const cplx<T>* Z = src + l * ld;
      T* o = rO + l * ldr;
      if (bc_iv(bc)) {
        const T s = (T)1 / (T)n;  // 2·(1/2n)
        cplx<T> c = cmul(tw[4 * k + 1], Z[k]);
        const T A = s * c.x, B = -s * c.y;  // DN: the two outputs trade places
        o[2 * k] = (bc == BC_DN) ? B : A;
        o[n - 1 - 2 * k] = (bc == BC_DN) ? A : B;
      } else if (bc == BC_P) {
        o[2 * k] = Z[k].x * inv_m;
        o[2 * k + 1] = Z[k].y * inv_m;
      } else {
        const int i0 = mk_idx(2 * k, n, m), i1 = mk_idx(2 * k + 1, n, m);
        T v0 = Z[k].x * inv_m, v1 = Z[k].y * inv_m;
        if (bc == BC_DD) {
          if (i0 & 1) v0 = -v0;
          if (i1 & 1) v1 = -v1;
        }
        o[i0] = v0;
        o[i1] = v1;
      }
    }
  }
  __syncthreads();

  // ---- 5. store ----------------------------------------------------------------------
  T tmax = (T)0;  // max |new value| before widening (a 64-bit integer max would use the FP64 pipe)
  for (int idx = threadIdx.x; idx < L * n; idx += blockDim.x) {
    int l, e, z;
    size_t g;
    if (a.axis == 0) {
      l = idx / n;
      e = idx - l * n;
      if (l >= nlines_here) continue;
      size_t ln = (size_t)grp * L + l;
      g = ln * n + e;
      z = (int)(ln / ny);
    } else {
      e = idx / L;
      l = idx - e * L;
      g = ybase + (size_t)e * nx + l;
      z = zb;
    }
    T v = rO[l * ldr + e];
    if (!FWD && a.plane_scale) v *= a.plane_scale[z];
    const TO x = st_cvt<TO, T>::f(v);
    if constexpr (sizeof(TO) == 8) {
      if (out) {
        if constexpr (sizeof(T) == 4) {
          if (a.base32) out[g] = widen_f32(a.base32[g]) + x;
          else out[g] = a.accumulate ? out[g] + x : x;
        } else {
          out[g] = a.accumulate ? out[g] + x : x;
        }
      }
      tmax = fmax(tmax, fabs(v));
      if constexpr (sizeof(T) == 4)
        if (a.out2) a.out2[g] = v;
    } else {
      out[g] = a.accumulate ? out[g] + x : x;
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

}  // namespace ps
