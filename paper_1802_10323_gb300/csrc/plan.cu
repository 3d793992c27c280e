// plan.cu — plans, tables and the C-ABI entry points of ps_poisson.h.
//
// Tables are computed on the host in FP64 (Table 1 eigenvalues through the
// sin² form, Table 2 twiddles, the z coefficients of Eq. 4 on the faces) and
// cast once for the FP32 kernels. Solves only enqueue kernels on the caller's
// stream.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include <type_traits>

#include "internal.h"
#include "xform_fast.cuh"

using namespace ps;

namespace {

thread_local char g_create_err[256] = "";

// cos and sin of 2π t / N for N divisible by 8, reduced to [0, π/4] so that
// multiples of N/8 come out exact.
void cis(long t, long N, double* c, double* s) {
  t %= N;
  if (t < 0) t += N;
  const long q = t / (N / 4), r = t % (N / 4);
  const bool flip = 2 * r > N / 4;
  const long rr = flip ? (N / 4 - r) : r;
  const double ang = 2.0 * M_PI * (double)rr / (double)N;
  double c0 = cos(ang), s0 = sin(ang);
  if (flip) {
    double tmp = c0;
    c0 = s0;
    s0 = tmp;
  }
  // rotate by q quarter turns
  double cc = c0, ss = s0;
  for (long i = 0; i < q; ++i) {
    double t2 = cc;
    cc = -ss;
    ss = t2;
  }
  *c = cc;
  *s = ss;
}

struct AxisTab {
  int n = 0, m = 0, bc = 0, nstages = 0;
  int radix[kMaxStages] = {0};
  cplx<double>* tw64 = nullptr;
  cplx<float>* tw32 = nullptr;
  double* lam64 = nullptr;
  float* lam32 = nullptr;
};

bool size_ok(int n) {
  if (n < 2 || n > kMaxN || (n & 1)) return false;
  int m = n / 2;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

int make_radix(int m, int* radix) {
  int ns = 0;
  while (m % 4 == 0) { radix[ns++] = 4; m /= 4; }
  while (m % 2 == 0) { radix[ns++] = 2; m /= 2; }
  while (m % 3 == 0) { radix[ns++] = 3; m /= 3; }
  return ns;
}

// θ_q of Table 1 as a multiple of π/(4n): θ_q = π·j/(4n).
long theta_j(int bc, int n, int q) {
  switch (bc) {
    case BC_P: return 4L * ((q + 1) / 2);  // ⌈q/2⌉·π/n; Nyquist q = n−1 gives π/2
    case BC_NN: return 2L * q;
    case BC_DD: return 2L * (q + 1);
    case BC_FD: return 2L * q;             // x/y face unknowns: kπ/2n (q = 0: the wall row)
    default: return 2L * q + 1;            // ND, and DN (the reversed ND axis)
  }
}

std::vector<double> eig_scaled(int bc, int n, double h) {
  std::vector<double> lam(n);
  for (int q = 0; q < n; ++q) {
    double c, s;
    cis(theta_j(bc, n, q), 8L * n, &c, &s);  // sin(π j / 4n) = sin(2π j / 8n)
    lam[q] = -4.0 * s * s / (h * h);
  }
  if (bc == BC_FD) lam[0] = -1.0 / (h * h);  // the wall face's own row −u_0/Δ²
  return lam;
}

void split_df(double d, float2* out) {
  float h = (float)d;
  float l = (float)(d - (double)h);
  out->x = h;
  out->y = l;
}

}  // namespace

// Kernel kinds for the optional timing; each kind moves a fixed number of bytes
// per grid point (the FP32 refinement path has separate kinds for its FP64-input
// x pass, its storing and accumulating x passes and its check-only residual).
enum Kind { K_XF = 0, K_XF64IN, K_YF, K_Z, K_ZS, K_YB, K_XB, K_XB64ST, K_XB64ACC, K_RES, K_CHK,
            K_CTL, K_VER, K_RES0, K_RES3, K_XB64BASE, K_MAT, K_RESOUT, K_NSPRED, K_NSPROJ, K_NSPRES,
            K_TRANSP, K_NKINDS };
static const char* kKindName[K_NKINDS] = {"x_fwd", "x_fwd_f64in", "y_fwd", "z_solve",
                                          "z_singular", "y_bwd", "x_bwd", "x_bwd_f64store",
                                          "x_bwd_f64acc", "residual", "residual_check", "control",
                                          "residual_exact", "residual_first", "residual_first3",
                                          "x_bwd_f64base", "materialize", "residual_out",
                                          "ns_predict", "ns_projection", "ns_pressure", "transpose"};
constexpr int kProfMax = 4096;

struct Prof {
  int on = 0;
  int n = 0;
  std::vector<cudaEvent_t> ev;  // 2 per recorded launch
  std::vector<int> kind;
};

// ps_solve_host with refinement: the copy of f overlaps the first solve's x and y
// passes (per chunk of planes), the copy of p the passes after the first correction.
constexpr int kPipeMax = 8;
struct HostPipe {
  int nch = 0;
  int z[kPipeMax + 1] = {};
  cudaEvent_t in[kPipeMax] = {};   // chunk c of f is on the device
  cudaEvent_t out[kPipeMax] = {};  // chunk c of p = Φ_0 + e written by the first correction
  bool chunk_out = true;           // the first correction writes p chunk by chunk (records out)
  bool p_recorded = false;
};
// ps_solve_host_seq: per device slot, the chunk events of f, the solve's end (f and
// the slot's p free for the next copy in) and the end of the copy of p out
constexpr int kSeqComp = kPipeMax, kSeqOut = kPipeMax + 1, kSeqEv = kPipeMax + 2;

struct ps_plan {
  Prof prof;
  cudaStream_t copy_stream = nullptr;          // ps_solve_host: host <-> device copies
  cudaEvent_t pipe_ev[2 * kPipeMax + 1] = {};  // chunks of f in, chunks of p ready, call start
  cudaStream_t out_stream = nullptr;           // ps_solve_host_seq: device -> host copies
  cudaEvent_t seq_ev[2][kSeqEv] = {};
  ps_info* info_pinned = nullptr;              // ps_solve_host_seq: each problem's ps_info
  int info_cap = 0;
  int nx, ny, nz;
  double dx, dy;
  int bcx, bcy, bcz;
  ps_precision prec;
  double rtol;
  int max_iter;
  int singular, periodic_z;
  size_t N;
  AxisTab ax, ay;
  // z tables
  double *za64, *zb64, *zc64, *dzf64, *idzf64, *idzc64;
  float *za32, *zb32, *zc32, *dzf32, *idzf32, *idzc32;
  float2 *zlo, *zhi;
  float2* zres;  // residual passes m ≥ 1: (a_k, c_k, w_c) per plane, Dirichlet ghost sign folded in
  double asum;   // max over rows of Σ_j |w_j| (those passes' accumulator binade)
  double wsum;  // Σ Δz^f (the per-plane weights of the singular mean, times nx·ny)
  double anorm; // an upper bound of ‖A‖∞ (the drift bound of the incremental residual)
  double alpha = 0.0;  // Helmholtz shift: the plan solves (A − α·I)·p = f
  df nalpha = {0.f, 0.f};  // −α in double-float (residual pass 0)
  int lowx, lowy;  // FP32 non-periodic z: rectangle of columns solved in FP64 (tridiag.cu)
  df idx2, idy2;
  void* dev;    // one allocation for all of the above
  int resid_blocks;     // CTAs of a residual pass (max over the two shapes: partials size)
  int resid_blocks3;    // … of a three-level pass (incremental pass 0, exact pass)
  int resid_blocks2;    // … of pass 0 (two-level)
  int resid_blocksA;    // … of the passes m ≥ 1
  char err[256];
};

namespace {

std::atomic<int> g_inject_alloc{0};

ps_status fail(ps_plan* p, ps_status st, const char* msg) {
  if (p) snprintf(p->err, sizeof(p->err), "%s", msg);
  else snprintf(g_create_err, sizeof(g_create_err), "%s", msg);
  return st;
}

ps_status cuda_fail(ps_plan* p, cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s [%s]", where, cudaGetErrorString(e), g_launch_diag);
  return fail(p, e == cudaErrorMemoryAllocation ? PS_OUT_OF_MEMORY : PS_CUDA_ERROR, buf);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WsLayout {
  size_t ctrl, partial, info, w, rh, rl, u0, scr_c, scr_u, zlow, total;
};

WsLayout ws_layout(const ps_plan* p) {
  WsLayout L{};
  size_t off = 0;
  L.ctrl = off;
  off += align256(sizeof(Ctrl));
  L.partial = off;
  off += align256((size_t)p->resid_blocks * 4 * sizeof(float));
  L.info = off;
  off += align256(sizeof(ps_info));
  const size_t tz = (p->prec == PS_FP64) ? sizeof(double) : sizeof(float);
  L.w = off;
  L.rh = off;
  L.rl = off;
  if (p->prec == PS_FP32_REFINE) {
    off += align256(p->N * sizeof(float));
    L.rh = off;  // the residual r = rh + rl of the refinement (double-float)
    off += align256(p->N * sizeof(float));
    L.rl = off;
    off += align256(p->N * sizeof(float));
    L.u0 = off;  // Φ_0, the FP32 solve (operand of residual pass 0, base of the first correction)
    off += align256(p->N * sizeof(float));
  }
  L.scr_c = off;
  off += align256(p->N * tz);
  L.scr_u = off;
  if (p->periodic_z) off += align256(p->N * tz);
  L.zlow = off;
  off += align256((size_t)2 * p->nz * p->lowx * p->lowy * sizeof(double));
  L.total = off;
  return L;
}

template <class T>
XformArgs<T> xargs(const ps_plan* p, int axis, const void* in, void* out, const T* scale,
                   int accumulate, const int* skip) {
  XformArgs<T> a{};
  const AxisTab& t = axis == 0 ? p->ax : p->ay;
  a.in = in;
  a.out = out;
  a.n = t.n;
  a.m = t.m;
  a.axis = axis;
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.nlines = (axis == 0) ? p->ny * p->nz : p->nx * p->nz;
  a.bc = t.bc;
  a.nstages = t.nstages;
  for (int i = 0; i < kMaxStages; ++i) a.radix[i] = t.radix[i];
  if constexpr (sizeof(T) == 8) a.tw = reinterpret_cast<const cplx<T>*>(t.tw64);
  else a.tw = reinterpret_cast<const cplx<T>*>(t.tw32);
  a.plane_scale = scale;
  a.accumulate = accumulate;
  a.skip = skip;
  return a;
}

template <class T>
ZArgs<T> zargs(const ps_plan* p, T* data, void* ws, const WsLayout& L, const int* skip) {
  ZArgs<T> a{};
  char* w = static_cast<char*>(ws);
  a.data = data;
  a.scr_c = reinterpret_cast<T*>(w + L.scr_c);
  a.scr_u = p->periodic_z ? reinterpret_cast<T*>(w + L.scr_u) : nullptr;
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  if constexpr (sizeof(T) == 8) {
    a.lamx = p->ax.lam64; a.lamy = p->ay.lam64;
    a.za = p->za64; a.zb = p->zb64; a.zc = p->zc64; a.dzf = p->dzf64;
  } else {
    a.lamx = p->ax.lam32; a.lamy = p->ay.lam32;
    a.za = p->za32; a.zb = p->zb32; a.zc = p->zc32; a.dzf = p->dzf32;
  }
  a.periodic = p->periodic_z;
  a.singular = p->singular;
  a.skip = skip;
  if constexpr (sizeof(T) == 4) {
    a.lowx = p->lowx;
    a.lowy = p->lowy;
    a.lamx64 = p->ax.lam64;
    a.lamy64 = p->ay.lam64;
    a.za64 = p->za64;
    a.zb64 = p->zb64;
    a.zc64 = p->zc64;
    a.dzf64 = p->dzf64;
    a.scr64 = reinterpret_cast<double*>(w + L.zlow);
  }
  return a;
}

// The same z systems on planes stored transposed ([n_x][n_y], y fastest), as the
// long y lines leave them: the column index runs over q_y first, so the x and y
// roles (lengths, eigenvalues, the FP64 low-wavenumber rectangle) swap. The
// elimination scratch is `scratch` (an idle array of n_x·n_y·n_z values of T)
// instead of the workspace array that now holds the data.
template <class T>
ZArgs<T> zargs_t(const ps_plan* p, T* data, void* ws, const WsLayout& L, const int* skip, T* scratch) {
  ZArgs<T> a = zargs<T>(p, data, ws, L, skip);
  std::swap(a.nx, a.ny);
  std::swap(a.lamx, a.lamy);
  a.scr_c = scratch;
  if constexpr (sizeof(T) == 4) {
    std::swap(a.lowx, a.lowy);
    std::swap(a.lamx64, a.lamy64);
  }
  return a;
}

template <class T, class TI, class TO, bool FWD>
cudaError_t launch_long(int m, FastArgs<T> a, cudaStream_t st) {
  switch (m) {
    case 1024: return launch_xform_long<T, TI, TO, 1024, FWD>(a, st);
    case 2048: return launch_xform_long<T, TI, TO, 2048, FWD>(a, st);
    default: return launch_xform_long<T, TI, TO, 4096, FWD>(a, st);
  }
}

// One pass of line transforms along x (axis 0) or y (axis 1): the register-resident
// kernels for n ∈ {128, 256, 512, 1024} when the tile fits; for n ∈ {2048, 4096,
// 8192} the one-line-per-CTA kernel (y lines: transposed into yscr, an idle
// workspace array of n_x·n_y·n_z values of T, and back); else the generic one.
template <class T, class TI, class TO, bool FWD>
cudaError_t line_xform(const ps_plan* p, int axis, const void* in, void* out, const T* scale,
                       int accumulate, const int* skip, cudaStream_t st,
                       unsigned long long* amax = nullptr, float* out2 = nullptr,
                       const float* base32 = nullptr, int zn = 0, void* yscr = nullptr) {
  const AxisTab& t = axis == 0 ? p->ax : p->ay;
  const bool long_m = (t.m == 1024 || t.m == 2048 || t.m == 4096) && zn == 0 && t.bc != BC_FD;
  if (long_m && (axis == 0 || (yscr && std::is_same<TI, T>::value && std::is_same<TO, T>::value &&
                               !accumulate && !amax && !out2 && !base32))) {
    FastArgs<T> a{};
    a.axis = 0;
    a.bc = t.bc;
    if constexpr (sizeof(T) == 8) a.tw = reinterpret_cast<const cplx<T>*>(t.tw64);
    else a.tw = reinterpret_cast<const cplx<T>*>(t.tw32);
    a.plane_scale = scale;
    a.accumulate = accumulate;
    a.skip = skip;
    a.amax = amax;
    a.out2 = out2;
    a.base32 = base32;
    a.nx = t.n;
    a.nz = p->nz;
    if (axis == 0) {
      a.in = in;
      a.out = out;
      a.ny = p->ny;  // lines per plane
      a.nlines = p->ny * p->nz;
      return launch_long<T, TI, TO, FWD>(t.m, a, st);
    }
    // y: every plane [n_y][n_x] → [n_x][n_y] in yscr, the lines there, and back
    T* sc = static_cast<T*>(yscr);
    cudaError_t e = launch_plane_transpose<T>(static_cast<const T*>(in), sc, p->ny, p->nx, p->nz, skip, st);
    if (e != cudaSuccess) return e;
    a.in = sc;
    a.out = sc;
    a.ny = p->nx;  // lines per plane
    a.nlines = p->nx * p->nz;
    if ((e = launch_long<T, T, T, FWD>(t.m, a, st)) != cudaSuccess) return e;
    return launch_plane_transpose<T>(sc, static_cast<T*>(out), p->nx, p->ny, p->nz, skip, st);
  }
  const int lpc_y = (sizeof(T) == 4 && sizeof(TI) == 4 && sizeof(TO) == 4) ? 16 : 8;
  const bool fast_ok = (t.m == 64 || t.m == 128 || t.m == 256 || t.m == 512) && t.bc != BC_FD &&
                       (axis == 0 || p->nx % lpc_y == 0);
  if (fast_ok) {
    FastArgs<T> a{};
    a.in = in;
    a.out = out;
    a.axis = axis;
    a.nx = p->nx;
    a.ny = p->ny;
    a.nz = p->nz;
    a.bc = t.bc;
    a.nlines = (axis == 0) ? p->ny * p->nz : p->nx * p->nz;
    if (zn > 0) {  // the planes at in/out only (the caller offsets the pointers)
      a.nz = zn;
      a.nlines = (axis == 0) ? p->ny * zn : p->nx * zn;
    }
    if constexpr (sizeof(T) == 8) a.tw = reinterpret_cast<const cplx<T>*>(t.tw64);
    else a.tw = reinterpret_cast<const cplx<T>*>(t.tw32);
    a.plane_scale = scale;
    a.accumulate = accumulate;
    a.skip = skip;
    a.amax = amax;
    a.out2 = out2;
    a.base32 = base32;
    if (axis == 1 && std::is_same<TI, T>::value && std::is_same<TO, T>::value && p->nx % 16 == 0 &&
        !accumulate && !amax && !out2 && !base32) {
      switch (t.m) {
        case 64: return launch_xform_col<T, 64, FWD>(a, st);
        case 128: return launch_xform_col<T, 128, FWD>(a, st);
        case 256: return launch_xform_col<T, 256, FWD>(a, st);
        default: return launch_xform_col<T, 512, FWD>(a, st);
      }
    }
    if (axis == 0) {
      switch (t.m) {
        case 64: return launch_xform_row<T, TI, TO, 64, FWD>(a, st);
        case 128: return launch_xform_row<T, TI, TO, 128, FWD>(a, st);
        case 256: return launch_xform_row<T, TI, TO, 256, FWD>(a, st);
        default: return launch_xform_row<T, TI, TO, 512, FWD>(a, st);
      }
    }
    switch (t.m) {
      case 64: return launch_xform_fast<T, TI, TO, 64, FWD>(a, st);
      case 128: return launch_xform_fast<T, TI, TO, 128, FWD>(a, st);
      case 256: return launch_xform_fast<T, TI, TO, 256, FWD>(a, st);
      default: return launch_xform_fast<T, TI, TO, 512, FWD>(a, st);
    }
  }
  XformArgs<T> ga = xargs<T>(p, axis, in, out, scale, accumulate, skip);
  ga.amax = amax;
  ga.out2 = out2;
  ga.base32 = base32;
  return launch_xform<T, TI, TO, FWD>(ga, st);
}

// y lines of n_y ∈ {2048, 4096, 8192} (not face-centred): the one-line-per-CTA
// kernel on planes transposed into the scratch array.
bool y_long(const ps_plan* p) {
  const AxisTab& t = p->ay;
  return (t.m == 1024 || t.m == 2048 || t.m == 4096) && t.bc != BC_FD;
}



// Launch `fn` on `st`, bracketed by profiling events when enabled on the plan.
template <class F>
cudaError_t run(ps_plan* pl, int kind, cudaStream_t st, F&& fn) {
  Prof& pr = pl->prof;
  const bool rec = pr.on && pr.n < kProfMax;
  if (rec) cudaEventRecord(pr.ev[2 * pr.n], st);
  cudaError_t e = fn();
  if (rec) {
    cudaEventRecord(pr.ev[2 * pr.n + 1], st);
    pr.kind[pr.n] = kind;
    ++pr.n;
  }
  return e;
}

// One y pass. Long y lines (y_long): the one-line-per-CTA kernel on planes left
// transposed — forward, data [n_z][n_y][n_x] → yt [n_z][n_x][n_y] and transformed;
// backward, yt transformed in place and transposed back into data — so that the z
// solve between them runs on yt (zargs_t) and each solve pays two plane transposes,
// not four; the transposes are timed as their own kind. Otherwise `other`.
template <class T, bool FWD, class F>
cudaError_t y_pass(ps_plan* pl, Kind kind, bool yl, T* data, T* yt, const int* skip, cudaStream_t st, F&& other) {
  if (!yl) return run(pl, kind, st, other);
  const AxisTab& t = pl->ay;
  FastArgs<T> a{};
  a.axis = 0;
  a.bc = t.bc;
  if constexpr (sizeof(T) == 8) a.tw = reinterpret_cast<const cplx<T>*>(t.tw64);
  else a.tw = reinterpret_cast<const cplx<T>*>(t.tw32);
  a.skip = skip;
  a.nx = t.n;
  a.nz = pl->nz;
  a.in = yt;
  a.out = yt;
  a.ny = pl->nx;  // lines per plane
  a.nlines = pl->nx * pl->nz;
  cudaError_t e;
  if (FWD && (e = run(pl, K_TRANSP, st, [&] {
                return launch_plane_transpose<T>(data, yt, pl->ny, pl->nx, pl->nz, skip, st);
              })) != cudaSuccess)
    return e;
  if ((e = run(pl, kind, st, [&] { return launch_long<T, T, T, FWD>(t.m, a, st); })) != cudaSuccess) return e;
  if (!FWD)
    return run(pl, K_TRANSP, st, [&] { return launch_plane_transpose<T>(yt, data, pl->nx, pl->ny, pl->nz, skip, st); });
  return cudaSuccess;
}

// The plain five-pass solve in one precision, in place on `p` after the first pass.
template <class T>
ps_status solve_plain(ps_plan* pl, const T* f, T* p, void* ws, cudaStream_t st, ps_info* info,
                      bool transpose) {
  const WsLayout L = ws_layout(pl);
  const T* sin_ = nullptr;
  const T* sout = nullptr;
  if (transpose) {
    if constexpr (sizeof(T) == 8) { sin_ = pl->idzf64; sout = pl->dzf64; }
    else { sin_ = pl->idzf32; sout = pl->dzf32; }
  }
  cudaError_t e;
  if ((e = run(pl, K_XF, st, [&] { return line_xform<T, T, T, true>(pl, 0, f, p, sin_, 0, nullptr, st); })) != cudaSuccess)
    return cuda_fail(pl, e, "x forward");
  void* yscr = static_cast<char*>(ws) + L.scr_c;  // idle outside the z solve
  // long y lines: the z solve runs on the transposed planes in yscr, p is its scratch
  const bool yl = y_long(pl);
  T* yt = static_cast<T*>(yscr);
  if ((e = y_pass<T, true>(pl, K_YF, yl, p, yt, nullptr, st, [&] {
         return line_xform<T, T, T, true>(pl, 1, p, p, nullptr, 0, nullptr, st);
       })) != cudaSuccess)
    return cuda_fail(pl, e, "y forward");
  const ZArgs<T> za = yl ? zargs_t<T>(pl, yt, ws, L, nullptr, p) : zargs<T>(pl, p, ws, L, nullptr);
  if ((e = run(pl, K_Z, st, [&] {
         if constexpr (sizeof(T) == 4)
           if (!pl->periodic_z) return launch_zsolve_ckpt(za, st);
         return launch_zsolve<T>(za, st);
       })) != cudaSuccess)
    return cuda_fail(pl, e, "z solve");
  if (pl->singular && !(sizeof(T) == 4 && !pl->periodic_z && pl->lowx > 0) &&
      (e = run(pl, K_ZS, st, [&] { return launch_zsingular<T>(za, st); })) != cudaSuccess)
    return cuda_fail(pl, e, "z singular column");
  if ((e = y_pass<T, false>(pl, K_YB, yl, p, yt, nullptr, st, [&] {
         return line_xform<T, T, T, false>(pl, 1, p, p, nullptr, 0, nullptr, st);
       })) != cudaSuccess)
    return cuda_fail(pl, e, "y backward");
  if ((e = run(pl, K_XB, st, [&] { return line_xform<T, T, T, false>(pl, 0, p, p, sout, 0, nullptr, st); })) != cudaSuccess)
    return cuda_fail(pl, e, "x backward");
  if (info && (e = run(pl, K_CTL, st, [&] { return launch_info_plain(info, st); })) != cudaSuccess)
    return cuda_fail(pl, e, "info");
  return PS_OK;
}

// FP32 bulk solve with FP64 iterative refinement (residual in double-float).
ps_status solve_refine(ps_plan* pl, const double* f, double* p, void* ws, cudaStream_t st,
                       ps_info* info, HostPipe* hp = nullptr) {
  const WsLayout L = ws_layout(pl);
  char* wb = static_cast<char*>(ws);
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(wb + L.ctrl);
  float* partial = reinterpret_cast<float*>(wb + L.partial);
  float* w = reinterpret_cast<float*>(wb + L.w);
  const int* skip = &ctrl->converged;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st)) != cudaSuccess) return cuda_fail(pl, e, "reset");
  float* rh = reinterpret_cast<float*>(wb + L.rh);
  float* rl = reinterpret_cast<float*>(wb + L.rl);
  float* u0 = reinterpret_cast<float*>(wb + L.u0);
  void* yscr = wb + L.scr_c;  // the transposed y lines of n ≥ 2048 (idle outside the z solve)
  const ZArgs<float> zw = zargs<float>(pl, w, ws, L, skip);
  // long y lines: between the y passes the planes stay transposed in yscr, and the
  // z solve runs there with w (idle then) as its scratch
  float* yt = static_cast<float*>(yscr);
  const ZArgs<float> zwt = zargs_t<float>(pl, yt, ws, L, skip, w);
  // One FP32 solve (c = 0: of f; c ≥ 1: of r = rh, the c-th correction) through w.
  // The x backward writes Φ_0 to u0 only (c = 0; the FP64 p is written by the first
  // correction as Φ_0 + e, or from Φ_0 alone if the loop ends at pass 0), then
  // p = Φ_0 + e (c = 1) or p += e (c ≥ 2), keeping e in w for the next residual
  // pass; max|Φ_0| or max|e| go to ctrl.
  auto correction = [&](int c) -> cudaError_t {
    const bool first = (c == 0);
    cudaError_t r;
    if (first && hp) {  // f arrives in chunks of planes: x and y of each chunk as it lands
      for (int ch = 0; ch < hp->nch; ++ch) {
        const int zn = hp->z[ch + 1] - hp->z[ch];
        const size_t off = (size_t)hp->z[ch] * pl->nx * pl->ny;
        if ((r = cudaStreamWaitEvent(st, hp->in[ch], 0)) != cudaSuccess) return r;
        if ((r = run(pl, K_XF64IN, st, [&] {
               return line_xform<float, double, float, true>(pl, 0, f + off, w + off, nullptr, 0, skip, st,
                                                             nullptr, nullptr, nullptr, zn);
             })) != cudaSuccess)
          return r;
        if ((r = run(pl, K_YF, st, [&] {
               return line_xform<float, float, float, true>(pl, 1, w + off, w + off, nullptr, 0, skip, st,
                                                            nullptr, nullptr, nullptr, zn);
             })) != cudaSuccess)
          return r;
      }
    } else {
      if (first)
        r = run(pl, K_XF64IN, st, [&] { return line_xform<float, double, float, true>(pl, 0, f, w, nullptr, 0, skip, st); });
      else
        r = run(pl, K_XF, st, [&] { return line_xform<float, float, float, true>(pl, 0, rh, w, nullptr, 0, skip, st); });
      if (r != cudaSuccess) return r;
      if ((r = y_pass<float, true>(pl, K_YF, y_long(pl), w, yt, skip, st, [&] {
             return line_xform<float, float, float, true>(pl, 1, w, w, nullptr, 0, skip, st);
           })) != cudaSuccess)
        return r;
    }
    // (chunked host input, whose y lines of n ≤ 1024 never take the long kernel, keeps
    // the planes untransposed)
    const bool ytr = y_long(pl) && !(first && hp);
    const ZArgs<float>& za = ytr ? zwt : zw;
    if ((r = run(pl, K_Z, st, [&] {
           return pl->periodic_z ? launch_zsolve<float>(za, st) : launch_zsolve_ckpt(za, st);
         })) != cudaSuccess)
      return r;
    if (pl->singular && (pl->periodic_z || pl->lowx == 0) &&
        (r = run(pl, K_ZS, st, [&] { return launch_zsingular<float>(za, st); })) != cudaSuccess) return r;
    if ((r = y_pass<float, false>(pl, K_YB, ytr, w, yt, skip, st, [&] {
           return line_xform<float, float, float, false>(pl, 1, w, w, nullptr, 0, skip, st, nullptr, nullptr,
                                                         nullptr, 0, yscr);
         })) != cudaSuccess)
      return r;
    if (first)
      return run(pl, K_XB64ST, st, [&] {
        return line_xform<float, float, double, false>(pl, 0, w, nullptr, nullptr, 0, skip, st, &ctrl->pmax, u0);
      });
    if (hp && hp->chunk_out && c == 1) {  // p is final here unless a later correction runs: chunk by chunk
      for (int ch = 0; ch < hp->nch; ++ch) {
        const int zn = hp->z[ch + 1] - hp->z[ch];
        const size_t off = (size_t)hp->z[ch] * pl->nx * pl->ny;
        if ((r = run(pl, K_XB64BASE, st, [&] {
               return line_xform<float, float, double, false>(pl, 0, w + off, p + off, nullptr, 0, skip, st,
                                                              &ctrl->dmax, w + off, u0 + off, zn);
             })) != cudaSuccess)
          return r;
        if ((r = cudaEventRecord(hp->out[ch], st)) != cudaSuccess) return r;
      }
      hp->p_recorded = true;
      return cudaSuccess;
    }
    return run(pl, c == 1 ? K_XB64BASE : K_XB64ACC, st, [&] {
      return line_xform<float, float, double, false>(pl, 0, w, p, nullptr, c == 1 ? 0 : 1, skip, st, &ctrl->dmax,
                                                     w, c == 1 ? u0 : nullptr);
    });
  };
  ResidArgs ra{};
  ra.p = p;
  ra.f = f;
  ra.rh_in = rh;
  ra.rl_in = rl;
  ra.nx = pl->nx;
  ra.ny = pl->ny;
  ra.nz = pl->nz;
  ra.bcx = pl->bcx;
  ra.bcy = pl->bcy;
  ra.bcz = pl->bcz;
  ra.idx2 = pl->idx2;
  ra.idy2 = pl->idy2;
  ra.zlo = pl->zlo;
  ra.zhi = pl->zhi;
  ra.zres = pl->zres;
  ra.asum = pl->asum;
  ra.nalpha = pl->nalpha;
  ra.wz = pl->dzf32;
  ra.mu = ctrl->mu;
  ra.singular = pl->singular;
  ra.red = ctrl->red;
  ra.partial = partial;
  ra.nblocks = pl->resid_blocks;  // (informational; each launch sizes its own grid)
  ra.skip = skip;
  const double wsum_total = pl->wsum * pl->nx * pl->ny;
  if ((e = correction(0)) != cudaSuccess) return cuda_fail(pl, e, "initial solve");
  // Passes m ≥ 1 first only check (no output: the loop usually ends there); if
  // their finalize finds no convergence, the pass is repeated to store r_m for the
  // next correction. Pass 0 stores r_0 at once (it almost never converges).
  for (int it = 0; it <= pl->max_iter; ++it) {
    const bool last = (it == pl->max_iter);
    ra.rh_out = (last || it > 0) ? nullptr : rh;
    ra.rl_out = (last || it > 0) ? nullptr : rl;
    ra.pmax_bits = it == 0 ? &ctrl->pmax : &ctrl->dmax;
    ra.u = it == 0 ? u0 : w;
    ra.skip = skip;
    if ((e = run(pl, (last || it > 0) ? K_CHK : K_RES0, st,
                 [&] { return launch_residual_inc(ra, it, 0, st); })) != cudaSuccess)
      return cuda_fail(pl, e, "residual");
    if ((e = run(pl, K_CTL, st, [&] {
           return launch_finalize(ctrl, partial, it == 0 ? pl->resid_blocks2 : pl->resid_blocksA, wsum_total,
                                  pl->singular, pl->rtol, it, 0, last ? 1 : 0, pl->anorm, nullptr, info, st);
         })) != cudaSuccess)
      return cuda_fail(pl, e, "finalize");
    if (it == 0) {
      // pass 0 again with the three-level split, only if its finalize asked for it
      ResidArgs r3 = ra;
      r3.skip = &ctrl->skip_redo;
      if ((e = run(pl, K_RES3, st, [&] { return launch_residual_inc(r3, 0, 1, st); })) != cudaSuccess)
        return cuda_fail(pl, e, "residual");
      if ((e = run(pl, K_CTL, st, [&] {
             return launch_finalize(ctrl, partial, pl->resid_blocks3, wsum_total, pl->singular,
                                    pl->rtol, 0, 1, last ? 1 : 0, pl->anorm, &ctrl->skip_redo, info, st);
           })) != cudaSuccess)
        return cuda_fail(pl, e, "finalize");
      // the loop ended at pass 0 (converged or max_iter = 0): p = Φ_0
      if ((e = run(pl, K_MAT, st, [&] { return launch_widen(u0, p, pl->N, &ctrl->nomat0, st); })) != cudaSuccess)
        return cuda_fail(pl, e, "store");
    }
    if (it > 0 && !last) {  // the output repeat of pass it, only if it did not converge
      ResidArgs ro = ra;
      ro.rh_out = rh;
      ro.rl_out = rl;
      ro.pmax_bits = &ctrl->dmax_prev;
      ro.skip = &ctrl->skip_out;
      if ((e = run(pl, K_RESOUT, st, [&] { return launch_residual_inc(ro, it, 0, st); })) != cudaSuccess)
        return cuda_fail(pl, e, "residual");
    }
    if (!last && (e = correction(it + 1)) != cudaSuccess) return cuda_fail(pl, e, "correction");
  }
  // Exact confirmation from the stored p, only when the drift bound of the
  // incremental passes was not small (both kernels return at once otherwise).
  ResidArgs rx = ra;
  rx.r = rh;
  rx.pmax_bits = &ctrl->pmax;
  rx.skip = &ctrl->vskip;
  if ((e = run(pl, K_VER, st, [&] { return launch_residual_exact(rx, st); })) != cudaSuccess)
    return cuda_fail(pl, e, "exact residual");
  if ((e = run(pl, K_CTL, st, [&] {
         return launch_finalize_exact(ctrl, partial, pl->resid_blocks3, wsum_total, pl->singular,
                                      pl->rtol, info, st);
       })) != cudaSuccess)
    return cuda_fail(pl, e, "finalize");
  return PS_OK;
}

ps_status check_solve_args(ps_plan* p, const void* f, const void* out, const void* ws) {
  if (!p) return fail(nullptr, PS_INVALID_ARG, "null plan");
  if (!f || !out) return fail(p, PS_INVALID_ARG, "null field pointer");
  if (!ws) return fail(p, PS_INVALID_ARG, "null workspace");
  if (((uintptr_t)ws) & 255) return fail(p, PS_INVALID_ARG, "workspace must be 256-byte aligned");
  // the transform kernels move lines with 16-byte vector accesses
  if ((((uintptr_t)f) | ((uintptr_t)out)) & 15) return fail(p, PS_INVALID_ARG, "f and p must be 16-byte aligned");
  return PS_OK;
}

}  // namespace

namespace ps {
void set_plan_error(ps_plan* plan, const char* msg) { fail(plan, PS_OK, msg); }

bool take_injected_alloc_failure() {
  int c = g_inject_alloc.load();
  while (c > 0)
    if (g_inject_alloc.compare_exchange_weak(c, c - 1)) return true;
  return false;
}

double ps_plan_internal_alpha(const ps_plan* p) { return p->alpha; }

void ps_plan_internal_tables(const ps_plan* p, const cplx<float>** twx, const cplx<float>** twy,
                             const float** lamx, const float** lamy, const float** za, const float** zb,
                             const float** zc, const float** dzf, const float2** zlo, const float2** zhi,
                             df* idx2, df* idy2, double* wsum_total, int* radx, int* rady, int* nstx,
                             int* nsty) {
  *twx = p->ax.tw32;
  *twy = p->ay.tw32;
  *lamx = p->ax.lam32;
  *lamy = p->ay.lam32;
  *za = p->za32;
  *zb = p->zb32;
  *zc = p->zc32;
  *dzf = p->dzf32;
  *zlo = p->zlo;
  *zhi = p->zhi;
  *idx2 = p->idx2;
  *idy2 = p->idy2;
  *wsum_total = p->wsum * p->nx * p->ny;
  for (int i = 0; i < kMaxStages; ++i) {
    radx[i] = p->ax.radix[i];
    rady[i] = p->ay.radix[i];
  }
  *nstx = p->ax.nstages;
  *nsty = p->ay.nstages;
}
}  // namespace ps

extern "C" {

ps_status ps_plan_create(ps_plan** out, int nx, int ny, int nz, double dx, double dy,
                         const double* zf, double dz, ps_bc bcx, ps_bc bcy, ps_bc bcz,
                         ps_precision prec, double rtol, int max_iter) {
  return ps_plan_create_helmholtz(out, nx, ny, nz, dx, dy, zf, dz, bcx, bcy, bcz, prec, rtol, max_iter, 0.0);
}

ps_status ps_plan_create_helmholtz(ps_plan** out, int nx, int ny, int nz, double dx, double dy,
                                   const double* zf, double dz, ps_bc bcx, ps_bc bcy, ps_bc bcz,
                                   ps_precision prec, double rtol, int max_iter, double alpha) {
  if (!out) return fail(nullptr, PS_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (!(alpha >= 0.0) || !std::isfinite(alpha))
    return fail(nullptr, PS_INVALID_ARG, "the Helmholtz shift alpha must be finite and >= 0");
  if ((unsigned)bcx > 5u || (unsigned)bcy > 5u || (unsigned)bcz > 5u)
    return fail(nullptr, PS_INVALID_ARG, "unknown boundary condition");
  if ((unsigned)prec > 2u) return fail(nullptr, PS_INVALID_ARG, "unknown precision");
  if (!(dx > 0) || !(dy > 0)) return fail(nullptr, PS_INVALID_ARG, "dx and dy must be > 0");
  if (!zf && !(dz > 0)) return fail(nullptr, PS_INVALID_ARG, "dz must be > 0 when zf is NULL");
  if (!size_ok(nx) || !size_ok(ny))
    return fail(nullptr, PS_UNSUPPORTED_SIZE, "nx, ny must be even, 2..8192, with n/2 = 2^a 3^b");
  if ((bcx == PS_BC_FACE_DIRICHLET && nx > 4096) || (bcy == PS_BC_FACE_DIRICHLET && ny > 4096))
    return fail(nullptr, PS_UNSUPPORTED_SIZE, "face-centred x or y lines must have n <= 4096");
  if (nz < 2 || nz > 8192) return fail(nullptr, PS_UNSUPPORTED_SIZE, "nz must be in 2..8192");
  if (prec == PS_FP32_REFINE && (max_iter < 0 || !(rtol > 0)))
    return fail(nullptr, PS_INVALID_ARG, "refinement needs rtol > 0 and max_iter >= 0");
  std::vector<double> faces(nz + 1);
  for (int k = 0; k <= nz; ++k) faces[k] = zf ? zf[k] : k * dz;
  for (int k = 0; k < nz; ++k)
    if (!(faces[k + 1] > faces[k])) return fail(nullptr, PS_INVALID_ARG, "z faces must increase");

  ps_plan* p = new (std::nothrow) ps_plan();
  if (!p) return fail(nullptr, PS_OUT_OF_MEMORY, "host allocation failed");
  p->nx = nx; p->ny = ny; p->nz = nz; p->dx = dx; p->dy = dy;
  p->bcx = bcx; p->bcy = bcy; p->bcz = bcz;
  p->prec = prec; p->rtol = rtol; p->max_iter = max_iter;
  p->N = (size_t)nx * ny * nz;
  p->periodic_z = (bcz == PS_BC_PERIODIC);
  auto pn = [](int b) { return b == PS_BC_PERIODIC || b == PS_BC_NEUMANN_NEUMANN; };
  p->singular = pn(bcx) && pn(bcy) && pn(bcz) && alpha == 0.0;  // α > 0: no null space
  p->alpha = alpha;
  {
    float2 t;
    split_df(-alpha, &t);
    p->nalpha = df{t.x, t.y};
  }
  p->resid_blocks3 = residual_blocks(nx, ny, nz, 1);
  p->resid_blocks2 = residual_blocks(nx, ny, nz, 0);
  p->resid_blocksA = residual_blocks(nx, ny, nz, 2);
  p->resid_blocks = std::max(p->resid_blocks3, std::max(p->resid_blocks2, p->resid_blocksA));

  // ---- z metric (finite-volume form of Eq. 4 on the faces) ----
  std::vector<double> dzf(nz), dzc(nz > 1 ? nz - 1 : 0), za(nz, 0.0), zb(nz, 0.0), zc(nz, 0.0);
  std::vector<float2> zlo(nz), zhi(nz);
  for (int k = 0; k < nz; ++k) dzf[k] = faces[k + 1] - faces[k];
  for (int k = 0; k + 1 < nz; ++k) dzc[k] = 0.5 * (faces[k + 2] - faces[k]);
  std::vector<double> lo(nz, 0.0), hi(nz, 0.0);  // residual coefficients
  for (int k = 1; k < nz; ++k) za[k] = lo[k] = 1.0 / (dzf[k] * dzc[k - 1]);
  for (int k = 0; k + 1 < nz; ++k) zc[k] = hi[k] = 1.0 / (dzf[k] * dzc[k]);
  for (int k = 0; k < nz; ++k) zb[k] = -(za[k] + zc[k]);
  if (bcz == PS_BC_PERIODIC) {
    const double hp = 0.5 * (dzf[0] + dzf[nz - 1]);
    za[0] = lo[0] = 1.0 / (dzf[0] * hp);
    zc[nz - 1] = hi[nz - 1] = 1.0 / (dzf[nz - 1] * hp);
    zb[0] -= za[0];
    zb[nz - 1] -= zc[nz - 1];
  } else {
    if (bcz == PS_BC_DIRICHLET_DIRICHLET || bcz == PS_BC_DIRICHLET_NEUMANN) {
      zb[0] -= 2.0 / (dzf[0] * dzf[0]);
      lo[0] = 1.0 / (dzf[0] * dzf[0]);
    }
    if (bcz == PS_BC_DIRICHLET_DIRICHLET || bcz == PS_BC_NEUMANN_DIRICHLET) {
      zb[nz - 1] -= 2.0 / (dzf[nz - 1] * dzf[nz - 1]);
      hi[nz - 1] = 1.0 / (dzf[nz - 1] * dzf[nz - 1]);
    }
  }
  if (bcz == PS_BC_FACE_DIRICHLET) {
    // unknowns on the z faces: plane k is face k, face 0 the stored bottom wall and face
    // nz the implicit top wall (both 0). Row k ≥ 1 on the volume between the centres of
    // cells k−1 and k; row 0 is −p_0. For the residual stencils both ends take the
    // Dirichlet ghost rule (ghost = −p): lo_0 = 1/2 makes row 0 read −p_0, and hi_{nz−1}
    // = up/2 makes the top row see the zero wall node.
    std::fill(za.begin(), za.end(), 0.0);
    std::fill(zc.begin(), zc.end(), 0.0);
    std::fill(lo.begin(), lo.end(), 0.0);
    std::fill(hi.begin(), hi.end(), 0.0);
    zb[0] = -1.0;
    lo[0] = 0.5;
    for (int k = 1; k < nz; ++k) {
      const double h = dzc[k - 1];
      const double dn = 1.0 / (dzf[k - 1] * h), up = 1.0 / (dzf[k] * h);
      za[k] = lo[k] = dn;
      zb[k] = -(dn + up);
      if (k + 1 < nz) zc[k] = hi[k] = up;
      else hi[k] = 0.5 * up;
    }
  }
  double wsum = 0.0;
  for (int k = 0; k < nz; ++k) {
    split_df(lo[k], &zlo[k]);
    split_df(hi[k], &zhi[k]);
    wsum += dzf[k];
  }
  p->wsum = wsum;
  {
    float2 t;
    split_df(1.0 / (dx * dx), &t);
    p->idx2 = df{t.x, t.y};
    split_df(1.0 / (dy * dy), &t);
    p->idy2 = df{t.x, t.y};
  }
  {
    // every row: |diagonal| + Σ|off-diagonal| ≤ 2·(off-diagonal sum) + Dirichlet terms
    double zmax = 0.0;
    for (int k = 0; k < nz; ++k) {
      const double zr = std::fabs(za[k]) + std::fabs(zb[k]) + std::fabs(zc[k]);
      zmax = zr > zmax ? zr : zmax;
    }
    p->anorm = 8.0 / (dx * dx) + 8.0 / (dy * dy) + zmax + alpha;
  }
  // Sum form of a row for the residual passes m ≥ 1: A·e = Σ_j w_j·e_j over x±1,
  // y±1, z±1 and the centre (w_c = −Σ of the others). The ghost plane at a
  // Dirichlet z end is loaded as a copy of the boundary plane, so its coefficient
  // carries the ghost's sign (ghost = −Φ).
  std::vector<float2> zres(3 * (size_t)nz);
  {
    const double ix2 = 1.0 / (dx * dx), iy2 = 1.0 / (dy * dy);
    const bool dlo = (bcz == PS_BC_DIRICHLET_DIRICHLET || bcz == PS_BC_DIRICHLET_NEUMANN ||
                      bcz == PS_BC_FACE_DIRICHLET);
    const bool dhi = (bcz == PS_BC_DIRICHLET_DIRICHLET || bcz == PS_BC_NEUMANN_DIRICHLET ||
                      bcz == PS_BC_FACE_DIRICHLET);
    double asum = 0.0;
    for (int k = 0; k < nz; ++k) {
      const double cl = (k == 0 && dlo) ? -lo[k] : lo[k];
      const double ch = (k == nz - 1 && dhi) ? -hi[k] : hi[k];
      split_df(cl, &zres[3 * (size_t)k]);
      split_df(ch, &zres[3 * (size_t)k + 1]);
      split_df(-(2.0 * ix2 + 2.0 * iy2 + lo[k] + hi[k]) - alpha, &zres[3 * (size_t)k + 2]);
      const double rs = 4.0 * ix2 + 4.0 * iy2 + 2.0 * (lo[k] + hi[k]) + alpha;
      asum = rs > asum ? rs : asum;
    }
    p->asum = asum;
  }

  // ---- axis tables ----
  AxisTab* axes[2] = {&p->ax, &p->ay};
  const int ns[2] = {nx, ny};
  const int bcs[2] = {bcx, bcy};
  const double hs[2] = {dx, dy};
  size_t bytes = 0;
  for (int a = 0; a < 2; ++a) {
    const int n = ns[a];
    bytes += align256(8 * n * sizeof(cplx<double>)) + align256(8 * n * sizeof(cplx<float>));
    bytes += align256(n * sizeof(double)) + align256(n * sizeof(float));
  }
  bytes += 6 * align256(nz * sizeof(double)) + 6 * align256(nz * sizeof(float)) +
           2 * align256(nz * sizeof(float2)) + align256(3 * nz * sizeof(float2));
  char* dev = nullptr;
  cudaError_t e = take_injected_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&dev, bytes);
  if (e != cudaSuccess) {
    delete p;
    char buf[200];
    snprintf(buf, sizeof(buf), "cudaMalloc of plan tables: %s", cudaGetErrorString(e));
    return fail(nullptr, e == cudaErrorMemoryAllocation ? PS_OUT_OF_MEMORY : PS_CUDA_ERROR, buf);
  }
  p->dev = dev;
  size_t off = 0;
  {
    // FP32 paths with a non-periodic z: columns whose z system has κ ≈ ‖T_z‖/|λ| > 10^4
    // are solved in FP64 (tridiag.cu). λ grows with q along each axis, so they lie in
    // the rectangle q_x < lowx, q_y < lowy; at most 1/8 of the columns. A Helmholtz
    // shift adds α to every |λ| (all terms of the diagonal shift have one sign).
    p->lowx = p->lowy = 0;
    if (prec != PS_FP64 && bcz != PS_BC_PERIODIC) {
      double zmax = 0.0;
      for (int k = 0; k < nz; ++k)
        zmax = std::max(zmax, std::fabs(za[k]) + std::fabs(zb[k]) + std::fabs(zc[k]));
      const double thr = zmax / 1e4;
      const std::vector<double> lx = eig_scaled(bcx, nx, dx), ly = eig_scaled(bcy, ny, dy);
      int qx = 0, qy = 0;
      while (qx < nx && std::fabs(lx[qx]) + alpha < thr) ++qx;
      while (qy < ny && std::fabs(ly[qy]) + alpha < thr) ++qy;
      while ((size_t)qx * qy * 8 > (size_t)nx * ny && qy > 1) --qy;
      while ((size_t)qx * qy * 8 > (size_t)nx * ny && qx > 1) --qx;
      if ((size_t)qx * qy * 8 <= (size_t)nx * ny && qx > 0 && qy > 0) {
        p->lowx = qx;
        p->lowy = qy;
      }
    }
  }
  auto take = [&](size_t nbytes) { char* q = dev + off; off += align256(nbytes); return q; };
  std::vector<char> host(bytes, 0);
  auto hput = [&](void* devp, const void* src, size_t nbytes) {
    memcpy(host.data() + (static_cast<char*>(devp) - dev), src, nbytes);
  };
  for (int a = 0; a < 2; ++a) {
    AxisTab& t = *axes[a];
    const int n = ns[a];
    t.n = n;
    t.bc = bcs[a];
    t.m = t.bc == BC_FD ? n : n / 2;  // FD: the n-point FFT of the odd extension (xform_dev.cuh)
    t.nstages = make_radix(t.m, t.radix);
    t.tw64 = reinterpret_cast<cplx<double>*>(take(8 * n * sizeof(cplx<double>)));
    t.tw32 = reinterpret_cast<cplx<float>*>(take(8 * n * sizeof(cplx<float>)));
    t.lam64 = reinterpret_cast<double*>(take(n * sizeof(double)));
    t.lam32 = reinterpret_cast<float*>(take(n * sizeof(float)));
    std::vector<cplx<double>> tw64(8 * n);
    std::vector<cplx<float>> tw32(8 * n);
    for (int i = 0; i < 8 * n; ++i) {
      double c, s;
      cis(i, 8L * n, &c, &s);
      tw64[i] = {c, -s};  // e^{−2πi t/(8n)}
      tw32[i] = {(float)c, (float)-s};
    }
    std::vector<double> lam = eig_scaled(t.bc, n, hs[a]);
    std::vector<float> lam32(lam.begin(), lam.end());
    hput(t.tw64, tw64.data(), tw64.size() * sizeof(tw64[0]));
    hput(t.tw32, tw32.data(), tw32.size() * sizeof(tw32[0]));
    hput(t.lam64, lam.data(), n * sizeof(double));
    hput(t.lam32, lam32.data(), n * sizeof(float));
  }
  double** d64[6] = {&p->za64, &p->zb64, &p->zc64, &p->dzf64, &p->idzf64, &p->idzc64};
  float** d32[6] = {&p->za32, &p->zb32, &p->zc32, &p->dzf32, &p->idzf32, &p->idzc32};
  std::vector<double> idzf(nz), idzc(nz, 0.0);
  for (int k = 0; k < nz; ++k) idzf[k] = 1.0 / dzf[k];
  for (int k = 1; k < nz; ++k) idzc[k] = 1.0 / dzc[k - 1];
  if (bcz == PS_BC_PERIODIC) idzc[0] = 1.0 / (0.5 * (dzf[0] + dzf[nz - 1]));
  // the z solves' diagonal b_k carries the Helmholtz shift (−α on every row of Eq. 5)
  std::vector<double> zbs(zb);
  for (int k = 0; k < nz; ++k) zbs[k] -= alpha;
  const std::vector<double>* srcs[6] = {&za, &zbs, &zc, &dzf, &idzf, &idzc};
  for (int i = 0; i < 6; ++i) {
    *d64[i] = reinterpret_cast<double*>(take(nz * sizeof(double)));
    *d32[i] = reinterpret_cast<float*>(take(nz * sizeof(float)));
    std::vector<float> f32(srcs[i]->begin(), srcs[i]->end());
    hput(*d64[i], srcs[i]->data(), nz * sizeof(double));
    hput(*d32[i], f32.data(), nz * sizeof(float));
  }
  p->zlo = reinterpret_cast<float2*>(take(nz * sizeof(float2)));
  p->zhi = reinterpret_cast<float2*>(take(nz * sizeof(float2)));
  p->zres = reinterpret_cast<float2*>(take(3 * nz * sizeof(float2)));
  hput(p->zlo, zlo.data(), nz * sizeof(float2));
  hput(p->zhi, zhi.data(), nz * sizeof(float2));
  hput(p->zres, zres.data(), 3 * nz * sizeof(float2));
  e = cudaMemcpy(dev, host.data(), bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    delete p;
    return fail(nullptr, PS_CUDA_ERROR, "copy of plan tables failed");
  }
  p->err[0] = 0;
  *out = p;
  return PS_OK;
}

ps_status ps_workspace_bytes(const ps_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return fail(nullptr, PS_INVALID_ARG, "null argument");
  *bytes = ws_layout(plan).total;
  return PS_OK;
}

ps_status ps_solve(ps_plan* plan, const double* f, double* p, void* ws, void* stream, ps_info* info) {
  ps_status s = check_solve_args(plan, f, p, ws);
  if (s != PS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->prec == PS_FP64) return solve_plain<double>(plan, f, p, ws, st, info, false);
  if (plan->prec == PS_FP32_REFINE) {
    if (f == p) return fail(plan, PS_INVALID_ARG, "in-place solve is not allowed with refinement");
    return solve_refine(plan, f, p, ws, st, info);
  }
  return fail(plan, PS_INVALID_ARG, "FP32 plans take float fields: use ps_solve_f32");
}

ps_status ps_solve_f32(ps_plan* plan, const float* f, float* p, void* ws, void* stream, ps_info* info) {
  ps_status s = check_solve_args(plan, f, p, ws);
  if (s != PS_OK) return s;
  if (plan->prec != PS_FP32) return fail(plan, PS_INVALID_ARG, "ps_solve_f32 needs a PS_FP32 plan");
  return solve_plain<float>(plan, f, p, ws, static_cast<cudaStream_t>(stream), info, false);
}

ps_status ps_solve_transpose(ps_plan* plan, const double* g, double* p, void* ws, void* stream,
                             ps_info* info) {
  ps_status s = check_solve_args(plan, g, p, ws);
  if (s != PS_OK) return s;
  if (plan->bcz == PS_BC_FACE_DIRICHLET)
    return fail(plan, PS_INVALID_ARG, "no transpose solve for face unknowns in z");
  if (plan->prec == PS_FP64)
    return solve_plain<double>(plan, g, p, ws, static_cast<cudaStream_t>(stream), info, true);
  return fail(plan, PS_INVALID_ARG, "ps_solve_transpose needs a PS_FP64 plan");
}

ps_status ps_solve_transpose_f32(ps_plan* plan, const float* g, float* p, void* ws, void* stream,
                                 ps_info* info) {
  ps_status s = check_solve_args(plan, g, p, ws);
  if (s != PS_OK) return s;
  if (plan->bcz == PS_BC_FACE_DIRICHLET)
    return fail(plan, PS_INVALID_ARG, "no transpose solve for face unknowns in z");
  if (plan->prec != PS_FP32) return fail(plan, PS_INVALID_ARG, "needs a PS_FP32 plan");
  return solve_plain<float>(plan, g, p, ws, static_cast<cudaStream_t>(stream), info, true);
}

// The chunked copy of f feeds the register-resident x and y kernels of the refined
// solve (chunk c's first x and y passes start as it lands).
static bool host_pipe_ok(const ps_plan* plan) {
  return plan->prec == PS_FP32_REFINE && plan->nz >= 2 && plan->ax.bc != BC_FD && plan->ay.bc != BC_FD &&
         plan->nx % 16 == 0 && (plan->ax.m >= 64 && plan->ax.m <= 512) && (plan->ay.m >= 64 && plan->ay.m <= 512) &&
         !(plan->ax.m & (plan->ax.m - 1)) && !(plan->ay.m & (plan->ay.m - 1));
}

ps_status ps_solve_host(ps_plan* plan, const double* f_host, double* p_host, double* f_dev,
                        double* p_dev, void* ws, void* stream, ps_info* info_host) {
  ps_status s = check_solve_args(plan, f_dev, p_dev, ws);
  if (s != PS_OK) return s;
  if (!f_host || !p_host) return fail(plan, PS_INVALID_ARG, "null host pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = plan->N * sizeof(double);
  ps_info* info_dev = reinterpret_cast<ps_info*>(static_cast<char*>(ws) + ws_layout(plan).info);
  cudaError_t e;
  // Refinement with the register-resident x and y kernels: the copy of f in chunks
  // of planes on a side stream, each chunk's first x and y passes as it lands; the
  // copy of each chunk of p as soon as the first correction's x pass has written it
  // (overlapping the rest of that pass and of the loop), and p again after the loop
  // if a later correction changed it.
  const bool pipe = f_dev != p_dev && host_pipe_ok(plan);
  if (pipe) {
    if (!plan->copy_stream) {
      if ((e = cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(plan, e, "copy stream");
      for (auto& ev : plan->pipe_ev)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
          return cuda_fail(plan, e, "copy events");
    }
    cudaStream_t cs = plan->copy_stream;
    HostPipe hp;
    hp.nch = plan->nz < kPipeMax ? plan->nz : kPipeMax;
    for (int c = 0; c <= hp.nch; ++c) hp.z[c] = (int)((long long)plan->nz * c / hp.nch);
    for (int c = 0; c < hp.nch; ++c) {
      hp.in[c] = plan->pipe_ev[c];
      hp.out[c] = plan->pipe_ev[kPipeMax + c];
    }
    cudaEvent_t start = plan->pipe_ev[2 * kPipeMax];
    // the copies wait for the caller's earlier work on its stream (which may use f_dev)
    if ((e = cudaEventRecord(start, st)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, start, 0)) != cudaSuccess)
      return cuda_fail(plan, e, "copy stream order");
    const size_t plane = (size_t)plan->nx * plan->ny;
    for (int c = 0; c < hp.nch; ++c) {
      const size_t off = (size_t)hp.z[c] * plane, n = (size_t)(hp.z[c + 1] - hp.z[c]) * plane;
      if ((e = cudaMemcpyAsync(f_dev + off, f_host + off, n * sizeof(double), cudaMemcpyHostToDevice, cs)) !=
              cudaSuccess ||
          (e = cudaEventRecord(hp.in[c], cs)) != cudaSuccess)
        return cuda_fail(plan, e, "host to device copy");
    }
    s = solve_refine(plan, f_dev, p_dev, ws, st, info_dev, &hp);
    if (s != PS_OK) {
      cudaStreamSynchronize(cs);
      return s;
    }
    for (int c = 0; hp.p_recorded && c < hp.nch; ++c) {
      const size_t off = (size_t)hp.z[c] * plane, n = (size_t)(hp.z[c + 1] - hp.z[c]) * plane;
      if ((e = cudaStreamWaitEvent(cs, hp.out[c], 0)) != cudaSuccess ||
          (e = cudaMemcpyAsync(p_host + off, p_dev + off, n * sizeof(double), cudaMemcpyDeviceToHost, cs)) !=
              cudaSuccess)
        return cuda_fail(plan, e, "device to host copy");
    }
    ps_info rec{};
    if ((e = cudaMemcpyAsync(&rec, info_dev, sizeof(ps_info), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(plan, e, "info copy");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess || (e = cudaStreamSynchronize(cs)) != cudaSuccess)
      return cuda_fail(plan, e, "stream synchronize");
    // p changed after the early copy unless the loop stopped at the first correction
    if (!hp.p_recorded || rec.iterations != 1) {
      if ((e = cudaMemcpyAsync(p_host, p_dev, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(plan, e, "device to host copy");
    }
    if (info_host) *info_host = rec;
    return PS_OK;
  }
  e = cudaMemcpyAsync(f_dev, f_host, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(plan, e, "host to device copy");
  s = ps_solve(plan, f_dev, p_dev, ws, stream, info_dev);
  if (s != PS_OK) return s;
  if ((e = cudaMemcpyAsync(p_host, p_dev, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(plan, e, "device to host copy");
  if (info_host && (e = cudaMemcpyAsync(info_host, info_dev, sizeof(ps_info), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(plan, e, "info copy");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(plan, e, "stream synchronize");
  return PS_OK;
}

ps_status ps_solve_host_seq(ps_plan* plan, int count, const double* const* f_host, double* const* p_host,
                            double* const* f_dev, double* const* p_dev, void* ws, void* stream,
                            ps_info* info_host) {
  if (!plan) return fail(nullptr, PS_INVALID_ARG, "null plan");
  if (count < 0) return fail(plan, PS_INVALID_ARG, "negative count");
  if (count == 0) return PS_OK;
  if (!f_host || !p_host || !f_dev || !p_dev) return fail(plan, PS_INVALID_ARG, "null pointer array");
  for (int s = 0; s < count; ++s)
    if (!f_host[s] || !p_host[s]) return fail(plan, PS_INVALID_ARG, "null host pointer");
  for (int d = 0; d < 2; ++d) {
    ps_status st = check_solve_args(plan, f_dev[d], p_dev[d], ws);
    if (st != PS_OK) return st;
  }
  const size_t bytes = plan->N * sizeof(double);
  {  // the four device buffers must be disjoint
    const char* b[4] = {reinterpret_cast<const char*>(f_dev[0]), reinterpret_cast<const char*>(f_dev[1]),
                        reinterpret_cast<const char*>(p_dev[0]), reinterpret_cast<const char*>(p_dev[1])};
    for (int u = 0; u < 4; ++u)
      for (int v = u + 1; v < 4; ++v)
        if (b[u] < b[v] + bytes && b[v] < b[u] + bytes)
          return fail(plan, PS_INVALID_ARG, "the device buffers of the two slots overlap");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!host_pipe_ok(plan)) {  // no chunked pipeline for this plan: one problem after another
    for (int s = 0; s < count; ++s) {
      const ps_status r = ps_solve_host(plan, f_host[s], p_host[s], f_dev[0], p_dev[0], ws, stream,
                                        info_host ? info_host + s : nullptr);
      if (r != PS_OK) return r;
    }
    return PS_OK;
  }
  cudaError_t e;
  if (!plan->copy_stream || !plan->out_stream) {
    if (!plan->copy_stream) {
      if ((e = cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(plan, e, "copy stream");
      for (auto& ev : plan->pipe_ev)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
          return cuda_fail(plan, e, "copy events");
    }
    if ((e = cudaStreamCreateWithFlags(&plan->out_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(plan, e, "copy-out stream");
    for (auto& row : plan->seq_ev)
      for (auto& ev : row)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
          return cuda_fail(plan, e, "sequence events");
  }
  if (info_host && plan->info_cap < count) {
    if (plan->info_pinned) cudaFreeHost(plan->info_pinned);
    plan->info_pinned = nullptr;
    plan->info_cap = 0;
    if ((e = cudaHostAlloc(&plan->info_pinned, (size_t)count * sizeof(ps_info), cudaHostAllocDefault)) != cudaSuccess) {
      plan->info_pinned = nullptr;
      return cuda_fail(plan, e, "pinned info buffer");
    }
    plan->info_cap = count;
  }
  cudaStream_t cin = plan->copy_stream, cout = plan->out_stream;
  ps_info* info_dev = reinterpret_cast<ps_info*>(static_cast<char*>(ws) + ws_layout(plan).info);
  auto drain = [&]() {  // (on an error: let every enqueued copy and launch finish)
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(cin);
    cudaStreamSynchronize(cout);
  };
  // the copies wait for the caller's earlier work on its stream (which may use the buffers)
  cudaEvent_t start = plan->pipe_ev[2 * kPipeMax];
  if ((e = cudaEventRecord(start, st)) != cudaSuccess || (e = cudaStreamWaitEvent(cin, start, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(cout, start, 0)) != cudaSuccess)
    return cuda_fail(plan, e, "copy stream order");
  const size_t plane = (size_t)plan->nx * plan->ny;
  for (int s = 0; s < count; ++s) {
    const int d = s & 1;
    cudaEvent_t* ev = plan->seq_ev[d];
    HostPipe hp;
    hp.nch = plan->nz < kPipeMax ? plan->nz : kPipeMax;
    hp.chunk_out = false;
    for (int c = 0; c <= hp.nch; ++c) hp.z[c] = (int)((long long)plan->nz * c / hp.nch);
    for (int c = 0; c < hp.nch; ++c) hp.in[c] = ev[c];
    // copy in: slot d's f is free once problem s − 2's solve has ended
    if (s >= 2 && (e = cudaStreamWaitEvent(cin, ev[kSeqComp], 0)) != cudaSuccess) {
      drain();
      return cuda_fail(plan, e, "copy stream order");
    }
    for (int c = 0; c < hp.nch; ++c) {
      const size_t off = (size_t)hp.z[c] * plane, n = (size_t)(hp.z[c + 1] - hp.z[c]) * plane;
      if ((e = cudaMemcpyAsync(f_dev[d] + off, f_host[s] + off, n * sizeof(double), cudaMemcpyHostToDevice, cin)) !=
              cudaSuccess ||
          (e = cudaEventRecord(hp.in[c], cin)) != cudaSuccess) {
        drain();
        return cuda_fail(plan, e, "host to device copy");
      }
    }
    // solve: slot d's p is free once problem s − 2's copy out has ended
    if (s >= 2 && (e = cudaStreamWaitEvent(st, ev[kSeqOut], 0)) != cudaSuccess) {
      drain();
      return cuda_fail(plan, e, "stream order");
    }
    const ps_status r = solve_refine(plan, f_dev[d], p_dev[d], ws, st, info_dev, &hp);
    if (r != PS_OK) {
      drain();
      return r;
    }
    if (info_host &&
        (e = cudaMemcpyAsync(plan->info_pinned + s, info_dev, sizeof(ps_info), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess) {
      drain();
      return cuda_fail(plan, e, "info copy");
    }
    // copy out after the solve, while the next problem's copy in and solve proceed
    if ((e = cudaEventRecord(ev[kSeqComp], st)) != cudaSuccess || (e = cudaStreamWaitEvent(cout, ev[kSeqComp], 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(p_host[s], p_dev[d], bytes, cudaMemcpyDeviceToHost, cout)) != cudaSuccess ||
        (e = cudaEventRecord(ev[kSeqOut], cout)) != cudaSuccess) {
      drain();
      return cuda_fail(plan, e, "device to host copy");
    }
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess || (e = cudaStreamSynchronize(cin)) != cudaSuccess ||
      (e = cudaStreamSynchronize(cout)) != cudaSuccess)
    return cuda_fail(plan, e, "stream synchronize");
  if (info_host) memcpy(info_host, plan->info_pinned, (size_t)count * sizeof(ps_info));
  return PS_OK;
}

ps_status ps_profile_enable(ps_plan* plan, int enable) {
  if (!plan) return fail(nullptr, PS_INVALID_ARG, "null plan");
  Prof& pr = plan->prof;
  if (enable && pr.ev.empty()) {
    pr.ev.resize(2 * kProfMax);
    pr.kind.resize(kProfMax);
    for (auto& ev : pr.ev) {
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_fail(plan, e, "cudaEventCreate");
    }
  }
  pr.on = enable ? 1 : 0;
  pr.n = 0;
  return PS_OK;
}

ps_status ps_profile_read(ps_plan* plan, ps_kernel_stat* stats, int max, int* count) {
  if (!plan || !stats || !count) return fail(nullptr, PS_INVALID_ARG, "null argument");
  Prof& pr = plan->prof;
  std::vector<float> ms(pr.n, 0.f);
  float kmax[K_NKINDS] = {0};
  for (int i = 0; i < pr.n; ++i) {
    cudaError_t e = cudaEventSynchronize(pr.ev[2 * i + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[i], pr.ev[2 * i], pr.ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(plan, e, "event timing");
    if (ms[i] > kmax[pr.kind[i]]) kmax[pr.kind[i]] = ms[i];
  }
  int c = 0;
  for (int k = 0; k < K_NKINDS && c < max; ++k) {
    ps_kernel_stat& st = stats[c];
    memset(&st, 0, sizeof(st));
    snprintf(st.name, sizeof(st.name), "%s", kKindName[k]);
    for (int i = 0; i < pr.n; ++i) {
      if (pr.kind[i] != k) continue;
      st.launches++;
      st.total_ms += ms[i];
      if (ms[i] >= 0.25f * kmax[k]) {
        st.active_launches++;
        st.active_ms += ms[i];
      }
    }
    ++c;
  }
  *count = c;
  pr.n = 0;
  return PS_OK;
}

// ---- projection step around the solve (Eqs. 2b–2c) -----------------------------

}  // extern "C"

namespace {
template <class T>
ProjArgs<T> proj_args(const ps_plan* p) {
  ProjArgs<T> a{};
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.per[0] = p->bcx == PS_BC_PERIODIC;
  a.per[1] = p->bcy == PS_BC_PERIODIC;
  a.per[2] = p->bcz == PS_BC_PERIODIC;
  a.idx = (T)(1.0 / p->dx);
  a.idy = (T)(1.0 / p->dy);
  if constexpr (sizeof(T) == 8) { a.idzf = p->idzf64; a.idzc = p->idzc64; }
  else { a.idzf = p->idzf32; a.idzc = p->idzc32; }
  return a;
}

ps_status projection_op(ps_plan* p, int op, const void* x0, const void* x1, void* y, void* stream) {
  if (!p) return fail(nullptr, PS_INVALID_ARG, "null plan");
  if (!x0 || !y || ((op == 1 || op == 3) && !x1)) return fail(p, PS_INVALID_ARG, "null field pointer");
  auto pn = [](int b) { return b == PS_BC_PERIODIC || b == PS_BC_NEUMANN_NEUMANN; };
  if (!pn(p->bcx) || !pn(p->bcy) || !pn(p->bcz))
    return fail(p, PS_INVALID_ARG, "projection needs periodic or Neumann-Neumann axes");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = (p->prec == PS_FP32) ? launch_projection<float>(op, proj_args<float>(p), x0, x1, y, st)
                                       : launch_projection<double>(op, proj_args<double>(p), x0, x1, y, st);
  return e == cudaSuccess ? PS_OK : cuda_fail(p, e, "projection kernel");
}
}  // namespace

extern "C" {

ps_status ps_div(ps_plan* plan, const void* u, void* f, void* stream) {
  return projection_op(plan, 0, u, nullptr, f, stream);
}
ps_status ps_grad_correct(ps_plan* plan, const void* ustar, const void* phi, void* u, void* stream) {
  return projection_op(plan, 1, ustar, phi, u, stream);
}
ps_status ps_grad_adjoint(ps_plan* plan, const void* g, void* h, void* stream) {
  return projection_op(plan, 2, g, nullptr, h, stream);
}
ps_status ps_div_adjoint_correct(ps_plan* plan, const void* g, const void* s, void* out, void* stream) {
  return projection_op(plan, 3, g, s, out, stream);
}

ps_status ps_ns_substep(ps_plan* plan, int k, double dt, double nu, void* u, void* ustar, void* ad, void* p,
                        void* phi, void* rhs, void* ws, void* stream, ps_info* info) {
  if (!plan) return fail(nullptr, PS_INVALID_ARG, "null plan");
  if (!u || !ustar || !ad || !p || !phi || !rhs || !ws) return fail(plan, PS_INVALID_ARG, "null pointer");
  if ((((uintptr_t)u) | ((uintptr_t)ustar) | ((uintptr_t)ad) | ((uintptr_t)p) | ((uintptr_t)phi) |
       ((uintptr_t)rhs)) & 15)
    return fail(plan, PS_INVALID_ARG, "the substep's arrays must be 16-byte aligned");
  {
    // Every array is read and written at different stages (p += Φ reads phi, the
    // solve overwrites ws and phi, the divergence writes rhs from ustar), so any
    // overlap of their byte ranges changes the result: refuse it.
    const size_t es = plan->prec == PS_FP32 ? sizeof(float) : sizeof(double);
    size_t wsb = 0;
    ps_workspace_bytes(plan, &wsb);
    const struct { const char* name; uintptr_t lo; size_t bytes; } arr[7] = {
        {"u", (uintptr_t)u, 3 * plan->N * es},       {"ustar", (uintptr_t)ustar, 3 * plan->N * es},
        {"ad", (uintptr_t)ad, 3 * plan->N * es},     {"p", (uintptr_t)p, plan->N * es},
        {"phi", (uintptr_t)phi, plan->N * es},       {"rhs", (uintptr_t)rhs, plan->N * es},
        {"ws", (uintptr_t)ws, wsb}};
    for (int i = 0; i < 7; ++i)
      for (int j = i + 1; j < 7; ++j)
        if (arr[i].bytes && arr[j].bytes && arr[i].lo < arr[j].lo + arr[j].bytes &&
            arr[j].lo < arr[i].lo + arr[i].bytes) {
          char msg[128];
          snprintf(msg, sizeof(msg), "%s and %s overlap: u, ustar, ad, p, phi, rhs and ws must be disjoint",
                   arr[i].name, arr[j].name);
          return fail(plan, PS_INVALID_ARG, msg);
        }
  }
  if (k < 1 || k > 3) return fail(plan, PS_INVALID_ARG, "the RK3 substep k must be 1, 2 or 3");
  if (!(dt > 0.0) || !std::isfinite(dt) || !(nu >= 0.0) || !std::isfinite(nu))
    return fail(plan, PS_INVALID_ARG, "dt must be > 0 and nu >= 0 (finite)");
  auto pw = [](int b) { return b == PS_BC_PERIODIC || b == PS_BC_NEUMANN_NEUMANN; };
  if (!pw(plan->bcx) || !pw(plan->bcy) || !pw(plan->bcz))
    return fail(plan, PS_INVALID_ARG, "the substep needs each axis periodic or Neumann (no-slip walls)");
  if (plan->alpha != 0.0) return fail(plan, PS_INVALID_ARG, "the substep needs a Poisson plan (alpha = 0)");
  static const double kAlpha[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
  static const double kBeta[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};
  const double al = kAlpha[k - 1], be = kBeta[k - 1], ga = al + be;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t N = plan->N;
  auto body = [&](auto tag) -> ps_status {
    using T = decltype(tag);
    NsArgs<T> a{};
    a.nx = plan->nx;
    a.ny = plan->ny;
    a.nz = plan->nz;
    a.per_x = plan->bcx == PS_BC_PERIODIC;
    a.per_y = plan->bcy == PS_BC_PERIODIC;
    a.per_z = plan->bcz == PS_BC_PERIODIC;
    a.idx = (T)(1.0 / plan->dx);
    a.idy = (T)(1.0 / plan->dy);
    a.idx2 = (T)(1.0 / (plan->dx * plan->dx));
    a.idy2 = (T)(1.0 / (plan->dy * plan->dy));
    a.qx = (T)(0.25 / plan->dx);
    a.qy = (T)(0.25 / plan->dy);
    if constexpr (sizeof(T) == 8) { a.idzf = plan->idzf64; a.idzc = plan->idzc64; }
    else { a.idzf = plan->idzf32; a.idzc = plan->idzc32; }
    a.nu = (T)nu;
    a.dt = (T)dt;
    a.alpha = (T)al;
    a.beta = (T)be;
    a.gamma = (T)ga;
    {
      const double c[11] = {1.0 / plan->dx, 1.0 / plan->dy, 1.0 / (plan->dx * plan->dx),
                            1.0 / (plan->dy * plan->dy), 0.25 / plan->dx, 0.25 / plan->dy, nu, dt, al, be, ga};
      for (int q = 0; q < 11; ++q) {
        const float h = (float)c[q];
        a.dc[q] = make_float2(h, (float)(c[q] - (double)h));
      }
    }
    cudaError_t e;
    if ((e = run(plan, K_NSPRED, st, [&] { return launch_ns_predict<T>(a, u, p, ad, ustar, ad, st); })) !=
        cudaSuccess)
      return cuda_fail(plan, e, "substep predictor");
    const ProjArgs<T> pa = proj_args<T>(plan);
    if ((e = run(plan, K_NSPROJ, st, [&] { return launch_projection<T>(0, pa, ustar, nullptr, rhs, st); })) !=
        cudaSuccess)
      return cuda_fail(plan, e, "substep divergence");
    ps_status s;
    if constexpr (sizeof(T) == 4)
      s = ps_solve_f32(plan, static_cast<const float*>(rhs), static_cast<float*>(phi), ws, stream, info);
    else
      s = ps_solve(plan, static_cast<const double*>(rhs), static_cast<double*>(phi), ws, stream, info);
    if (s != PS_OK) return s;
    if ((e = run(plan, K_NSPROJ, st, [&] { return launch_projection<T>(1, pa, ustar, phi, u, st); })) !=
        cudaSuccess)
      return cuda_fail(plan, e, "substep projection");
    if ((e = run(plan, K_NSPRES, st, [&] { return launch_ns_pressure<T>(N, 1.0 / (ga * dt), p, phi, st); })) !=
        cudaSuccess)
      return cuda_fail(plan, e, "substep pressure update");
    return PS_OK;
  };
  return plan->prec == PS_FP32 ? body(float{}) : body(double{});
}

ps_status ps_plan_destroy(ps_plan* plan) {
  if (!plan) return PS_OK;
  for (auto& ev : plan->prof.ev) cudaEventDestroy(ev);
  for (auto& ev : plan->pipe_ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& row : plan->seq_ev)
    for (auto& ev : row)
      if (ev) cudaEventDestroy(ev);
  if (plan->copy_stream) cudaStreamDestroy(plan->copy_stream);
  if (plan->out_stream) cudaStreamDestroy(plan->out_stream);
  if (plan->info_pinned) cudaFreeHost(plan->info_pinned);
  if (plan->dev) cudaFree(plan->dev);
  delete plan;
  return PS_OK;
}

const char* ps_last_error(const ps_plan* plan) { return plan ? plan->err : g_create_err; }

ps_status ps_inject_alloc_failures(int count) {
  if (count < 0) return PS_INVALID_ARG;
  g_inject_alloc.store(count);
  return PS_OK;
}

}  // extern "C"
