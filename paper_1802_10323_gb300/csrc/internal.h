// internal.h — declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/ps_poisson.h"
#include "common.cuh"

namespace ps {

enum { BC_P = 0, BC_NN = 1, BC_DD = 2, BC_ND = 3, BC_DN = 4, BC_FD = 5 /* z only: face unknowns */ };
// ND and DN share the DCT-IV line transform: DN is the ND problem on the reversed
// line, so on the physical side of a transform the two reals x_{2p} and x_{n−1−2p}
// trade places; the spectral side, the tables and the eigenvalues are ND's.
__host__ __device__ inline bool bc_iv(int bc) { return bc == BC_ND || bc == BC_DN; }
// Longest x or y line: lines of n ≤ 1024 run in the register-resident transform
// kernels; longer ones in the shared-memory kernel, one line per CTA (two buffers
// of n/2 + 1 complex values: 131 KB for an FP64 line of 8192)
constexpr int kMaxN = 8192;
constexpr int kMaxStages = 12;
extern thread_local char g_launch_diag[256];  // configuration of the last failed launch
// Test hook (ps_inject_alloc_failures): true while injected device-allocation failures
// remain; each call consumes one.
bool take_injected_alloc_failure();

// Arguments of one batch of line transforms (x or y).
template <class T>
struct XformArgs {
  const void* in;
  void* out;
  int n, m;          // line length and half length
  int axis;          // 0 = x (contiguous rows), 1 = y (strided by nx)
  int nx, ny, nz;
  int nlines;        // x: nz*ny rows
  int L;             // lines per CTA (set by the launcher)
  int bc;
  int nstages;
  int radix[kMaxStages];
  const cplx<T>* tw;        // e^{−2πi t/(8n)}, t = 0 … 8n−1
  const T* plane_scale;     // per-z factor on load (fwd) / store (bwd), or null
  int accumulate;           // store: out = out + v
  const int* skip;          // if non-null and *skip != 0 the kernel returns at once
  unsigned long long* amax; // FP64 output: atomicMax of |transform output| bit patterns, or null
  float* out2;              // FP64 output: also store the FP32 transform output here, or null
  const float* base32;      // FP64 output: out = widen(base32) + v instead of (out +) v, or null
};

template <class T, class TI, class TO, bool FWD>
cudaError_t launch_xform(XformArgs<T> a, cudaStream_t st);

// z tridiagonal solves of Eq. 5, one per (q_x, q_y) column.
template <class T>
struct ZArgs {
  T* data;                  // [nz][ny][nx], spectral in x and y; overwritten with Φ̂
  T* scr_c;                 // scratch, nx*ny*nz (eliminated upper diagonal)
  T* scr_u;                 // scratch for the periodic (Sherman–Morrison) column, or null
  int nx, ny, nz;
  const T* lamx;            // λ_qx/Δx², nx
  const T* lamy;            // λ_qy/Δy², ny
  const T* za;              // a_k (sub-diagonal; a_0 = wrap coupling when periodic)
  const T* zb;              // b_k (diagonal incl. Dirichlet ghost terms)
  const T* zc;              // c_k (super-diagonal; c_{n−1} = wrap coupling when periodic)
  const T* dzf;             // cell widths (weights of the singular column)
  int periodic;
  int singular;             // column (0,0) is singular: handled by the fix-up kernel
  const int* skip;
  // FP32 path, non-periodic z: the columns q_x < lowx, q_y < lowy (the worst-conditioned,
  // see tridiag.cu) are solved in FP64 by extra CTAs of the same launch (0: none).
  int lowx, lowy;
  const double *lamx64, *lamy64, *za64, *zb64, *zc64, *dzf64;
  double* scr64;            // 2·nz·lowx·lowy doubles
};

template <class T>
cudaError_t launch_zsolve(ZArgs<T> a, cudaStream_t st);
template <class T>
cudaError_t launch_zsingular(ZArgs<T> a, cudaStream_t st);
cudaError_t launch_zsolve_ckpt(ZArgs<float> a, cudaStream_t st);  // FP32, non-periodic

// Residuals of the refinement (residual.cu): incremental passes on an FP32
// operand with a double-float base, and the exact pass from the FP64 solution.
struct ResidArgs {
  const double* p;          // exact pass: the stored FP64 solution
  const double* f;          // exact pass and incremental pass 0: the right-hand side
  float* r;                 // exact pass: FP32 residual out (n_x·n_y·n_z floats)
  const float* u;           // incremental: FP32 operand (Φ_0 in pass 0, the last correction later)
  const float* rh_in;       // incremental pass ≥ 1: r_{m−1} = rh + rl
  const float* rl_in;
  float* rh_out;            // incremental: r_m = rh + rl out, or both null (norms only)
  float* rl_out;
  int nx, ny, nz;
  int bcx, bcy, bcz;        // ends: see residual.cu
  df idx2, idy2;            // 1/Δx², 1/Δy²
  const float2* zlo;        // coefficient of (Φ_{k−1} − Φ_k), ghost rules folded in
  const float2* zhi;        // coefficient of (Φ_{k+1} − Φ_k)
  const float2* zres;       // passes m ≥ 1: per plane (a_k, c_k, w_c) in double-float, the
                            // Dirichlet ghost sign folded into a_0 / c_{n−1} (see residual.cu)
  double asum;              // max over planes of Σ_j |w_j| (the 7 coefficients of a row)
  df nalpha;                // −α of a Helmholtz plan (A − α·I), double-float; zero otherwise
  const float* wz;          // Δz^f_k (weights of the mean, singular problems)
  const float* mu;          // double-float volume-weighted mean of f (singular)
  const unsigned long long* pmax_bits;  // bit pattern of max|operand| (sets the fixed-point scale)
  int singular;
  int* red;                 // per-call reduction words (see residual.cu)
  float* partial;           // per-block double-float weighted sums (2 floats per block) ×2
  int nblocks;
  int zchunk;               // planes per CTA (set by the launcher)
  const int* skip;
};

// CTAs (= partial sums) of a residual pass: which = 0 pass 0 (two-level split),
// 1 three-level split (pass 0 repeated, exact pass), 2 passes m ≥ 1
int residual_blocks(int nx, int ny, int nz, int which);
cudaError_t launch_residual_inc(const ResidArgs& a, int pass, int split3, cudaStream_t st);
cudaError_t launch_residual_exact(const ResidArgs& a, cudaStream_t st);

// Control block at the start of the workspace.
struct Ctrl {
  int converged;            // set when ‖r‖ ≤ rtol·‖f_c‖ (refinement done)
  int iterations;
  int status;
  int vskip;                // 1: the exact confirmation pass is not needed
  int red[8];               // reduction words of the current residual pass (r: 0–1, f: 2–3)
  double rel, rnorm, fnorm;
  float mu[2];              // double-float weighted mean of f, set by the first finalize
  double mf;                // the same mean in FP64
  unsigned long long pmax;  // bit pattern of max|Φ| after the first FP32 solve
  unsigned long long dmax;  // bit pattern of max|e| of the last correction
  double bnd;               // accumulated drift bound of the incremental residual
  int skip_redo;            // 0: pass 0 is repeated with the three-level split
  int nomat0;               // 0: the loop ended at pass 0, p is written from Φ_0
  int skip_out;             // 0: a pass m ≥ 1 found no convergence; it is repeated with its output
  int pad2;
  unsigned long long dmax_prev;  // max|e| of the correction the current pass used
};

cudaError_t launch_finalize(Ctrl* ctrl, const float* partial, int nblocks, double wsum_total,
                            int singular, double rtol, int iteration, int attempt, int last,
                            double anorm, const int* skip, ps_info* info, cudaStream_t st);
// p = Φ_0 (widened exactly) unless *skip.
cudaError_t launch_widen(const float* u, double* p, size_t n, const int* skip, cudaStream_t st);
cudaError_t launch_finalize_exact(Ctrl* ctrl, const float* partial, int nblocks, double wsum_total,
                                  int singular, double rtol, ps_info* info, cudaStream_t st);
cudaError_t launch_info_plain(ps_info* info, cudaStream_t st);

// Staggered divergence / gradient of the projection step and their adjoints.
template <class T>
struct ProjArgs {
  int nx, ny, nz;
  int per[3];
  T idx, idy;
  const T* idzf;
  const T* idzc;
};
// op: 0 f = D u; 1 u = u* − G φ; 2 h = Gᵀ g; 3 out = g − Dᵀ s
template <class T>
cudaError_t launch_projection(int op, const ProjArgs<T>& a, const void* x0, const void* x1, void* y,
                              cudaStream_t st);

// One RK3 substep around the solve (navier_stokes.cu): the predictor (2a) and the
// pressure update (2d). idzf[k] = 1/Δz^f_k; idzc[k] = 1/(centre distance between
// cells k−1 and k), idzc[0] the periodic wrap.
template <class T>
struct NsArgs {
  int nx, ny, nz;
  int per_x, per_y, per_z;  // axis periodic (else no-slip walls at both ends)
  T idx, idy, idx2, idy2;   // 1/Δx, 1/Δy, 1/Δx², 1/Δy²
  T qx, qy;                 // ¼/Δx, ¼/Δy (flux differences of products of two sums)
  const T* idzf;
  const T* idzc;
  T nu, dt, alpha, beta, gamma;
  // FP64 fields: idx, idy, idx2, idy2, qx, qy, nu, dt, alpha, beta, gamma split into
  // hi + lo floats on the host (the predictor's double-float constants, read as
  // operands from the parameter bank instead of held in registers)
  float2 dc[11];
};
template <class T>
cudaError_t launch_ns_predict(const NsArgs<T>& a, const void* u3, const void* p, const void* ad_prev,
                              void* ustar, void* ad_out, cudaStream_t st);
template <class T>
cudaError_t launch_ns_pressure(size_t N, double scale, void* p, void* phi, cudaStream_t st);

// Record a message for ps_last_error(plan).
void set_plan_error(ps_plan* plan, const char* msg);

// The FP32 tables of a plan (used by the batched solve).
double ps_plan_internal_alpha(const ps_plan* p);  // the plan's Helmholtz shift (0: Poisson)
void ps_plan_internal_tables(const ps_plan* p, const cplx<float>** twx, const cplx<float>** twy,
                             const float** lamx, const float** lamy, const float** za, const float** zb,
                             const float** zc, const float** dzf, const float2** zlo, const float2** zhi,
                             df* idx2, df* idy2, double* wsum_total, int* radx, int* rady, int* nstx,
                             int* nsty);

}  // namespace ps
