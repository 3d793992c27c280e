// batch.cu — many independent grids solved by one persistent launch.
//
// Every grid is its own problem of §2.1 (sizes, spacings, z faces and BC pairs
// per grid) solved in FP32 with FP64 iterative refinement. The work of all
// grids is cut into tasks (grid, stage, tile): x/y line groups of the
// transforms (Table 2), blocks of z columns (Eq. 5), the singular column,
// residual tiles and the per-grid convergence test. A task table ordered by
// stage (then grid, then tile) is walked by one persistent kernel whose CTAs
// take the next task from a global counter. A task may start once every task of
// the previous non-empty stage of its own grid is done (per-(grid, stage)
// completion counters, release/acquire fences). All CTAs are resident and tasks
// are taken in table order, so every task a CTA waits for has been taken by a
// running CTA. Waits are bounded by a wall-clock limit: on expiry the kernel
// raises an abort flag, every later task is skipped, and the grids report
// PS_TIMEOUT instead of hanging. The whole solve is two memsets, the persistent
// kernel and a small record kernel, so it can be captured in a CUDA graph.
//
// Tile sizes (lines per transform task, points per residual task) come from a
// scale factor chosen by ps_batch_autotune (timed candidates; optional JSON
// cache named by PS_AUTOTUNE_CACHE).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "tridiag_dev.cuh"
#include "xform_dev.cuh"

namespace ps {

template <class T>
int pick_lines(int n, int axis, int nx, int nlines);

enum BStage { BS_XF64 = 0, BS_XF, BS_YF, BS_Z, BS_ZS, BS_YB, BS_XBST, BS_XBACC, BS_RES, BS_CHK, BS_FIN };

struct BGrid {
  int nx, ny, nz, bcx, bcy, bcz, singular, periodic_z;
  int mx, my, nstx, nsty;
  int radx[kMaxStages], rady[kMaxStages];
  int Lx, Ly;              // lines per transform task
  int res_chunk;           // points per residual task
  int ntask[4];            // x tasks, y tasks, z tasks, residual tasks
  const cplx<float>* twx;
  const cplx<float>* twy;
  const float *lamx, *lamy, *za, *zb, *zc, *dzf;
  const float2 *zlo, *zhi;
  df idx2, idy2;
  int shift;               // Helmholtz grid: the residual row also holds −α·Φ
  df nalpha;               // −α in double-float
  double wsum_total;
  size_t ws_off;           // this grid's slice: partials | w | scr | scr_u
  size_t off_w, off_scr, off_scru;
};

struct BatchArgs {
  const BGrid* grids;
  const int4* tasks;       // (grid, stage, tile, 0)
  int ntasks, nstage;
  const int* need;         // [grid][stage] task counts
  const int* dep;          // [grid][stage] stage to wait for, or −1
  const int* stage_type;   // [stage]
  const int* stage_it;     // [stage] refinement iteration
  int* done;               // [grid][stage] completed tasks
  int* next;               // task counter
  int* abort;              // wait expired
  Ctrl* ctrl;              // [grid]
  char* ws;
  double* const* f;
  double* const* p;
  ps_info* infos;
  double rtol;
  int max_iter;
  unsigned long long wait_ns;
  int inject;              // test hook: one dependency that is never satisfied
};

__device__ XformArgs<float> bx_args(const BGrid& G, int axis, const void* in, void* out, int acc,
                                    unsigned long long* amax) {
  XformArgs<float> a{};
  a.in = in;
  a.out = out;
  a.axis = axis;
  a.nx = G.nx;
  a.ny = G.ny;
  a.nz = G.nz;
  if (axis == 0) {
    a.n = 2 * G.mx; a.m = G.mx; a.L = G.Lx; a.nlines = G.ny * G.nz; a.bc = G.bcx;
    a.nstages = G.nstx; a.tw = G.twx;
    for (int i = 0; i < kMaxStages; ++i) a.radix[i] = G.radx[i];
  } else {
    a.n = 2 * G.my; a.m = G.my; a.L = G.Ly; a.nlines = G.nx * G.nz; a.bc = G.bcy;
    a.nstages = G.nsty; a.tw = G.twy;
    for (int i = 0; i < kMaxStages; ++i) a.radix[i] = G.rady[i];
  }
  a.plane_scale = nullptr;
  a.accumulate = acc;
  a.skip = nullptr;
  a.amax = amax;
  return a;
}

__device__ ZArgs<float> bz_args(const BGrid& G, char* ws) {
  ZArgs<float> z{};
  z.data = reinterpret_cast<float*>(ws + G.ws_off + G.off_w);
  z.scr_c = reinterpret_cast<float*>(ws + G.ws_off + G.off_scr);
  z.scr_u = G.periodic_z ? reinterpret_cast<float*>(ws + G.ws_off + G.off_scru) : nullptr;
  z.nx = G.nx; z.ny = G.ny; z.nz = G.nz;
  z.lamx = G.lamx; z.lamy = G.lamy;
  z.za = G.za; z.zb = G.zb; z.zc = G.zc; z.dzf = G.dzf;
  z.periodic = G.periodic_z;
  z.singular = G.singular;
  z.skip = nullptr;
  return z;
}

enum { BEND_WRAP = 0, BEND_N = 1, BEND_D = 2 };
__device__ __forceinline__ int bend_lo(int bc) {
  return bc == BC_P ? BEND_WRAP : ((bc == BC_DD || bc == BC_DN || bc == BC_FD) ? BEND_D : BEND_N);
}
__device__ __forceinline__ int bend_hi(int bc) {
  return bc == BC_P ? BEND_WRAP : ((bc == BC_DD || bc == BC_ND || bc == BC_FD) ? BEND_D : BEND_N);
}
// (neighbour − Φ_c) under the end's ghost rule; q is the neighbour if inner or wrapped
__device__ __forceinline__ df bnb(int kind, bool inner, const double* q, df pc) {
  if (inner || kind == BEND_WRAP) return df_sub(df_from_f64(*q), pc);
  if (kind == BEND_N) return df{0.f, 0.f};
  return df{-2.f * pc.h, -2.f * pc.l};
}

// One residual tile: points [t·chunk, (t+1)·chunk) of grid G, r = (f − μ) − A·Φ in
// double-float, FP32 r written (unless check), reductions into the grid's words.
__device__ void residual_tile(const BGrid& G, const double* f, const double* p, float* r, Ctrl* c,
                              float* partial, int t, bool first) {
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const size_t N = (size_t)nx * ny * nz, sxy = (size_t)nx * ny;
  const size_t g0 = (size_t)t * G.res_chunk, g1 = min(N, g0 + G.res_chunk);
  const int xl = bend_lo(G.bcx), xh = bend_hi(G.bcx), yl = bend_lo(G.bcy), yh = bend_hi(G.bcy);
  const int zl = bend_lo(G.bcz), zh = bend_hi(G.bcz);
  const df mu = G.singular ? df{c->mu[0], c->mu[1]} : df{0.f, 0.f};
  float rmax = -INFINITY, rmin = INFINITY, fmx = -INFINITY, fmn = INFINITY;
  df wr = {0.f, 0.f}, wf = {0.f, 0.f};
  for (size_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const int i = (int)(g % nx);
    const size_t tt = g / nx;
    const int j = (int)(tt % ny), k = (int)(tt / ny);
    const double* pp = p + g;
    const df pc = df_from_f64(*pp);
    const df dxm = bnb(xl, i > 0, (i > 0) ? pp - 1 : pp + (nx - 1), pc);
    const df dxp = bnb(xh, i < nx - 1, (i < nx - 1) ? pp + 1 : pp - (nx - 1), pc);
    const df dym = bnb(yl, j > 0, (j > 0) ? pp - nx : pp + (size_t)(ny - 1) * nx, pc);
    const df dyp = bnb(yh, j < ny - 1, (j < ny - 1) ? pp + nx : pp - (size_t)(ny - 1) * nx, pc);
    const df dzm = bnb(zl, k > 0, (k > 0) ? pp - sxy : pp + (size_t)(nz - 1) * sxy, pc);
    const df dzp = bnb(zh, k < nz - 1, (k < nz - 1) ? pp + sxy : pp - (size_t)(nz - 1) * sxy, pc);
    const float2 cl = G.zlo[k], ch = G.zhi[k];
    df ap = df_add(df_add(df_mul(df_add(dxm, dxp), G.idx2), df_mul(df_add(dym, dyp), G.idy2)),
                   df_add(df_mul(dzm, df{cl.x, cl.y}), df_mul(dzp, df{ch.x, ch.y})));
    if (G.shift) ap = df_add(ap, df_mul(pc, G.nalpha));
    const df fv = df_from_f64(f[g]);
    const df rv = df_sub(G.singular ? df_sub(fv, mu) : fv, ap);
    const float rf = df_to_f32(rv), ff = df_to_f32(fv);
    if (r) r[g] = rf;
    rmax = fmaxf(rmax, rf); rmin = fminf(rmin, rf);
    fmx = fmaxf(fmx, ff); fmn = fminf(fmn, ff);
    if (G.singular) {
      const df w = {G.dzf[k], 0.f};
      wr = df_add(wr, df_mul(rv, w));
      if (first) wf = df_add(wf, df_mul(fv, w));
    }
  }
  __shared__ float sred[8][8];
  for (int o = 16; o > 0; o >>= 1) {
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    fmx = fmaxf(fmx, __shfl_xor_sync(0xffffffffu, fmx, o));
    fmn = fminf(fmn, __shfl_xor_sync(0xffffffffu, fmn, o));
    wr = df_add(wr, df{__shfl_xor_sync(0xffffffffu, wr.h, o), __shfl_xor_sync(0xffffffffu, wr.l, o)});
    wf = df_add(wf, df{__shfl_xor_sync(0xffffffffu, wf.h, o), __shfl_xor_sync(0xffffffffu, wf.l, o)});
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sred[wid][0] = rmax; sred[wid][1] = rmin; sred[wid][2] = fmx; sred[wid][3] = fmn;
    sred[wid][4] = wr.h; sred[wid][5] = wr.l; sred[wid][6] = wf.h; sred[wid][7] = wf.l;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      rmax = fmaxf(rmax, sred[w][0]); rmin = fminf(rmin, sred[w][1]);
      fmx = fmaxf(fmx, sred[w][2]); fmn = fminf(fmn, sred[w][3]);
      wr = df_add(wr, df{sred[w][4], sred[w][5]});
      wf = df_add(wf, df{sred[w][6], sred[w][7]});
    }
    atomicMax(&c->red[0], f32_key(rmax));
    atomicMin(&c->red[1], f32_key(rmin));
    atomicMax(&c->red[2], f32_key(fmx));
    atomicMin(&c->red[3], f32_key(fmn));
    reinterpret_cast<float4*>(partial)[t] = make_float4(wr.h, wr.l, wf.h, wf.l);
  }
}

__device__ void reset_red(Ctrl* c) {
  c->red[0] = f32_key(-INFINITY);
  c->red[1] = f32_key(INFINITY);
  c->red[2] = f32_key(-INFINITY);
  c->red[3] = f32_key(INFINITY);
}

// Convergence test of one grid (one CTA).
__device__ void finalize_grid(const BGrid& G, Ctrl* c, const float* partial, double rtol, int it,
                              bool last, ps_info* info) {
  __shared__ df s1[32], s2[32];
  df ar = {0.f, 0.f}, af = {0.f, 0.f};
  if (G.singular) {
    const float4* pv = reinterpret_cast<const float4*>(partial);
    for (int b = threadIdx.x; b < G.ntask[3]; b += blockDim.x) {
      const float4 v = pv[b];
      ar = df_add(ar, df{v.x, v.y});
      af = df_add(af, df{v.z, v.w});
    }
    for (int o = 16; o > 0; o >>= 1) {
      ar = df_add(ar, df{__shfl_xor_sync(0xffffffffu, ar.h, o), __shfl_xor_sync(0xffffffffu, ar.l, o)});
      af = df_add(af, df{__shfl_xor_sync(0xffffffffu, af.h, o), __shfl_xor_sync(0xffffffffu, af.l, o)});
    }
    if ((threadIdx.x & 31) == 0) { s1[threadIdx.x >> 5] = ar; s2[threadIdx.x >> 5] = af; }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double mr = 0.0, mf = 0.0;
  if (G.singular) {
    double a1 = 0.0, a2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a1 += (double)s1[w].h + (double)s1[w].l;
      a2 += (double)s2[w].h + (double)s2[w].l;
    }
    mr = a1 / G.wsum_total;
    if (it == 0) {
      mf = a2 / G.wsum_total;
      c->mf = mf;
      const float h = (float)mf;
      c->mu[0] = h;
      c->mu[1] = (float)(mf - (double)h);
    } else {
      mf = c->mf;
    }
  }
  const double rmax = key_f32(c->red[0]), rmin = key_f32(c->red[1]);
  const double vmax = key_f32(c->red[2]), vmin = key_f32(c->red[3]);
  const double rn = fmax(rmax - mr, mr - rmin), fn = fmax(vmax - mf, mf - vmin);
  const double rel = fn > 0 ? rn / fn : (rn > 0 ? INFINITY : 0.0);
  c->rel = rel; c->rnorm = rn; c->fnorm = fn; c->iterations = it;
  const bool ok = rel <= rtol;
  if (ok || last) {
    c->status = ok ? PS_OK : PS_NOT_CONVERGED;
    if (info) {
      info->status = c->status; info->iterations = it; info->rel_residual = rel;
      info->r_norm = rn; info->f_norm = fn;
    }
  }
  reset_red(c);
  __threadfence();
  if (ok) c->converged = 1;
}

__global__ void __launch_bounds__(256, 4) batch_kernel(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_task, s_run;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(A.next, 1);
    __syncthreads();
    const int t = s_task;
    if (t >= A.ntasks) break;
    const int4 tk = A.tasks[t];
    const int g = tk.x, s = tk.y, idx = tk.z;
    const BGrid& G = A.grids[g];
    Ctrl* c = A.ctrl + g;
    if (threadIdx.x == 0) {
      bool ok = true;
      const int d = A.dep[g * A.nstage + s];
      if (d >= 0) {
        const int need = A.need[g * A.nstage + d] + ((A.inject && g == 0 && s == d + 1) ? 1 : 0);
        const unsigned long long t0 = gtimer();
        while (ld_acquire(&A.done[g * A.nstage + d]) < need) {
          if (ld_acquire(A.abort)) { ok = false; break; }
          if (gtimer() - t0 > A.wait_ns) {  // bounded wait: give up, report, let every task drain
            atomicExch(A.abort, 1);
            ok = false;
            break;
          }
          __nanosleep(256);
        }
      }
      __threadfence();
      s_run = ok && !ld_acquire(A.abort) && !ld_acquire(&c->converged);
    }
    __syncthreads();
    __threadfence();  // every thread orders its task reads after the acquire above
    if (s_run) {
      const int type = A.stage_type[s];
      char* ws = A.ws;
      float* w = reinterpret_cast<float*>(ws + G.ws_off + G.off_w);
      float* partial = reinterpret_cast<float*>(ws + G.ws_off);
      switch (type) {
        case BS_XF64:
          xform_group<float, double, float, true>(bx_args(G, 0, A.f[g], w, 0, nullptr), idx, smem);
          break;
        case BS_XF:
          xform_group<float, float, float, true>(bx_args(G, 0, w, w, 0, nullptr), idx, smem);
          break;
        case BS_YF:
          xform_group<float, float, float, true>(bx_args(G, 1, w, w, 0, nullptr), idx, smem);
          break;
        case BS_Z:
          zsolve_column<float>(bz_args(G, ws), idx * blockDim.x + threadIdx.x);
          break;
        case BS_ZS:
          zsingular_block<float>(bz_args(G, ws), smem);
          break;
        case BS_YB:
          xform_group<float, float, float, false>(bx_args(G, 1, w, w, 0, nullptr), idx, smem);
          break;
        case BS_XBST:
          if (idx == 0 && threadIdx.x == 0) reset_red(c);
          xform_group<float, float, double, false>(bx_args(G, 0, w, A.p[g], 0, nullptr), idx, smem);
          break;
        case BS_XBACC:
          xform_group<float, float, double, false>(bx_args(G, 0, w, A.p[g], 1, nullptr), idx, smem);
          break;
        case BS_RES:
        case BS_CHK:
          residual_tile(G, A.f[g], A.p[g], type == BS_RES ? w : nullptr, c, partial, idx,
                        A.stage_it[s] == 0);
          break;
        default:  // BS_FIN
          finalize_grid(G, c, partial, A.rtol, A.stage_it[s], A.stage_it[s] == A.max_iter,
                        A.infos ? A.infos + g : nullptr);
          break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&A.done[g * A.nstage + s], 1);
    }
  }
}

// Per-grid record after the persistent kernel: a timed-out batch reports
// PS_TIMEOUT for every grid that had not converged.
__global__ void batch_record_kernel(const int* abort, Ctrl* ctrl, ps_info* infos, int count) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count || !infos) return;
  if (*abort && !ctrl[g].converged) {
    infos[g].status = PS_TIMEOUT;
    infos[g].iterations = ctrl[g].iterations;
    infos[g].rel_residual = ctrl[g].rel;
    infos[g].r_norm = ctrl[g].rnorm;
    infos[g].f_norm = ctrl[g].fnorm;
  }
}

}  // namespace ps

using namespace ps;

struct ps_batch {
  int count = 0;
  ps_precision prec = PS_FP32_REFINE;
  double rtol = 1e-10;
  int max_iter = 3;
  std::vector<ps_plan*> plans;
  std::vector<ps_grid_desc> descs;
  std::vector<std::vector<double>> faces;  // each grid's z faces (empty: uniform dz)
  std::vector<double> alphas;              // each grid's Helmholtz shift
  int nstage = 0, ntasks = 0;
  void* dev = nullptr;         // grids, tasks, need, dep, stage tables
  BGrid* d_grids = nullptr;
  int4* d_tasks = nullptr;
  int *d_need = nullptr, *d_dep = nullptr, *d_stype = nullptr, *d_sit = nullptr;
  size_t head_bytes = 0, ws_bytes = 0;
  size_t smem = 0;
  int blocks = 0;
  int scale = 2;               // tile scale (autotuned)
  double wait_s = 2.0;
  int inject = 0;
  char err[256] = "";
};

namespace {

thread_local char g_batch_err[256] = "";

ps_status bfail(ps_batch* b, ps_status st, const char* msg) {
  snprintf(b ? b->err : g_batch_err, 256, "%s", msg);
  return st;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Tile scales the autotuner times (and the only ones a cache entry may name).
constexpr int kScales[] = {1, 2, 4, 8, 16, 32, 64};
constexpr int kNumScales = (int)(sizeof(kScales) / sizeof(kScales[0]));
bool is_candidate_scale(int sc) {
  for (int i = 0; i < kNumScales; ++i)
    if (kScales[i] == sc) return true;
  return false;
}

// Build the device tables for the current tile scale.
ps_status build_tables(ps_batch* b) {
  if (b->dev) {
    cudaFree(b->dev);
    b->dev = nullptr;
  }
  const int G = b->count;
  // stage list (same for every grid)
  std::vector<int> stype, sit;
  auto add = [&](int t, int it) { stype.push_back(t); sit.push_back(it); };
  add(BS_XF64, 0); add(BS_YF, 0); add(BS_Z, 0); add(BS_ZS, 0); add(BS_YB, 0); add(BS_XBST, 0);
  for (int it = 0; it <= b->max_iter; ++it) {
    add(it == b->max_iter ? BS_CHK : BS_RES, it);
    add(BS_FIN, it);
    if (it < b->max_iter) {
      add(BS_XF, it); add(BS_YF, it); add(BS_Z, it); add(BS_ZS, it); add(BS_YB, it); add(BS_XBACC, it);
    }
  }
  const int S = (int)stype.size();
  b->nstage = S;
  std::vector<BGrid> grids(G);
  std::vector<int> need((size_t)G * S, 0), dep((size_t)G * S, -1);
  size_t ws_off = a256(sizeof(int) * 4 + sizeof(int) * (size_t)G * S) + a256(sizeof(Ctrl) * (size_t)G);
  b->head_bytes = ws_off;
  size_t smem = 0;
  for (int g = 0; g < G; ++g) {
    ps_plan* pl = b->plans[g];
    const ps_grid_desc& d = b->descs[g];
    BGrid& B = grids[g];
    memset(&B, 0, sizeof(B));
    B.nx = d.nx; B.ny = d.ny; B.nz = d.nz;
    B.bcx = d.bcx; B.bcy = d.bcy; B.bcz = d.bcz;
    auto pn = [](int v) { return v == PS_BC_PERIODIC || v == PS_BC_NEUMANN_NEUMANN; };
    const double alpha = ps_plan_internal_alpha(pl);  // its z tables carry the shift already
    B.shift = alpha != 0.0;
    B.nalpha = df{(float)(-alpha), (float)(-alpha - (double)(float)(-alpha))};
    B.singular = pn(d.bcx) && pn(d.bcy) && pn(d.bcz) && !B.shift;
    B.periodic_z = d.bcz == PS_BC_PERIODIC;
    ps_plan_internal_tables(pl, &B.twx, &B.twy, &B.lamx, &B.lamy, &B.za, &B.zb, &B.zc, &B.dzf, &B.zlo,
                            &B.zhi, &B.idx2, &B.idy2, &B.wsum_total, B.radx, B.rady, &B.nstx, &B.nsty);
    B.mx = d.nx / 2;
    B.my = d.ny / 2;
    const size_t N = (size_t)d.nx * d.ny * d.nz;
    // tiles: lines per task within 48 KB of shared memory, scaled by the tuned factor
    auto lines_for = [&](int m, int axis) {
      int L = 4 * b->scale;
      const int cap = (int)(48 * 1024 / (2 * (size_t)(m + 1) * sizeof(cplx<float>)));
      L = std::max(1, std::min(L, cap));
      if (axis == 1) while (L > 1 && d.nx % L) --L;
      return L;
    };
    B.Lx = lines_for(B.mx, 0);
    B.Ly = lines_for(B.my, 1);
    B.res_chunk = 2048 * b->scale;
    B.ntask[0] = (d.ny * d.nz + B.Lx - 1) / B.Lx;
    B.ntask[1] = d.nz * (d.nx / B.Ly);
    B.ntask[2] = (d.nx * d.ny + 255) / 256;
    B.ntask[3] = (int)((N + B.res_chunk - 1) / B.res_chunk);
    smem = std::max(smem, 2 * (size_t)B.Lx * (B.mx + 1) * sizeof(cplx<float>));
    smem = std::max(smem, 2 * (size_t)B.Ly * (B.my + 1) * sizeof(cplx<float>));
    smem = std::max(smem, 2 * (size_t)d.nz * sizeof(float));
    // workspace slice: partials | w | scr | scr_u
    B.ws_off = ws_off;
    size_t o = a256((N + 2047) / 2048 * 4 * sizeof(float));  // partials for the finest tiling
    B.off_w = o;
    o += a256(N * sizeof(float));
    B.off_scr = o;
    o += a256(N * sizeof(float));
    B.off_scru = o;
    if (B.periodic_z) o += a256(N * sizeof(float));
    ws_off += o;
    for (int s = 0; s < S; ++s) {
      int n = 0;
      switch (stype[s]) {
        case BS_XF64: case BS_XF: case BS_XBST: case BS_XBACC: n = B.ntask[0]; break;
        case BS_YF: case BS_YB: n = B.ntask[1]; break;
        case BS_Z: n = B.ntask[2]; break;
        case BS_ZS: n = B.singular ? 1 : 0; break;
        case BS_RES: case BS_CHK: n = B.ntask[3]; break;
        default: n = 1; break;
      }
      need[(size_t)g * S + s] = n;
    }
    int last = -1;
    for (int s = 0; s < S; ++s) {
      dep[(size_t)g * S + s] = last;
      if (need[(size_t)g * S + s] > 0) last = s;
    }
  }
  b->ws_bytes = ws_off;
  b->smem = smem;
  // task table, stage-major
  std::vector<int4> tasks;
  for (int s = 0; s < S; ++s)
    for (int g = 0; g < G; ++g)
      for (int t = 0; t < need[(size_t)g * S + s]; ++t) tasks.push_back(make_int4(g, s, t, 0));
  b->ntasks = (int)tasks.size();
  const size_t bytes = a256(sizeof(BGrid) * G) + a256(sizeof(int4) * tasks.size()) +
                       2 * a256(sizeof(int) * (size_t)G * S) + 2 * a256(sizeof(int) * S);
  char* dev = nullptr;
  cudaError_t e = take_injected_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&dev, bytes);
  if (e != cudaSuccess) return bfail(b, PS_OUT_OF_MEMORY, "cudaMalloc of batch tables failed");
  b->dev = dev;
  size_t off = 0;
  auto put = [&](const void* src, size_t n) {
    char* dst = dev + off;
    off += a256(n);
    return cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice) == cudaSuccess ? dst : nullptr;
  };
  b->d_grids = reinterpret_cast<BGrid*>(put(grids.data(), sizeof(BGrid) * G));
  b->d_tasks = reinterpret_cast<int4*>(put(tasks.data(), sizeof(int4) * tasks.size()));
  b->d_need = reinterpret_cast<int*>(put(need.data(), sizeof(int) * need.size()));
  b->d_dep = reinterpret_cast<int*>(put(dep.data(), sizeof(int) * dep.size()));
  b->d_stype = reinterpret_cast<int*>(put(stype.data(), sizeof(int) * S));
  b->d_sit = reinterpret_cast<int*>(put(sit.data(), sizeof(int) * S));
  if (!b->d_grids || !b->d_tasks || !b->d_need || !b->d_dep || !b->d_stype || !b->d_sit)
    return bfail(b, PS_CUDA_ERROR, "copy of batch tables failed");
  if (b->smem > 200 * 1024) return bfail(b, PS_UNSUPPORTED_SIZE, "batch grids too large for one CTA's tiles");
  e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  if (e != cudaSuccess) return bfail(b, PS_CUDA_ERROR, "cudaFuncSetAttribute (batch kernel)");
  int bps = 0, dev_id = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_kernel, 256, b->smem);
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
  b->blocks = std::max(1, bps) * sms;  // every CTA resident: waits can always be met
  return PS_OK;
}

}  // namespace

extern "C" {

ps_status ps_batch_create(ps_batch** out, int count, const ps_grid_desc* descs, ps_precision prec,
                          double rtol, int max_iter) {
  return ps_batch_create_helmholtz(out, count, descs, prec, rtol, max_iter, nullptr);
}

ps_status ps_batch_create_helmholtz(ps_batch** out, int count, const ps_grid_desc* descs, ps_precision prec,
                                    double rtol, int max_iter, const double* alphas) {
  if (!out) return bfail(nullptr, PS_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (count < 1 || count > 4096 || !descs) return bfail(nullptr, PS_INVALID_ARG, "count must be 1..4096");
  if (prec != PS_FP32_REFINE) return bfail(nullptr, PS_INVALID_ARG, "the batched solve runs PS_FP32_REFINE");
  if (!(rtol > 0) || max_iter < 0 || max_iter > 16)
    return bfail(nullptr, PS_INVALID_ARG, "needs rtol > 0 and 0 <= max_iter <= 16");
  ps_batch* b = new (std::nothrow) ps_batch();
  if (!b) return bfail(nullptr, PS_OUT_OF_MEMORY, "host allocation failed");
  b->count = count;
  b->rtol = rtol;
  b->max_iter = max_iter;
  b->descs.assign(descs, descs + count);
  b->faces.resize(count);
  b->alphas.assign(count, 0.0);
  for (int g = 0; g < count; ++g) {
    const ps_grid_desc& d = descs[g];
    if (d.bcx == PS_BC_FACE_DIRICHLET || d.bcy == PS_BC_FACE_DIRICHLET) {
      char msg[128];
      snprintf(msg, sizeof(msg), "grid %d: face-centred x or y unknowns are not supported by the batched solve", g);
      ps_batch_destroy(b);
      return bfail(nullptr, PS_INVALID_ARG, msg);
    }
    if (d.zf) b->faces[g].assign(d.zf, d.zf + (d.nz > 0 ? d.nz + 1 : 0));  // host copy: autotune cache key
    if (alphas) b->alphas[g] = alphas[g];
    ps_plan* pl = nullptr;
    ps_status st = ps_plan_create_helmholtz(&pl, d.nx, d.ny, d.nz, d.dx, d.dy, d.zf, d.dz, d.bcx, d.bcy,
                                            d.bcz, PS_FP32_REFINE, rtol, max_iter, alphas ? alphas[g] : 0.0);
    if (st != PS_OK) {
      char msg[256];
      snprintf(msg, sizeof(msg), "grid %d: %s", g, ps_last_error(nullptr));
      ps_batch_destroy(b);
      return bfail(nullptr, st, msg);
    }
    b->plans.push_back(pl);
    b->descs[g].zf = nullptr;  // the plan keeps its own copy of the faces
  }
  ps_status st = build_tables(b);
  if (st != PS_OK) {
    snprintf(g_batch_err, sizeof(g_batch_err), "%s", b->err);
    ps_batch_destroy(b);
    return st;
  }
  *out = b;
  return PS_OK;
}

ps_status ps_batch_workspace_bytes(const ps_batch* b, size_t* bytes) {
  if (!b || !bytes) return bfail(nullptr, PS_INVALID_ARG, "null argument");
  *bytes = b->ws_bytes;
  return PS_OK;
}

ps_status ps_batch_solve(ps_batch* b, double* const* f_dev, double* const* p_dev, void* ws, void* stream,
                         ps_info* infos) {
  if (!b || !f_dev || !p_dev || !ws) return bfail(b, PS_INVALID_ARG, "null argument");
  if (((uintptr_t)ws) & 255) return bfail(b, PS_INVALID_ARG, "workspace must be 256-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  // head: next, abort, pad | done[grid][stage] | ctrl[grid]
  cudaError_t e = cudaMemsetAsync(w, 0, b->head_bytes, st);
  if (e != cudaSuccess) return bfail(b, PS_CUDA_ERROR, "cudaMemsetAsync (batch head)");
  BatchArgs A{};
  A.grids = b->d_grids;
  A.tasks = b->d_tasks;
  A.ntasks = b->ntasks;
  A.nstage = b->nstage;
  A.need = b->d_need;
  A.dep = b->d_dep;
  A.stage_type = b->d_stype;
  A.stage_it = b->d_sit;
  A.next = reinterpret_cast<int*>(w);
  A.abort = reinterpret_cast<int*>(w) + 1;
  A.done = reinterpret_cast<int*>(w) + 4;
  A.ctrl = reinterpret_cast<Ctrl*>(w + a256(sizeof(int) * 4 + sizeof(int) * (size_t)b->count * b->nstage));
  A.ws = w;
  A.f = f_dev;
  A.p = p_dev;
  A.infos = infos;
  A.rtol = b->rtol;
  A.max_iter = b->max_iter;
  A.wait_ns = (unsigned long long)(b->wait_s * 1e9);
  A.inject = b->inject;
  batch_kernel<<<b->blocks, 256, b->smem, st>>>(A);
  if ((e = cudaGetLastError()) != cudaSuccess) return bfail(b, PS_CUDA_ERROR, cudaGetErrorString(e));
  batch_record_kernel<<<(b->count + 127) / 128, 128, 0, st>>>(A.abort, A.ctrl, infos, b->count);
  if ((e = cudaGetLastError()) != cudaSuccess) return bfail(b, PS_CUDA_ERROR, cudaGetErrorString(e));
  return PS_OK;
}

ps_status ps_batch_autotune(ps_batch* b, double* const* f_dev, double* const* p_dev, void* ws, void* stream,
                            double* best_ms) {
  if (!b || !f_dev || !p_dev || !ws) return bfail(b, PS_INVALID_ARG, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // cache: PS_AUTOTUNE_CACHE names a JSON-lines file of {"key": ..., "scale": ..., "ms": ...}
  char dev_name[256] = "";
  {
    int d = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&d) == cudaSuccess && cudaGetDeviceProperties(&prop, d) == cudaSuccess)
      snprintf(dev_name, sizeof(dev_name), "%s", prop.name);
  }
  unsigned long long h = 1469598103934665603ull;  // FNV-1a over the grid descriptions
  auto mix = [&](const void* data, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
  };
  for (int g = 0; g < b->count; ++g) {
    // everything that decides a grid's work: sizes, BCs, spacings, z faces, shift
    const ps_grid_desc& d = b->descs[g];
    int ints[6] = {d.nx, d.ny, d.nz, (int)d.bcx, (int)d.bcy, (int)d.bcz};
    mix(ints, sizeof(ints));
    const double dbl[4] = {d.dx, d.dy, b->faces[g].empty() ? d.dz : 0.0, b->alphas[g]};
    mix(dbl, sizeof(dbl));
    if (!b->faces[g].empty()) mix(b->faces[g].data(), b->faces[g].size() * sizeof(double));
  }
  mix(&b->max_iter, sizeof(int));
  mix(&b->rtol, sizeof(double));
  mix(dev_name, strlen(dev_name));
  char key[64];
  snprintf(key, sizeof(key), "%016llx", h);
  const char* cache = getenv("PS_AUTOTUNE_CACHE");
  if (cache) {
    FILE* fp = fopen(cache, "r");
    if (fp) {
      char line[512];
      while (fgets(line, sizeof(line), fp)) {
        char k[64];
        int sc;
        double ms;
        if (sscanf(line, "{\"key\": \"%63[^\"]\", \"scale\": %d, \"ms\": %lf", k, &sc, &ms) == 3 &&
            strcmp(k, key) == 0 && is_candidate_scale(sc)) {
          fclose(fp);
          b->scale = sc;
          if (best_ms) *best_ms = ms;
          return build_tables(b);
        }
      }
      fclose(fp);
    }
  }
  double best = 1e300;
  int best_scale = b->scale;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int ci = 0; ci < kNumScales; ++ci) {
    b->scale = kScales[ci];
    ps_status s2 = build_tables(b);
    if (s2 != PS_OK) continue;
    ps_batch_solve(b, f_dev, p_dev, ws, stream, nullptr);  // warm
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) ps_batch_solve(b, f_dev, p_dev, ws, stream, nullptr);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / 3 < best) {
      best = ms / 3;
      best_scale = kScales[ci];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->scale = best_scale;
  ps_status s3 = build_tables(b);
  if (s3 != PS_OK) return s3;
  if (best_ms) *best_ms = best;
  if (cache) {
    FILE* fp = fopen(cache, "a");
    if (fp) {
      fprintf(fp, "{\"key\": \"%s\", \"scale\": %d, \"ms\": %.6f, \"device\": \"%s\"}\n", key,
              best_scale, best, dev_name);
      fclose(fp);
    }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PS_OK : bfail(b, PS_CUDA_ERROR, cudaGetErrorString(e));
}

int ps_batch_tile_scale(const ps_batch* b) { return b ? b->scale : 0; }

ps_status ps_batch_configure(ps_batch* b, double wait_limit_seconds, int flags) {
  if (!b || !(wait_limit_seconds > 0)) return bfail(b, PS_INVALID_ARG, "needs a batch and a positive wait limit");
  b->wait_s = wait_limit_seconds;
  b->inject = (flags & 1) ? 1 : 0;
  return PS_OK;
}

ps_status ps_batch_destroy(ps_batch* b) {
  if (!b) return PS_OK;
  for (ps_plan* p : b->plans) ps_plan_destroy(p);
  if (b->dev) cudaFree(b->dev);
  delete b;
  return PS_OK;
}

const char* ps_batch_last_error(const ps_batch* b) { return b ? b->err : g_batch_err; }

}  // extern "C"
