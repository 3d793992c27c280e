/*
 * ps_poisson.h — C ABI of the GB300 eigenfunction-expansion Poisson solver.
 *
 * The operation (Costa 2018, §2.1, Eq. 4): solve the second-order 7-point
 * finite-difference Poisson equation  A·Φ = f  on a cell-centred grid of
 * n_x × n_y × n_z cells, uniform in x and y, possibly stretched in z (footnote
 * to Eq. 5), with a homogeneous staggered boundary-condition pair per axis
 * (Table 1). The method: forward real-to-real transform along x, then y
 * (Table 2), one tridiagonal solve along z per wavenumber pair (Eq. 5), and the
 * inverse transforms (the three steps that close §2.1).
 *
 * Layout of every field: C order [n_z][n_y][n_x], x contiguous, one value per
 * cell centre. All field pointers passed to ps_solve* are DEVICE pointers owned
 * by the caller; plans own their tables. Every call returns a ps_status; no
 * exception or abort crosses this boundary. ps_last_error() gives a static
 * description of the last failure on a plan (or of the last failed create).
 *
 * Singular problems (every axis periodic or Neumann–Neumann, so constants are
 * in the null space): the solve returns the Φ that satisfies A·Φ = f_c, with
 * f_c = f minus its volume-weighted mean, and whose volume-weighted mean is 0.
 *
 * Streams are passed as `void*` holding a cudaStream_t (NULL = legacy default
 * stream). Solves only enqueue work on that stream: no host synchronisation,
 * no allocation. Results, including the ps_info record, are valid after the
 * stream has been synchronised.
 */
#ifndef PS_POISSON_H
#define PS_POISSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PS_OK = 0,
  PS_INVALID_ARG = 1,        /* null pointer, bad spacing, inconsistent sizes   */
  PS_UNSUPPORTED_SIZE = 2,   /* n odd, n < 2, n > 8192, or n/2 not 2^a·3^b     */
  PS_CUDA_ERROR = 3,         /* a CUDA runtime call failed (see ps_last_error)  */
  PS_OUT_OF_MEMORY = 4,      /* cudaMalloc of plan tables failed                */
  PS_NOT_CONVERGED = 5,      /* refinement did not reach rtol in max_iter       */
  PS_TIMEOUT = 6             /* a bounded device wait gave up (batched solve)   */
} ps_status;

/* Per-axis boundary-condition pair, Table 1 (staggered: the boundary is a
 * cell face). NEUMANN_DIRICHLET is Neumann at the low end, Dirichlet at the
 * high end. Forward transforms per Table 2: DFT (half-complex layout),
 * DCT-II, DST-II, DCT-IV; backward: 1/n IDFT, 1/(2n) DCT-III, 1/(2n) DST-III,
 * 1/(2n) DCT-IV. DIRICHLET_NEUMANN (not in Table 1) is the reverse pair,
 * solved as NEUMANN_DIRICHLET on the reversed axis: its transforms are the
 * DCT-IV ones applied to the reversed line (forward: (−1)^q times a DST-IV)
 * and its eigenvalues are NEUMANN_DIRICHLET's. */
typedef enum {
  PS_BC_PERIODIC = 0,
  PS_BC_NEUMANN_NEUMANN = 1,
  PS_BC_DIRICHLET_DIRICHLET = 2,
  PS_BC_NEUMANN_DIRICHLET = 3,
  PS_BC_DIRICHLET_NEUMANN = 4,
  PS_BC_FACE_DIRICHLET = 5   /* face unknowns between two walls: see below */
} ps_bc;
/* PS_BC_FACE_DIRICHLET (the wall-normal velocity of an implicit diffusion step,
 * §2; non-staggered unknowns, end of §2.1): the unknowns sit on the faces normal
 * to the axis, entry i of a line being face i (the low face of cell i); entry 0
 * is the low wall face and the high wall face n is implicit, both with value 0
 * (Dirichlet on the node). The caller keeps f zero on the wall faces, and the
 * solution is then zero there.
 *   z: row k ≥ 1 is the finite-volume second difference over the volume between
 *      the centres of cells k−1 and k; row 0 is −p_0 plus the x/y terms. No
 *      transpose solve (the operator is not symmetric under the Δz^f weight).
 *   x, y (uniform; n ≤ 4096): rows i ≥ 1 are the second difference between the
 *      wall nodes of value 0, row 0 has the axis part −p_0/Δ²; transformed by a
 *      DST-I of the interior faces with the wall entry copied (eigenvalues −1 and
 *      −4 sin²(πk/2n), divided by Δ²), done as an FFT of n complex points of the
 *      odd extension in the shared-memory transform kernel. Not with the batched
 *      solve, the projection operators or ps_ns_substep.
 * Not singular. */

/* Arithmetic of the solve.
 *   PS_FP64         all of the path in FP64 arithmetic (fields double).
 *   PS_FP32         all of the path in FP32 arithmetic (fields float).
 *   PS_FP32_REFINE  FP64 fields; FP32 bulk transforms and tridiagonal solves,
 *                   iterative refinement whose residual r = f − A·Φ is formed
 *                   in double-float (pairs of FP32) from the FP64 fields, until
 *                   ‖r‖∞ ≤ rtol·‖f_c‖∞ or max_iter corrections. */
typedef enum { PS_FP64 = 0, PS_FP32 = 1, PS_FP32_REFINE = 2 } ps_precision;

/* Device-side record written by every solve (caller allocates it in device
 * memory; read it after synchronising the stream). */
typedef struct {
  int status;             /* ps_status of the device work (OK, NOT_CONVERGED, TIMEOUT) */
  int iterations;         /* refinement corrections applied (0 for FP64 / FP32)        */
  double rel_residual;    /* ‖f_c − A·Φ‖∞ / ‖f_c‖∞ measured on the device (refine);   */
                          /* −1 when not measured (FP64 / FP32 modes)                  */
  double r_norm;          /* ‖f_c − A·Φ‖∞ (refine), else −1                            */
  double f_norm;          /* ‖f_c‖∞ (refine), else −1                                  */
} ps_info;

typedef struct ps_plan ps_plan;
typedef struct ps_batch ps_batch;

/* Create a plan (§2.1; Table 1 eigenvalues λ_q = −4 sin²θ_q / Δ² and the
 * Table 2 twiddles are computed here in FP64, cast once for FP32 paths; the
 * z coefficients follow the finite-volume form of Eq. 4 on the faces zf).
 *   nx, ny       cells along x and y; each even, 2 ≤ n ≤ 8192, n/2 = 2^a·3^b
 *                (lines of n ≤ 1024 run in register-resident transform kernels,
 *                longer ones one line per CTA in shared memory).
 *   nz           cells along z, 2 ≤ nz ≤ 8192.
 *   dx, dy       uniform spacings (> 0).
 *   zf           host array of nz+1 increasing face coordinates, or NULL for a
 *                uniform z of spacing dz (> 0). Copied; the caller keeps it.
 *   bcx,bcy,bcz  boundary pairs (Table 1).
 *   prec         arithmetic (see ps_precision).
 *   rtol         refinement target on ‖r‖∞/‖f_c‖∞ (PS_FP32_REFINE only).
 *   max_iter     maximum refinement corrections (PS_FP32_REFINE only, ≥ 0).
 * Allocates the plan's device tables on the current device. On failure *out is
 * NULL and the status says why. */
ps_status ps_plan_create(ps_plan** out, int nx, int ny, int nz, double dx, double dy,
                         const double* zf, double dz, ps_bc bcx, ps_bc bcy, ps_bc bcz,
                         ps_precision prec, double rtol, int max_iter);

/* Helmholtz variant (§2: integrating the diffusion term implicitly needs one
 * Helmholtz equation per velocity component; §4 reports it done with the same
 * method). The plan solves (A − α·I)·p = f, A the operator of Eq. 4, with a
 * shift α ≥ 0 (a Crank–Nicolson step of ∂u/∂t = ν∇²u has α = 2/(ν·Δt)). The
 * transforms of Table 2 diagonalise the identity too, so only the diagonal of
 * every z system of Eq. 5 moves by −α. Arguments and results as
 * ps_plan_create, which is this call with α = 0; every solve entry point takes
 * the plan (ps_solve_transpose applies (A − α·I)⁻ᵀ). With α > 0 no problem is
 * singular: f is used as given and p carries no mean constraint. The boundary
 * pairs are the staggered ones of Table 1 (cell-centred unknowns).
 * PS_INVALID_ARG when α is negative or not finite. */
ps_status ps_plan_create_helmholtz(ps_plan** out, int nx, int ny, int nz, double dx, double dy,
                                   const double* zf, double dz, ps_bc bcx, ps_bc bcy, ps_bc bcz,
                                   ps_precision prec, double rtol, int max_iter, double alpha);

/* Bytes of device workspace a solve on this plan needs (caller allocates it,
 * 256-byte aligned, and may reuse it across solves on the same stream). */
ps_status ps_workspace_bytes(const ps_plan* plan, size_t* bytes);

/* Solve A·p = f (Eq. 4) for FP64 fields (plans with PS_FP64 or
 * PS_FP32_REFINE). f, p: device arrays of nx·ny·nz doubles, each 16-byte aligned
 * (the transforms move lines with 16-byte accesses; PS_INVALID_ARG otherwise);
 * p == f (in place) is allowed for PS_FP64 only. ws: workspace of ps_workspace_bytes. stream:
 * cudaStream_t as void*. info: device ps_info (may be NULL). */
ps_status ps_solve(ps_plan* plan, const double* f, double* p, void* ws, void* stream,
                   ps_info* info);

/* Same for FP32 fields (plans with PS_FP32), f and p 16-byte aligned. p == f allowed. */
ps_status ps_solve_f32(ps_plan* plan, const float* f, float* p, void* ws, void* stream,
                       ps_info* info);

/* Apply the transpose of the solve map (for reverse-mode differentiation).
 * With A = W⁻¹S, W = diag(Δz^f_k), S symmetric, the transpose is
 * p = W · solve(W⁻¹ g); for singular problems the mean-removing projector is
 * transposed the same way. FP64 fields, PS_FP64 plans (PS_FP32 plans use
 * ps_solve_transpose_f32); p == g is allowed. */
ps_status ps_solve_transpose(ps_plan* plan, const double* g, double* p, void* ws, void* stream,
                             ps_info* info);

/* FP32-field variant of ps_solve_transpose (PS_FP32 plans). */
ps_status ps_solve_transpose_f32(ps_plan* plan, const float* g, float* p, void* ws, void* stream,
                                 ps_info* info);

/* Host-buffer convenience: copies f_host (pageable or pinned, nx·ny·nz
 * doubles) to the caller's device buffer f_dev, solves into p_dev, copies p_dev
 * back to p_host and the ps_info to info_host (may be NULL), then synchronises
 * the stream. Device buffers and workspace are the caller's. */
ps_status ps_solve_host(ps_plan* plan, const double* f_host, double* p_host, double* f_dev,
                        double* p_dev, void* ws, void* stream, ps_info* info_host);

/* A sequence of `count` independent solves from host memory with the same plan
 * (the operator of §2.1, Eq. 4; new right-hand sides), their copies pipelined:
 * problem s is copied in (f_host[s], nx·ny·nz doubles) while problem s − 1 is
 * solved, and copied out (to p_host[s]) while problem s + 1 is copied in and
 * solved, on two internal copy streams beside `stream`; the two directions of
 * the host link run at once. f_dev[2] and p_dev[2] are two device slots (each
 * nx·ny·nz doubles, 16-byte aligned, all four disjoint) that problems s and s + 1
 * alternate between; ws is one workspace (ps_workspace_bytes) shared by the
 * solves, which run in order on `stream`. info_host (NULL or `count` entries)
 * receives each solve's ps_info. The host buffers should be pinned for the copies
 * to overlap (pageable ones are correct but serialise); p_host entries may repeat
 * (the copies out run in order, the last one wins) and may equal f_host entries
 * of earlier problems only. The first copies wait for the caller's earlier work
 * on `stream`; the call returns when every copy and solve has ended. Each p
 * equals what ps_solve_host returns for the same f. Plans outside the chunked
 * pipeline (other than PS_FP32_REFINE with x and y lines of 128, 256, 512 or 1024 and
 * n_x a multiple of 16, n_z ≥ 2) run the problems one after another through
 * ps_solve_host with slot 0. Errors: PS_INVALID_ARG for a NULL array or pointer,
 * count < 0, misaligned or overlapping slots; CUDA errors as PS_CUDA_ERROR after
 * the enqueued work has drained. count = 0 does nothing. */
ps_status ps_solve_host_seq(ps_plan* plan, int count, const double* const* f_host, double* const* p_host,
                            double* const* f_dev, double* const* p_dev, void* ws, void* stream,
                            ps_info* info_host);

/* Solve without a caller-provided workspace (same arguments and results as
 * ps_solve, for PS_FP64 and PS_FP32_REFINE plans). The paper has no
 * counterpart: this is a convenience for callers that cannot allocate device
 * memory at solve time (for example code running under another framework's
 * memory pool, or an interface through which no workspace can be passed).
 * The workspace lives in one fixed 8 MiB device array compiled into the
 * library, which every GPU that loads the library keeps until the process
 * exits; plans whose ps_workspace_bytes exceeds 8 MiB are rejected with
 * PS_UNSUPPORTED_SIZE and a message in ps_last_error(plan). The workspace is
 * about 20 B per cell for PS_FP32_REFINE (24 B with a periodic z), 8 B per cell
 * for PS_FP64 (16 B with a periodic z), so the limit is near 4.2·10^5 cells
 * (3.5·10^5), resp. 1.0·10^6 cells (5.2·10^5); ps_workspace_bytes ≤ 8 MiB is the
 * exact test. The first call on a device looks up the array's device address
 * (a set-up step; make that first call before any stream capture); the address
 * is kept with the id of the CUDA context, and the first call in a new context
 * on that device (after cudaDeviceReset) looks it up again.
 * This entry point performs no device allocation. All calls share the one
 * array: calls whose GPU work overlaps (on different streams, or from
 * different threads) race on it and must be serialised by the caller. */
ps_status ps_solve_static(ps_plan* plan, const double* f, double* p, void* stream, ps_info* info);

/* Destroy a plan and free its device tables (NULL is accepted). */
ps_status ps_plan_destroy(ps_plan* plan);

/* Static, NUL-terminated description of the last failure on this plan (or,
 * for plan == NULL, of the last failed ps_plan_create / ps_batch_create). */
const char* ps_last_error(const ps_plan* plan);

/* ---- Projection step around the solve (Eqs. 2b–2c) ---------------------------
 * Staggered (MAC) velocity of §2: component c of a velocity field is stored
 * with the cell array's shape, and the three components are stacked: u is
 * 3·nx·ny·nz values, [u | v | w]. Entry i of a component along its own axis
 * is the face on the low side of cell i: on a periodic axis face 0 is the wrap
 * face; on a Neumann–Neumann axis (prescribed velocity, end of §2) face 0 is
 * the wall, carried through unchanged, and the high wall is implicit. D is the
 * cell divergence (wall faces excluded), G the face gradient (zero on walls),
 * with D·G equal to the operator of Eq. 4; the projection of Eqs. 2b–2c (γΔt
 * cancels) is u = u* − G·solve(D·u*). Only P and NN axes are accepted.
 * Field types follow the plan: float for PS_FP32 plans, double otherwise. All
 * pointers are device pointers; the calls enqueue one kernel on the stream. */

/* One substep k ∈ {1, 2, 3} of the low-storage RK3 fractional-step integration of
 * §2 around the solve (Eqs. 2a–2d), α_k = 8/15, 5/12, 3/4, β_k = 0, −17/60, −5/12,
 * γ_k = α_k + β_k:
 *   u* = u + Δt (α_k AD^k + β_k AD^{k−1} − γ_k G p),   AD = −(u·∇)u + ν∇²u,
 *   solve A Φ' = D u* (Φ' = γ_k Δt Φ),  u ← u* − G Φ',  p ← p + Φ,
 * on the staggered layout of the projection operators above. AD is second-order
 * central: advection in divergence form with arithmetic averages, the viscous term
 * the finite-volume second differences of Eq. 4, each on its component's control
 * volume. The plan must be a Poisson plan (α = 0) with each axis PERIODIC or
 * NEUMANN_NEUMANN; the latter means no-slip walls on that axis (the duct and cavity
 * cases of Table 3 have them on x and y): the normal component is 0 on the wall
 * faces, tangential ghosts are mirrored with the opposite sign.
 *   u      3·N stacked faces [u | v | w]: u^k in, u^{k+1} out (divergence-free).
 *   ustar  3·N scratch (u*), distinct from u.
 *   ad     3·N: AD^{k−1} in (not read when k = 1), AD^k out (in place).
 *   p      N cells: p^{k−1/2} in, p^{k+1/2} out.
 *   phi    N cells: Φ out.   rhs: N cells of scratch (D u*), distinct from phi.
 *   ws     the solve's workspace (ps_workspace_bytes); info as for ps_solve.
 * The byte ranges of u, ustar, ad, p, phi, rhs and ws must be pairwise disjoint
 * (PS_INVALID_ARG naming the overlapping pair otherwise).
 * Field types follow the plan (float for PS_FP32, double otherwise); device
 * pointers, each 16-byte aligned (PS_INVALID_ARG otherwise); enqueued on the
 * stream (four kernels and the solve). */
ps_status ps_ns_substep(ps_plan* plan, int k, double dt, double nu, void* u, void* ustar, void* ad, void* p,
                        void* phi, void* rhs, void* ws, void* stream, ps_info* info);

/* f = D·u* (cell-centred right-hand side of Eq. 2b). */
ps_status ps_div(ps_plan* plan, const void* u, void* f, void* stream);
/* u = u* − G·φ (Eq. 2c). u may equal ustar. */
ps_status ps_grad_correct(ps_plan* plan, const void* ustar, const void* phi, void* u, void* stream);
/* h = Gᵀ·g (cells from a stacked face field g): first step of the projection's
 * vector–Jacobian product. */
ps_status ps_grad_adjoint(ps_plan* plan, const void* g, void* h, void* stream);
/* out = g − Dᵀ·s (stacked faces): last step of the vector–Jacobian product
 * ḡ* = ḡ − Dᵀ·solveᵀ(Gᵀ·ḡ). out may equal g. */
ps_status ps_div_adjoint_correct(ps_plan* plan, const void* g, const void* s, void* out, void* stream);

/* ---- Per-kernel timing (optional) --------------------------------------------
 * When enabled on a plan, every kernel launch of its solves is bracketed by a
 * pair of CUDA events recorded on the solve's stream (no host synchronisation
 * is added to the solve). ps_profile_read synchronises those events, sums the
 * durations per kernel kind and clears the record. A launch whose duration is
 * below a quarter of the longest launch of its kind in the window counts as
 * "skipped" (refinement kernels return at once after convergence). */
typedef struct {
  char name[24];          /* kernel kind: x_fwd, x_fwd_f64in, y_fwd, z_solve, z_singular,
                             y_bwd, x_bwd, x_bwd_f64store, x_bwd_f64acc, residual,
                             residual_check, control, …, and for ps_ns_substep
                             ns_predict, ns_projection, ns_pressure */
  int launches;           /* all launches in the window                         */
  int active_launches;    /* launches that did work (see above)                 */
  double total_ms;        /* summed duration of all launches                    */
  double active_ms;       /* summed duration of the active launches             */
} ps_kernel_stat;

/* Turn event bracketing on (1) or off (0); up to 4096 launches are recorded
 * per window, later ones are dropped and counted in the next read's totals as
 * missing. */
ps_status ps_profile_enable(ps_plan* plan, int enable);

/* Fill up to `max` entries (one per kernel kind), set *count, clear the window. */
ps_status ps_profile_read(ps_plan* plan, ps_kernel_stat* stats, int max, int* count);

/* ---- Fault injection for tests (the paper has no counterpart) ----------------
 * The next `count` device allocations of ps_plan_create / ps_plan_create_helmholtz
 * / ps_batch_create fail on the host as if cudaMalloc had returned
 * cudaErrorMemoryAllocation (no device memory is touched): the create call returns
 * PS_OUT_OF_MEMORY, leaves *out NULL and frees what it had made. 0 disarms.
 * PS_INVALID_ARG for a negative count. Process-wide. */
ps_status ps_inject_alloc_failures(int count);

/* ---- Measurement utility (the paper has no counterpart) -----------------------
 * FP64 FMA throughput of the current device, in TFLOP/s (two FLOPs per FMA): one
 * launch of 8·(SM count) CTAs of 256 threads, each running eight independent
 * chains of `iters` FP64 fused multiply-adds, timed with CUDA events on `stream`
 * (after one short warm-up launch); *ms receives the timed launch's duration.
 * Synchronises the stream and allocates a small device buffer; not for the
 * solve path. The denominator of the plain FP64 solve's roofline, which is bound
 * by the FP64 pipe (1/64 of the FP32 rate on GB300), not by HBM. */
ps_status ps_probe_fp64(int iters, double* tflops, double* ms, void* stream);

/* ---- Batched solve: many independent grids, one persistent launch ----------
 * Each grid is an independent problem of §2.1 with its own sizes, spacings,
 * z faces and BC pairs. */
typedef struct {
  int nx, ny, nz;
  double dx, dy;
  const double* zf;   /* host, nz+1 faces, or NULL for uniform dz */
  double dz;
  ps_bc bcx, bcy, bcz;
} ps_grid_desc;

/* Create a batch of `count` grids (1 ≤ count ≤ 4096); precision
 * PS_FP32_REFINE (FP32 bulk, FP64 refinement), 0 ≤ max_iter ≤ 16. Tables for
 * every grid are built as in ps_plan_create. */
ps_status ps_batch_create(ps_batch** out, int count, const ps_grid_desc* descs,
                          ps_precision prec, double rtol, int max_iter);
/* The same with a Helmholtz shift per grid (see ps_plan_create_helmholtz): grid g
 * solves (A − alphas[g]·I)·p = f. alphas: host array of count values ≥ 0 (copied),
 * or NULL for all zero (ps_batch_create). PS_INVALID_ARG for a negative or
 * non-finite shift (the message names the grid). */
ps_status ps_batch_create_helmholtz(ps_batch** out, int count, const ps_grid_desc* descs,
                                    ps_precision prec, double rtol, int max_iter, const double* alphas);

/* Workspace bytes for one batched solve. */
ps_status ps_batch_workspace_bytes(const ps_batch* batch, size_t* bytes);

/* Solve every grid: f_dev[g], p_dev[g] are DEVICE arrays of DEVICE pointers
 * (count entries each) to the grids' FP64 fields. infos: device array of
 * `count` ps_info (may be NULL). One persistent kernel walks a task queue of
 * (grid, stage, tile); its inter-task waits are bounded and report
 * PS_TIMEOUT in the grid's ps_info instead of hanging. Capturable in a CUDA
 * graph (no host synchronisation, no allocation). */
ps_status ps_batch_solve(ps_batch* batch, double* const* f_dev, double* const* p_dev, void* ws,
                         void* stream, ps_info* infos);

/* Pick the tile sizes of the batched solve (lines per transform task, points
 * per residual task) by timing candidate scales on the caller's fields; the
 * choice is kept in the batch and, when the environment variable
 * PS_AUTOTUNE_CACHE names a file, appended to it as one JSON line keyed by a
 * hash of every grid's sizes, BCs, spacings, z faces and Helmholtz shift, the
 * batch's rtol and max_iter and the GPU name (later calls read it back instead
 * of timing, and return the stored time in best_ms). Runs several solves and synchronises the stream; not capturable.
 * best_ms (may be NULL) receives the time of one batched solve. */
ps_status ps_batch_autotune(ps_batch* batch, double* const* f_dev, double* const* p_dev, void* ws,
                            void* stream, double* best_ms);

/* Current tile scale of the batch: 2 after ps_batch_create, then whichever of
 * the autotuner's candidates 1, 2, 4, 8, 16, 32, 64 it picked. */
int ps_batch_tile_scale(const ps_batch* batch);

/* Wait limit of the persistent kernel's dependency waits, in seconds
 * (default 2). flags bit 0 makes one dependency of grid 0 unsatisfiable, so a
 * test can exercise the bounded wait: the solve then returns with PS_TIMEOUT
 * in the grids' ps_info instead of hanging. */
ps_status ps_batch_configure(ps_batch* batch, double wait_limit_seconds, int flags);

/* Static description of the last failure of ps_batch_* on this batch (or, for
 * NULL, of the last failed ps_batch_create). */
const char* ps_batch_last_error(const ps_batch* batch);

ps_status ps_batch_destroy(ps_batch* batch);

#ifdef __cplusplus
}
#endif

#endif /* PS_POISSON_H */
