/*
 * elas.h -- C ABI of the GB300 matrix-free voxel finite-element elasticity solver.
 *
 * The library computes the periodic voxel finite-element elasticity solve of ELAS3D-Xtal
 * (Jeong & Sundararaghavan, arXiv 2602.07354):
 *   - every voxel is a trilinear hexahedral element (Sec. 2.1.1); node (i,j,k) is the low corner
 *     of voxel (i,j,k) and indices wrap periodically (Sec. 2.1.1, Eq. 1);
 *   - each phase p carries a 6x6 stiffness, isotropic (Eqs. 2-3) or anisotropic and rotated into
 *     the sample frame by its Rodrigues vector (Eq. 4, Algorithm 1); pores have zero stiffness;
 *   - the applied macroscopic strain E (Eq. 5) enters through the energy of Eqs. 7-8; the
 *     library solves for the periodic fluctuation w of the total displacement u_m = E.X_m + w_m,
 *     i.e. A w + b = 0 with A = sum_e P_e^T K_e P_e and b = sum_e P_e^T K_e Ebar (Ebar_a = E.x_a);
 *   - by the matrix-free point-block Jacobi preconditioned conjugate gradient of Algorithm 2.
 *
 * Conventions used by every entry point:
 *   grid      nx, ny, nz >= 2 voxels (= nodes); N = nx*ny*nz; index(i,j,k) = i + nx*(j + ny*k).
 *   vectors   component-major, the "u(ns,3)" layout of Algorithm 2: v[c*N + node], c = 0,1,2
 *             (x, y, z components); 3N values.
 *   phases    phase_id[e] in [0, n_phases) or -1 for a pore (zero stiffness).  A phase whose
 *             6x6 stiffness is all zero also behaves as a pore.
 *   Voigt     order 11, 22, 33, 23, 13, 12.  Stiffness maps engineering strain to stress;
 *             stress vectors hold tensor components; strain inputs (strain[6]) hold TENSOR
 *             components E11, E22, E33, E23, E13, E12 (E23 = E32, not the engineering shear).
 *   units     any consistent set (the tests use GPa and voxel edge 1); the voxel edge drops out
 *             of stresses, displacements are in voxel units.
 *   memory    "dev" pointers are CUDA device memory on the context's device; "host" pointers are
 *             host memory.  Device buffers passed to a call are borrowed: they must stay valid
 *             until the context's stream has executed the work.  Host input arrays are copied
 *             during the call and stay owned by the caller.
 *   stream    every call enqueues its device work on the stream given at elas_create; calls
 *             that return host results (elas_pcg_solve's info, elas_stress's macro stress, the
 *             scalar outputs) synchronise that stream before returning.
 *   errors    every int-returning call returns ELAS_OK (0) or a negative ELAS_ERR_* code and
 *             never throws; elas_last_error(ctx) holds a message for the last failure.
 *   threads   one context, batch or server is driven by one host thread at a time (calls on the
 *             same object are not synchronised with each other); different objects may be used
 *             from different threads at once, each on its own stream.
 */
#ifndef ELAS_H
#define ELAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------------- */
#define ELAS_OK 0
#define ELAS_ERR_INVALID_ARG (-1)   /* bad dims, ids out of range, non-finite/non-symmetric C ... */
#define ELAS_ERR_WORKSPACE (-2)     /* workspace NULL, misaligned or smaller than required */
#define ELAS_ERR_CUDA (-3)          /* a CUDA runtime call failed (message has the CUDA error) */
#define ELAS_ERR_NONFINITE (-4)     /* a solve produced a NaN/Inf (info.status = ELAS_NONFINITE) */
#define ELAS_ERR_TIMEOUT (-5)       /* a bounded device-side wait expired */
#define ELAS_ERR_ADMISSION (-6)     /* request refused by the server's memory budget or queue */
#define ELAS_ERR_STATE (-7)         /* call not valid in the current state (e.g. no solve yet) */

/* ---- solve outcomes (elas_solve_info.status) ------------------------------------------ */
#define ELAS_CONVERGED 0
#define ELAS_MAX_ITER 1
#define ELAS_BREAKDOWN 2     /* h.Ah not positive and finite (relative reading of Alg. 2's guard) */
#define ELAS_NONFINITE 3
#define ELAS_CANCELLED 4     /* a served request withdrawn by elas_server_cancel */

/* ---- precision ------------------------------------------------------------------------- */
#define ELAS_PREC_FP64 0     /* every step in FP64 (the paper's precision, Sec. 2.1.2) */
#define ELAS_PREC_MIXED 1    /* FP32 operator/preconditioner/vectors, FP64 w, reductions and
                                periodic FP64 true-residual replacement */

/* ---- arithmetic of the FP64 operator products --------------------------------------------
 * The FP64 products (the operator of ELAS_PREC_FP64 solves and elas_apply, the FP64 residuals
 * of both precisions) are evaluated either in double-float arithmetic -- every FP64 value of the
 * element product carried as an unevaluated pair of floats (about 48 significant bits) and
 * operated on with error-free float transformations on the FP32 pipe -- or with native FP64
 * instructions.  Vectors, reductions, the Jacobi blocks and every stored value stay IEEE FP64 in
 * both forms; a product differs from the exact one by a few units of 2^-48 of its terms'
 * magnitude in the paired form (2^-53 natively).  The paired form needs the vector entries and
 * stiffness products to stay inside the float exponent range (|v| between about 1e-30 and 1e30;
 * any consistent units of stiffness and voxel-scale displacements qualify); outside it a product
 * overflows to a non-finite value, which a solve reports as ELAS_NONFINITE. */
#define ELAS_FP64_OP_PAIRED 0  /* default: double-float on the FP32 pipe (GB300 issues FP32 at
                                  64x its FP64 rate) */
#define ELAS_FP64_OP_NATIVE 1  /* IEEE FP64 instructions */

/* ---- stopping rule --------------------------------------------------------------------- */
#define ELAS_STOP_PRECOND 0  /* Algorithm 2: sqrt(z.g / z0.g0) < tol */
#define ELAS_STOP_TRUE 1     /* FP64 true relative residual ||A w + b||_2 / ||b||_2 <= tol */

/* ---- preconditioner ---------------------------------------------------------------------- */
#define ELAS_PRECOND_BLOCK 0   /* point-block Jacobi, Eq. 9: the inverse 3x3 diagonal block per node */
#define ELAS_PRECOND_SCALAR 1  /* point Jacobi, M = diag(A) (comparison variant, not in the paper) */
#define ELAS_PRECOND_NONE 2    /* M = I: the plain CG that Table 4 compares against */

typedef struct elas_ctx elas_ctx;

/* Result of a solve.  relres_true is always recomputed in FP64 from the returned w. */
typedef struct {
  int iters;               /* completed PCG iterations */
  int status;              /* ELAS_CONVERGED, ELAS_MAX_ITER, ELAS_BREAKDOWN, ELAS_NONFINITE,
                              ELAS_CANCELLED (served requests) */
  double relres_precond;   /* sqrt(z.g / z0.g0) at exit (recursive residual) */
  double relres_true;      /* ||A w + b|| / ||b|| in FP64 (0 when b = 0) */
  int n_replacements;      /* FP64 residual replacements performed (mixed precision) */
  int launches;            /* kernel launches this call enqueued (graph nodes included) */
  double seconds;          /* wall time of the call */
} elas_solve_info;

/* Optional solve controls; pass NULL for the defaults shown. */
typedef struct {
  int stop_rule;       /* ELAS_STOP_PRECOND for FP64 contexts, ELAS_STOP_TRUE for mixed (default) */
  int replace_every;   /* mixed: FP64 residual replacement interval in iterations (default 50) */
  int check_every;     /* iterations per device-side batch between host status reads (default 0:
                          chosen from the grid size) */
  int replace_drop;    /* mixed: also replace once the recursive residual norm has fallen by a
                          factor 10^replace_drop since the last replacement (0: off, the default);
                          replacements happen at the end of a device-side batch */
  int precond;         /* ELAS_PRECOND_BLOCK (default), ELAS_PRECOND_SCALAR or ELAS_PRECOND_NONE;
                          single-context solves only (batches and the server use the block form) */
} elas_solve_opts;

/* ---- constitutive helpers (host, FP64) -------------------------------------------------- */

/* Eqs. 2-3: isotropic stiffness from Young's modulus E and Poisson's ratio nu (-1 < nu < 0.5).
 * C6: host, 36 doubles, row-major Voigt matrix (written). */
int elas_isotropic_stiffness(double E, double nu, double* C6);

/* Algorithm 1, step 1: cubic crystal-frame stiffness (C11 on the normal diagonal, C12 off the
 * diagonal of the normal block, C44 on the shear diagonal).  C6: host, 36 doubles (written). */
int elas_cubic_stiffness(double c11, double c12, double c44, double* C6);

/* Eq. 4 / Algorithm 1: sample-frame stiffness of a crystal with orientation rho (Rodrigues
 * vector rho = tan(theta/2) n, the active crystal-to-sample rotation; Sec. 2.2.3), computed
 * with the 6x6 Bond matrix of the rotation.  C6_local, C6_global: host, 36 doubles. */
int elas_rotated_stiffness(const double* C6_local, const double* rho, double* C6_global);

/* ---- context ---------------------------------------------------------------------------- */

/* Bytes of device workspace elas_create needs for this grid, phase count and precision.
 * bytes: host, written. */
int elas_workspace_bytes(int nx, int ny, int nz, int n_phases, int precision, size_t* bytes);

/* Create a solver context (Sec. 2.1.3 stages 1-3: parameters, microstructure, stiffness).
 *   phase_id   host, N int32 (-1 = pore), copied to the device.
 *   C_local    host, n_phases*36 doubles: crystal-frame Voigt stiffness per phase (must be
 *              symmetric and finite; a zero matrix makes the phase a pore).
 *   rodrigues  host, n_phases*3 doubles or NULL (identity): per-phase orientation.
 *   precision  ELAS_PREC_FP64 or ELAS_PREC_MIXED.
 *   workspace  device, >= elas_workspace_bytes() bytes, 256-byte aligned; owned by the caller
 *              and used exclusively by this context until elas_destroy.
 *   cuda_stream  cudaStream_t on which all work of this context is enqueued (NULL = legacy
 *              default stream).
 * Builds the per-phase tables (rotation, scaled element coefficients) on the host in FP64 and
 * uploads them with the phase ids; returns without waiting for the uploads.  *out receives the
 * context. */
int elas_create(elas_ctx** out, int nx, int ny, int nz, const int32_t* phase_id, int n_phases,
                const double* C_local, const double* rodrigues, int precision, void* workspace,
                size_t ws_bytes, void* cuda_stream);

/* Release the host-side context (the workspace stays the caller's).  NULL is ignored. */
void elas_destroy(elas_ctx* ctx);

/* Message of the last failure on this context ("" if none); ctx NULL gives the last failure of
 * elas_create on this thread. */
const char* elas_last_error(const elas_ctx* ctx);

/* ---- the hot path ----------------------------------------------------------------------- */

/* Matrix-free operator product y = A u in FP64 (Sec. 2.1.2 "Ah = A h", Algorithm 2 step A):
 * the 27-point periodic stencil applied element by element.  u, y: device, 3N doubles each,
 * component-major; must not overlap. */
int elas_apply(elas_ctx* ctx, const double* u, double* y);

/* The same product in FP32 (the operator of the mixed-precision path).  u, y: device, 3N floats. */
int elas_apply_f32(elas_ctx* ctx, const float* u, float* y);

/* Select the arithmetic of this context's FP64 products (ELAS_FP64_OP_PAIRED, the default, or
 * ELAS_FP64_OP_NATIVE) for every later elas_apply, elas_residual and elas_pcg_solve.  The paper
 * computes in FP64 (Sec. 2.1.2); both forms meet it to a relative 1e-12 per product. */
int elas_set_fp64_operator(elas_ctx* ctx, int form);

/* Right-hand side b = sum_e P_e^T K_e Ebar of Eqs. 7-8 for applied strain E (tensor components
 * E11,E22,E33,E23,E13,E12, host).  b: device, 3N doubles. */
int elas_rhs(elas_ctx* ctx, const double* strain, double* b);

/* Gradient g = A w + b (Sec. 2.1.2, the "gb" of Algorithm 2) in FP64 for a given fluctuation w.
 * w, g: device, 3N doubles.  rnorm: host, receives ||g||_2 (may be NULL; then no sync). */
int elas_residual(elas_ctx* ctx, const double* strain, const double* w, double* g, double* rnorm);

/* Point-block Jacobi inverse of Eq. 9 in FP64 (every solve builds its own copy; this call builds
 * one into the caller's buffer): Minv: device, 6N doubles written as
 * six component-major planes (inverse entries 11, 22, 33, 23, 13, 12 of each symmetric 3x3
 * inverse block).  Nodes whose 8 voxels are all pores carry the identity. */
int elas_jacobi(elas_ctx* ctx, double* Minv);

/* Algorithm 2: build the point-block Jacobi preconditioner (Eq. 9, Algorithm 2 part 1), then solve
 * A w = -b for the applied strain (host, 6 tensor components) from w = 0 (the affine start
 * u0 = E.X of Eq. 5) with the point-block Jacobi PCG, until the stopping
 * rule holds at tol or max_iter iterations ran.  opts: host or NULL.  w_out: device, 3N doubles
 * (the periodic fluctuation; total u_m = E.X_m + w_m), or NULL to keep it inside the context
 * only.  info: host, written (may be NULL).  Returns ELAS_OK for converged, max-iter and
 * breakdown outcomes (see info.status) and ELAS_ERR_NONFINITE if the iteration produced a
 * non-finite value.  The fluctuation of the last solve stays in the context for elas_stress. */
int elas_pcg_solve(elas_ctx* ctx, const double* strain, double tol, int max_iter,
                   const elas_solve_opts* opts, double* w_out, elas_solve_info* info);

/* Voxel stress (stress_OpenMP / stress_fullfield_OpenMP of Sec. 2.1.3, Table 1): strain at the
 * voxel centroid (the exact voxel average of the trilinear field) eps = E + sym(grad w), stress
 * sigma = C eps, von Mises sigma_vm = sqrt(((s11-s22)^2+(s22-s33)^2+(s33-s11)^2)/2 +
 * 3(s23^2+s13^2+s12^2)), and the macroscopic stress (mean over all N voxels, pores count 0).
 *   strain  host, 6 tensor components (the load of w).
 *   w       device, 3N doubles, or NULL for the fluctuation of the last solve.
 *   stress  device, 6N doubles (component-major, Voigt order, tensor shears) or NULL.
 *   von_mises  device, N doubles or NULL.
 *   macro_stress  host, 6 doubles or NULL (synchronises the stream). */
int elas_stress(elas_ctx* ctx, const double* strain, const double* w, double* stress,
                double* von_mises, double* macro_stress);

/* ---- batched solves ----------------------------------------------------------------------- */

/* One RVE of a batch: grid, per-voxel phase ids and per-phase constants, with the meaning of the
 * same arguments of elas_create.  All pointers are host memory, read during elas_batch_create. */
typedef struct {
  int nx, ny, nz;
  const int32_t* phase_id;   /* N int32, -1 = pore */
  int n_phases;
  const double* C_local;     /* n_phases*36 */
  const double* rodrigues;   /* n_phases*3 or NULL */
} elas_rve;

typedef struct elas_batch elas_batch;

/* Bytes of device workspace for n_rve RVEs with n_rhs load cases each at this precision. */
int elas_batch_workspace_bytes(int n_rve, const elas_rve* rves, int n_rhs, int precision, size_t* bytes);

/* Create a batch: every (RVE, load case) pair becomes one problem, and all problems advance
 * together through Algorithm 2 in shared persistent launches (one operator, one update and one
 * direction launch per iteration for the whole batch), replayed as a captured CUDA graph.  A
 * problem's result does not depend on the other problems of the batch.  workspace: device,
 * >= elas_batch_workspace_bytes(), 256-byte aligned, caller-owned.  The paper solves one RVE and
 * one load at a time; batching several load cases of one RVE gives the columns of the effective
 * stiffness in one pass. */
int elas_batch_create(elas_batch** out, int n_rve, const elas_rve* rves, int n_rhs, int precision, void* workspace,
                      size_t ws_bytes, void* cuda_stream);

/* Per grid size in the batch, time candidate operator tilings and keep the fastest (the per-size
 * schedule, shared with elas_autotune).  Synchronises the stream. */
int elas_batch_autotune(elas_batch* b, int max_candidates);

/* Solve every problem: strains: host, n_rve*n_rhs*6 tensor components, load case r of RVE i at
 * offset (i*n_rhs + r)*6.  tol, max_iter, opts as in elas_pcg_solve.  infos: host, n_rve*n_rhs
 * entries (may be NULL).  Returns ELAS_ERR_NONFINITE if any problem met a non-finite value. */
int elas_batch_solve(elas_batch* b, const double* strains, double tol, int max_iter, const elas_solve_opts* opts,
                     elas_solve_info* infos);

/* Arithmetic of the batch's FP64 products for later solves, as elas_set_fp64_operator. */
int elas_batch_set_fp64_operator(elas_batch* b, int form);

/* Fluctuation w of one problem of the last solve.  w_out: device, 3N doubles. */
int elas_batch_fluctuation(elas_batch* b, int rve, int rhs, double* w_out);

/* Stress of one problem of the last solve, as elas_stress with w = that problem's fluctuation. */
int elas_batch_stress(elas_batch* b, int rve, int rhs, const double* strain, double* stress, double* von_mises,
                      double* macro_stress);

void elas_batch_destroy(elas_batch* b);
const char* elas_batch_last_error(const elas_batch* b);

/* ---- solve server (continuous batching) ---------------------------------------------------- */

/* A solve server admits requests (one RVE, one applied strain, a tolerance) as device memory
 * and slots free up, keeps every admitted request's CG state resident on the device, and
 * advances all of them together, K PCG iterations per step, in shared persistent launches
 * (Algorithm 2 for each request).  Requests that arrive while others run join at the next step.
 * A request's result is the same alone and in any mix.  The paper runs one solve at a time. */
typedef struct elas_server elas_server;

/* Workspace for a server with a device-memory budget for requests (bytes) and at most max_active
 * requests in flight: the budget plus the server's tables. */
int elas_server_workspace_bytes(size_t budget_bytes, int max_active, size_t* bytes);

/* precision: ELAS_PREC_MIXED (default stop rule: FP64 true residual) or ELAS_PREC_FP64
 * (Algorithm 2's rule); iters_per_step: K (0 = 50 mixed / 32 FP64).  workspace: device,
 * >= elas_server_workspace_bytes(), 256-byte aligned, caller-owned. */
int elas_server_create(elas_server** out, size_t budget_bytes, int max_active, int precision, int iters_per_step,
                       void* workspace, size_t ws_bytes, void* cuda_stream);

/* Queue a request.  rve: host, copied; strain: host, 6 tensor components.  *id: host, the
 * request id.  ELAS_ERR_ADMISSION if the request alone exceeds the budget (it is not queued). */
int elas_server_submit(elas_server* s, const elas_rve* rve, const double* strain, double tol, int max_iter,
                       long long* id);

/* One step: admit queued requests in arrival order while the next fits (memory and slots), run
 * K iterations of every admitted request, and retire the ones that stopped (their final FP64 w
 * and true residual are formed on the device).  Outputs (host, may be NULL): requests in flight,
 * still queued, and retired by this step.  Synchronises the stream once. */
int elas_server_step(elas_server* s, int* n_active, int* n_queued, int* n_finished);

/* Collect a retired request: *done = 1 and info (host), its fluctuation w (device, 3N doubles,
 * may be NULL) and its latency from submission to retirement in seconds (host, may be NULL);
 * its device memory returns to the budget.  *done = 0 if it has not finished yet. */
int elas_server_poll(elas_server* s, long long id, elas_solve_info* info, double* w_out, double* latency_s,
                     int* done);

/* Withdraw request id.  Queued: it leaves the queue and is reported finished with status
 * ELAS_CANCELLED, 0 iterations and no fluctuation (poll leaves w_out untouched).  Running: it
 * stops at the next step (no more iterations), its FP64 w and true residual are formed and it is
 * reported finished with status ELAS_CANCELLED.  Finished: nothing happens.  Unknown id:
 * ELAS_ERR_INVALID_ARG.  Call between steps (not concurrently with elas_server_step). */
int elas_server_cancel(elas_server* s, long long id);

/* Mixed-precision residual replacement policy for requests admitted from now on, with the
 * meaning of the elas_solve_opts fields: replace_every > 0 sets the interval in iterations
 * (default 50), replace_drop > 0 also replaces once the residual has fallen by 10^replace_drop
 * since the last replacement (default off).  Negative values: ELAS_ERR_INVALID_ARG. */
int elas_server_set_replacement(elas_server* s, int replace_every, int replace_drop);

/* Device bytes held by requests, requests in flight / queued, requests retired so far. */
int elas_server_stats(elas_server* s, size_t* bytes_in_use, int* n_active, int* n_queued, long long* n_done);

void elas_server_destroy(elas_server* s);
const char* elas_server_last_error(const elas_server* s);

/* App. C: maximum von Mises stress for the stress concentration K_t = sigma_max / sigma_nom.
 * smoothed = G * (vm M) / G * M with M the solid indicator (phase id >= 0) and G the periodic
 * Gaussian of standard deviation s_kernel voxels (the paper uses 0.4), truncated at radius
 * ceil(2 s_kernel) <= 4; defined in pores too (from the solid voxels in reach), 0 where no solid
 * voxel is in reach.  A hotspot is a solid voxel whose smoothed value no competing 26-neighbour
 * exceeds; neighbours: ELAS_HOTSPOT_ALL (every neighbour competes, pores included: the regional
 * maxima of the whole smoothed field that lie in the solid) or ELAS_HOTSPOT_SOLID (only solid
 * neighbours compete: the regional maxima of the field restricted to the solid, whose largest is
 * the largest smoothed value in the solid).  *sigma_max: the largest hotspot value (0 if there is
 * none); *voxel (may be NULL): the lowest voxel id holding it (-1 if none).  von_mises: device N
 * doubles (e.g. from elas_stress); smoothed: device N doubles, written.  Synchronises the
 * context's stream.  An unknown neighbours value: ELAS_ERR_INVALID_ARG. */
#define ELAS_HOTSPOT_ALL 0
#define ELAS_HOTSPOT_SOLID 1
int elas_hotspot(elas_ctx* ctx, const double* von_mises, double s_kernel, int neighbours, double* smoothed,
                 double* sigma_max, long long* voxel);

/* ---- microstructure generator (Sec. 2.2, upstream of the solve) ------------------------------
 * Grid conventions as for elas_create: voxel (i,j,k) has centre (i+1/2, j+1/2, k+1/2) in voxel
 * units, ids x fastest, the cell is periodic (minimum-image differences).  Both calls enqueue on
 * cuda_stream and synchronise it before returning; workspace: caller-owned device memory, 256-byte
 * aligned, at least elas_generate_workspace_bytes(nx, ny, nz, n_grains, n_pores) bytes (one
 * workspace serves both calls).  Errors: ELAS_ERR_INVALID_ARG, ELAS_ERR_WORKSPACE, ELAS_ERR_CUDA,
 * with the message in elas_generate_last_error() (per host thread). */
int elas_generate_workspace_bytes(int nx, int ny, int nz, int n_grains, int n_pores, size_t* bytes);

/* Algorithm 4: every voxel takes the grain l that minimises the weighted ellipsoidal distance
 * D^2 = (dx^2 + dy^2) / rt_l^2 + dz^2 / rl_l^2 (dx, dy, dz: minimum-image difference of the voxel
 * centre and seed l), ties to the lowest l; exactly the result of a brute-force scan.
 * seeds: host, n_grains x 3 doubles in [0, n_d); semi_axes: host, n_grains x 2 (rt, rl) > 0, or
 * NULL for plain Voronoi (rt = rl = 1); phase: device, nx*ny*nz int32 (written). */
int elas_assign_grains(int nx, int ny, int nz, const double* seeds, const double* semi_axes, int n_grains,
                       int32_t* phase, void* workspace, size_t ws_bytes, void* cuda_stream);

/* Algorithm 5 with rotated ellipsoids: pore p = 15 doubles (cx, cy, cz, a0, a1, a2, R00, R01, ...,
 * R22), R row-major with the principal axes as columns (a sphere of radius r: a = (r, r, r),
 * R = I).  Voxels whose centre satisfies sum_m (q_m / a_m)^2 <= 1, q = R^T d, are set to -1 (the
 * pore id); centres must lie in the grid and semi-axes below half the smallest grid dimension.
 * pores: host; phase: device, updated in place; *n_pore_voxels (host, may be NULL): voxels with a
 * negative id afterwards. */
int elas_stamp_pores(int nx, int ny, int nz, const double* pores, int n_pores, int32_t* phase,
                     long long* n_pore_voxels, void* workspace, size_t ws_bytes, void* cuda_stream);

/* Algorithm 3, grain count: N_g = ceil(V / V_mean) for a box lx x ly x lz (any length unit) with
 * the mean grain volume of a cylinder of diameter mean_d and height mean_alpha * mean_d,
 * V_mean = pi (mean_d/2)^2 mean_alpha mean_d.  *n_grains: host, written.  Host arithmetic only. */
int elas_grain_count(double lx, double ly, double lz, double mean_d, double mean_alpha, long long* n_grains);

/* Algorithm 3, seeding (Eq. 10): grain i takes the diameter d_i = exp(m_d + s_d z[2i]) and the aspect
 * ratio alpha_i = exp(m_a + s_a z[2i+1]), lognormal with the given mean and standard deviation of
 * the variate itself (s = sqrt(log(1 + (sd/mean)^2)), m = log(mean) - s^2/2), the prolate semi-axes
 * rt_i = d_i / 2 (transverse) and rl_i = alpha_i rt_i (along X3), and the seed
 * lo + u[3i..3i+2] (hi - lo), each product and sum rounded separately.
 *   lo, hi      host, 3 doubles each: the box (lo < hi on every axis).
 *   z           device, n_grains x 2 standard normal draws; u: device, n_grains x 3 draws in [0,1).
 *   seeds       device, n_grains x 3 (written); semi_axes: device, n_grains x 2 (rt, rl; written),
 *               the inputs of elas_assign_grains once copied to the host.
 * Enqueued on cuda_stream; returns without waiting.  The paper draws the variates inside the
 * algorithm; here they are inputs, so any generator can drive it. */
int elas_seed_grains(int n_grains, const double* lo, const double* hi, double mean_d, double sd_d, double mean_alpha,
                     double sd_alpha, const double* z, const double* u, double* seeds, double* semi_axes,
                     void* cuda_stream);

/* Algorithm 6: one Rodrigues vector rho = tan(theta/2) n per grain (device, n_grains x 3, written).
 *   ELAS_TEXTURE_FIBER   R = R_spin(phi) R_wobble R_base: R_base turns the crystal axis (host, 3
 *                        doubles; NULL = <101>) onto the sample axis (NULL = X3), R_spin turns by phi
 *                        about X3, R_wobble by theta about (cos alpha, sin alpha, 0); draws (device,
 *                        n_grains x 3) = (phi, alpha, theta) in radians, theta ~ N(0, spread^2) for
 *                        the paper's Gaussian spread.
 *   ELAS_TEXTURE_RANDOM  Shoemake's uniform quaternion (q_w, q_x, q_y, q_z) =
 *                        (sqrt(1-u1) sin 2pi u2, sqrt(1-u1) cos 2pi u2, sqrt(u1) sin 2pi u3,
 *                        sqrt(u1) cos 2pi u3) from draws (u1, u2, u3) in [0,1); the axes are unused.
 * rho = (q_x, q_y, q_z) / q_w, or 1e9 (q_x, q_y, q_z) when |q_w| < 1e-8 (the paper's half-turn guard,
 * applied to both branches).  Enqueued on cuda_stream; returns without waiting. */
#define ELAS_TEXTURE_FIBER 0
#define ELAS_TEXTURE_RANDOM 1
int elas_orientations(int n_grains, int texture, const double* crystal_axis, const double* sample_axis,
                      const double* draws, double* rho, void* cuda_stream);

const char* elas_generate_last_error(void);

/* ---- tuning ------------------------------------------------------------------------------ */

/* Time the operator product of this context's grid (its precision) under up to max_candidates
 * tile shapes / z-chunks (0 = 12), keep the fastest for this context and for every later context
 * or batch problem of the same grid size in the process (the per-size schedule).  The paper has
 * no counterpart: its cache-block size (Sec. 2.1.2) is tuned by hand.  Synchronises the stream;
 * overwrites the context's internal vectors (call it before a solve, not between a solve and
 * elas_stress(w = NULL)).  best_ms: host, the best time of one product (may be NULL). */
int elas_autotune(elas_ctx* ctx, int max_candidates, double* best_ms);

/* The per-size operator tilings chosen by elas_autotune / elas_batch_autotune in this process (the
 * autotuner's cache, used by every later context, batch problem or server request of that size),
 * as text: one line "nx ny nz elem_bytes sm_count tx ty kc" per grid size, precision (elem_bytes 8:
 * FP64, 4: FP32) and SM count.  buf (host, may be NULL) receives at most cap bytes, NUL-terminated;
 * *len (may be NULL) the full length without the NUL. */
int elas_tuning_export(char* buf, size_t cap, size_t* len);

/* Records tilings given as text in the export format (e.g. saved by an earlier process).  A line
 * that does not describe a valid tiling of its grid fails the call with ELAS_ERR_INVALID_ARG and
 * nothing is recorded; message in elas_last_error(NULL). */
int elas_tuning_import(const char* text);

/* ---- stress without allocation ----------------------------------------------------------- */

/* The paper has no counterpart to this entry point; it serves callers that cannot allocate.
 *
 * elas_stress_noalloc computes exactly what elas_stress computes (voxel stress, von Mises and
 * macroscopic stress of a fluctuation w under the applied strain) without a context and without
 * allocating any memory.  It is meant for code that must not call cudaMalloc, cudaMallocHost or
 * another allocating routine at the point of the call: work recorded while a CUDA graph is being
 * captured elsewhere in the process, real-time loops whose memory is fixed at start-up, plug-ins
 * inside a host framework that owns all device memory, or a server whose memory budget is spent.
 * (elas_create does not suit them: a context allocates a pinned status buffer and a stream.)
 *
 *   nx, ny, nz   grid, each >= 2.
 *   phase_id     device, N int32, each in [-1, n_phases); checked on the device before use.
 *   n_phases     0 .. ELAS_NOALLOC_MAX_PHASES.
 *   C_local      host, n_phases*36 doubles, crystal-frame stiffness (symmetric, finite).
 *   rodrigues    host, n_phases*3 doubles or NULL (identity).
 *   strain       host, 6 tensor components E11,E22,E33,E23,E13,E12.
 *   w            device, 3N doubles (component-major fluctuation).
 *   stress       device, 6N doubles or NULL;  von_mises: device, N doubles or NULL.
 *   macro_stress host, 6 doubles or NULL.
 *   cuda_stream  stream for the work; the call waits for it (id check, macro stress).  It must
 *                not be capturing (the call refuses a capturing stream with ELAS_ERR_INVALID_ARG);
 *                when another thread may be capturing, pass a non-blocking stream rather than the
 *                legacy default stream, which synchronises implicitly with other blocking streams.
 * Scratch: a fixed 1 MiB array compiled into the library, held by every GPU that loads it until
 * the process exits.  The first call on a device looks up that array's address and, under lazy
 * module loading, loads the library's device code, which can allocate: the promise of no
 * allocation holds from the second call on each device, so make one warm-up call per device at
 * start-up, before any stream capture begins.  All calls on a device share the array, which
 * keeps the last call's contents: calls whose work overlaps on the GPU race and must be ordered
 * by the caller.  Returns ELAS_OK, ELAS_ERR_INVALID_ARG (sizes, n_phases above the maximum,
 * non-finite or non-symmetric input, phase ids out of range, a capturing stream) or ELAS_ERR_CUDA;
 * it records no message (writing one could allocate). */
#define ELAS_NOALLOC_MAX_PHASES 4096
int elas_stress_noalloc(int nx, int ny, int nz, const int32_t* phase_id, int n_phases,
                        const double* C_local, const double* rodrigues, const double* strain,
                        const double* w, double* stress, double* von_mises, double* macro_stress,
                        void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* ELAS_H */
