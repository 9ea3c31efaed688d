/*
 * unocg.h -- C ABI of the GB300 (sm_103a) UNO-CG solver for periodic voxel homogenization.
 *
 * The solver is the preconditioned conjugate gradient method of Algorithm 1 with the unitary
 * neural operator (UNO) preconditioner of Sec. 5.2, i.e. Algorithm 2 ("UNO-CG"), applied to the
 * periodic FE homogenization problems of Sec. 6: thermal conduction (c = 1 DOF per node, Sec.
 * 6.1) and linear elasticity (c = 3, Sec. 6.2) on a regular grid of trilinear hexahedral voxels
 * (Sec. 4.1).  Every step of the solve runs in this library's CUDA kernels on one GPU.
 *
 * Conventions
 *   - Grid N1 x N2 x N3, node/voxel (i1, i2, i3) with i3 fastest; voxel edge h = L0 / N1.
 *   - Host field I/O uses the paper's interleaved DOF order (Sec. 2.1): value of component j
 *     at node i at index c*i + j (double precision).
 *   - Loads: thermal macroscopic gradients g_bar (3 values each); elastic macroscopic strains
 *     eps_bar in Mandel notation [11, 22, 33, sqrt2*12, sqrt2*13, sqrt2*23] (App. A).
 *   - A context holds B >= 1 instances of one grid size (a batch), each with the same number
 *     of phases; all instances share the load cases.
 *
 * Ownership and errors
 *   - Host pointers are read or written synchronously during the call and never retained.
 *   - The library owns every device buffer it allocates; `_dev` entry points take caller-owned
 *     device pointers plus a cudaStream_t (passed as void*; NULL is the legacy default stream),
 *     never free them, and enqueue work on that stream without blocking the host.  For the
 *     contexts (unocg_ctx, unocg_dir) that stream is ordered by events after the work already
 *     enqueued on the context's stream, and the context's later work after it; no event is
 *     added while either stream captures a CUDA graph (the capture then orders the work).
 *   - Every int-returning call returns UNOCG_OK (0) or a negative UNOCG_ERR_* code; the message
 *     of the last failure of a context is returned by unocg_last_error().
 */
#ifndef UNOCG_H
#define UNOCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define UNOCG_OK 0
#define UNOCG_ERR_INVALID_ARG -1    /* bad size, pointer, enum or unsupported grid */
#define UNOCG_ERR_OOM -2            /* device allocation failed */
#define UNOCG_ERR_NOT_SPD -3        /* weights fail the safety check lambda_min(Q(k)) > eps */
#define UNOCG_ERR_NOT_CONVERGED -4  /* max_iter reached before the tolerance */
#define UNOCG_ERR_BREAKDOWN -5      /* r.s <= 0, d.p <= 0 or a NaN/Inf in a reduction */
#define UNOCG_ERR_DEVICE_TIMEOUT -6 /* a bounded device-side wait gave up */
#define UNOCG_ERR_CUDA -7           /* a CUDA runtime call failed (message has the detail) */
#define UNOCG_ERR_STATE -8          /* call out of order (e.g. solve before microstructure) */

/* physics */
#define UNOCG_THERMAL 1 /* c = 1: conductivity kappa per phase, loads are gradients (3)   */
#define UNOCG_ELASTIC 3 /* c = 3: (E, nu) per phase, loads are Mandel strains (6)          */

/* preconditioners */
#define UNOCG_PRECOND_NONE 0
#define UNOCG_PRECOND_JACOBI 1 /* P = diag(K)^-1, Sec. 4.2                          */
#define UNOCG_PRECOND_UNO 2    /* P = T^H Q T, Eq. (FNOCG-prec-fields-disc)         */

/* precision */
#define UNOCG_FP64 0  /* every field and reduction in double precision                   */
#define UNOCG_MIXED 1 /* FP32 fields, K.u, transforms and block multiply; BF16 weights;
                         FP64 dot products, scalars, periodic true-residual replacement    */

/* weight kinds for unocg_set_uno_weights */
#define UNOCG_W_REFERENCE_MEDIUM 0 /* Q(k) = S_ref(k)^-1 (k != 0), Q(0) = 0: the FANS
                                      fundamental solution of Sec. 4.3.4 for a homogeneous
                                      medium with the arithmetic mean of the phase
                                      conductivities / Lame constants; `w` unused          */
#define UNOCG_W_BLOCKS 1           /* unique block entries on the half grid,
                                      [N1][N2][N3/2+1][C] in the paper's order (App. B.2)
                                      v1=Q11 v2=Q22 v3=Q12 v4=Q33 v5=Q23 v6=Q13 (C = 1 or 6) */
#define UNOCG_W_THETA 2            /* parameters theta [N1][N2][N3/2+1][C] mapped through the
                                      local parametrization psi (Sec. 5.2.2, App. B.1)        */
#define UNOCG_W_MODES 3            /* the paper's layout (Eq. (fnocg-parametrization)): inner
                                      bypass psi(w_0) on every mode plus psi(w_i) on the
                                      modes of K_M; set with unocg_set_uno_modes             */

/* dtypes of weight arrays */
#define UNOCG_DTYPE_F64 0
#define UNOCG_DTYPE_F32 1

typedef struct unocg_ctx unocg_ctx;

typedef struct {
  double tol;        /* relative residual: stop when ||r||_inf <= tol * ||r_0||_inf        */
  int max_iter;      /* iterations per (instance, load) before UNOCG_ERR_NOT_CONVERGED      */
  int precond;       /* UNOCG_PRECOND_*                                                     */
  int precision;     /* UNOCG_FP64 or UNOCG_MIXED                                           */
  int replace_every; /* MIXED: true-residual replacement after this many iterations since the
                        previous one, e.g. 50; 0 disables the periodic trigger              */
  int flexible;      /* 1: Polak-Ribiere coefficient (flexible CG), 0: Algorithm 1's        */
  int use_graph;     /* loop driver: 0 host-driven loop, one residual check per iteration;
                        1 one CUDA graph with conditional nodes (device-side control);
                        2 one persistent cooperative kernel with grid barriers (UNO only,
                          problems whose phase buffers fit in shared memory);
                        3 automatic: the driver chosen by unocg_autotune / unocg_set_tuning,
                          else 1                                                             */
  double replace_drop; /* MIXED: also replace once ||r||_inf has fallen below replace_drop
                          times its value at the previous replacement (reliable updates: the
                          FP32 solution increment since then stays small); 0 disables, 1e-3
                          keeps the iteration count of the FP64 path up to 256^3 grids      */
} unocg_solve_opts;

typedef struct {
  int status;          /* UNOCG_OK or the first failing per-(instance, load) status          */
  int max_iters;       /* largest iteration count over all (instance, load)                 */
  int* iters;          /* optional [B*L]: iterations                                        */
  double* rel_res;     /* optional [B*L]: final ||r||_inf / ||r_0||_inf (recursive residual) */
  double* true_rel_res;/* optional [B*L]: final ||f - K u||_inf / ||f||_inf in FP64         */
  int* load_status;    /* optional [B*L]: per (instance, load) status                       */
  int checks;          /* residual checks after CG steps (= loop bodies executed + 1)        */
  int replacements;    /* residual replacements executed (mixed precision)                  */
} unocg_solve_info;

/* Create a context for `batch` instances on an n1 x n2 x n3 grid (each n_i of the form
   2^a 3^b 5^c, n3 even, every n_i >= 2) with RVE edge L0 along axis 1.  Sec. 4.1.
   The transform passes keep whole lines in shared memory, which bounds n1 <= 287 and
   n2 <= 426; larger grids return UNOCG_ERR_INVALID_ARG.                                   */
int unocg_create(unocg_ctx** out, int physics, int batch, int n1, int n2, int n3, double L0);
void unocg_destroy(unocg_ctx* ctx);
const char* unocg_last_error(const unocg_ctx* ctx);

/* Tuning of the periodic solver: radix_order of the shared-memory Stockham plans (0: radix 8,
   4, 2, then 3, 5; 1: radix 4, 2, 3, 5; 2: radix 5, 3, then 4, 2; the register FFT passes of
   axes of 2^k and 3 x 2^k points have no radix choice) and the loop driver that use_graph = 3 takes (1 graph,
   2 persistent kernel when it fits).  Invalidates the captured graph.                       */
int unocg_set_tuning(unocg_ctx* ctx, int radix_order, int path);
/* Autotuner (batched solves, config sweeps): times `reps` solves of `opts` (after one warm-up
   solve each) for every radix order and loop driver, writes the mean ms to
   times[radix_order * 2 + (path - 1)] (double[6]; NaN where the persistent kernel does not
   fit) and keeps the fastest setting.  Needs the inputs and weights set.                    */
int unocg_autotune(unocg_ctx* ctx, const unocg_solve_opts* opts, int reps, double* times);

/* Tile of the FP32 thermal K d (the operator apply of Algorithm 2 in mixed precision).
   tile = -1: automatic (default); 0: the register column march (below 10^6 nodes per field) or
   the element kernel; k = 1..8: the TMA-staged kernel, whose block holds TY node rows over the
   whole N3 extent (N3 / 4 threads per row) and marches over P node planes, with
   (TY, P) = (4, 12), (8, 12), (2, 12), (8, 24), (16, 6), (4, 24), (16, 12), (8, 6); k = 9..16:
   the vector march with the shape of k - 8 (the same block layout, node planes read straight
   from global memory instead of staged by the TMA).  The TMA kernel needs N3 a multiple of 32
   up to 256, the vector march up to 512; both TY dividing N2 and 64 to 512 threads a block
   (a multiple of 32).  Unavailable shapes return UNOCG_ERR_INVALID_ARG.  Elastic problems
   ignore the setting.  unocg_get_ku_tile returns the tile the next solve uses (0..16).      */
int unocg_set_ku_tile(unocg_ctx* ctx, int tile);
int unocg_get_ku_tile(unocg_ctx* ctx, int* tile);
/* Stencil autotuner: times `reps` FP32 K d launches over all B x L fields of the context for
   the earlier kernels (times[0]), each TMA tile shape (times[1..8]) and each vector-march shape
   (times[9..16]), NaN where unavailable (times: double[17]), keeps the fastest
   (unocg_set_ku_tile) and returns its index in *best (may be NULL).  Needs
   the microstructure, properties and loads set.  UNOCG_ERR_DEVICE_TIMEOUT if a tile copy's
   bounded wait expired (the setting is then left unchanged).                               */
int unocg_autotune_ku(unocg_ctx* ctx, int reps, double* times, int* best);

/* Upper bound of any device-side wait of this context (the grid barrier of the persistent
   loop, the tile copies of the TMA-staged K d), in seconds (default 1).  A wait that expires makes every block of the launch return
   and the solve report UNOCG_ERR_DEVICE_TIMEOUT; the context stays usable.                 */
int unocg_set_wait_limit(unocg_ctx* ctx, double seconds);

/* Use `stream` (a cudaStream_t) for all work of this context; NULL = the context's own.    */
int unocg_set_stream(unocg_ctx* ctx, void* stream);

/* Voxel phase labels, uint8 [B][N1][N2][N3] (host), labels < n_phases (Sec. 6).           */
int unocg_set_microstructure(unocg_ctx* ctx, const uint8_t* phase, int n_phases);
/* Same from caller-owned device memory (enqueued on `stream`).                             */
int unocg_set_microstructure_dev(unocg_ctx* ctx, const uint8_t* phase_dev, int n_phases, void* stream);

/* Phase properties [B][n_phases] kappa (thermal) or [B][n_phases][2] (E, nu) (elastic).    */
int unocg_set_phase_properties(unocg_ctx* ctx, const double* props);

/* Macroscopic load cases: [n_loads][3] gradients or [n_loads][6] Mandel strains (finite, else
   UNOCG_ERR_INVALID_ARG).                                                                  */
int unocg_set_macro_load(unocg_ctx* ctx, int n_loads, const double* loads);

/* UNO weights (Eq. (fnocg-parametrization), Eq. (prec-sparse-def)); performs the safety check
   of the Remark after Algorithm 2 (lambda_min(Q(k)) > spd_eps for all k != 0) and returns
   UNOCG_ERR_NOT_SPD if it fails, also after rounding to BF16 for the mixed path.  `w` is host
   memory of `dtype`; shared by all instances (REFERENCE_MEDIUM is per instance).            */
int unocg_set_uno_weights(unocg_ctx* ctx, int kind, const void* w, int dtype, double spd_eps);

/* UNO weights in the paper's layout (Eq. (fnocg-operator), Eq. (fnocg-parametrization)):
   Q(k) = psi(w_0) + psi(w_i) if k is the i-th mode of K_M = [-M,M]^2 x [0,M] minus {0}
   (periodic row of Table (fnocg-mode-selection-2d); order: k1 slowest from -M, then k2 from
   -M, then k3 from 0), else psi(w_0).  w: host array [1 + n_modes][C] of `dtype`,
   n_modes = (2M+1)^2 (M+1) - 1; requires 2M+1 <= N1, 2M+1 <= N2, 2M <= N3, else
   UNOCG_ERR_INVALID_ARG.  Then as unocg_set_uno_weights (symmetrization of the
   self-conjugate planes, safety check with spd_eps, BF16 copy).                          */
int unocg_set_uno_modes(unocg_ctx* ctx, int M, const void* w, int dtype, double spd_eps);

/* Copy the expanded weights Q(k) of `instance` (unique entries [N1][N2][N3/2+1][C], paper's
   order, FP64, after the safety check and symmetrization) to host memory `out`.            */
int unocg_get_uno_weights(unocg_ctx* ctx, int instance, double* out);

/* Solve all (instance, load) systems K u = f to tolerance (Algorithm 1 / 2), then compute the
   zero-mean fluctuations and the averaged flux / stress.  Blocks until done.               */
int unocg_solve(unocg_ctx* ctx, const unocg_solve_opts* opts, unocg_solve_info* info);
/* Enqueue the same work on the context stream without waiting; read results with
   unocg_solve_wait.                                                                         */
int unocg_solve_async(unocg_ctx* ctx, const unocg_solve_opts* opts);
int unocg_solve_wait(unocg_ctx* ctx, unocg_solve_info* info);

/* Zero-mean fluctuation of one (instance, load): host double [N1*N2*N3*c], interleaved.    */
int unocg_get_fluctuation(unocg_ctx* ctx, int instance, int load, double* out);
/* Same into caller-owned device memory, layout [c][N1][N2][N3] (double).                   */
int unocg_get_fluctuation_dev(unocg_ctx* ctx, int instance, int load, double* out_dev, void* stream);

/* Averaged flux / stress per load (Sec. 6): out[B][dim][n_loads], out[b][i][l] = <C (eps_bar_l
   + eps(u_l))>_i (thermal dim 3: kappa_eff g_bar = -<q>; elastic dim 6, Mandel).  With the
   unit loads in order this is the effective tensor, row-major.                             */
int unocg_get_effective_tensor(unocg_ctx* ctx, double* out);

/* Derivative of the energy averages W_lm = <(eps_bar_l + eps(u_l)) . C (eps_bar_m + eps(u_m))>
   with respect to the phase properties (kappa_p; or E_p, nu_p): out[B][n_props][L][L].  K is
   self-adjoint, so the adjoint states are the forward solutions; needs a converged solve.  */
int unocg_get_sensitivity(unocg_ctx* ctx, double* out);

/* Solve several contexts together (e.g. one per grid size of an uneven batch; Sec. 5.5,
   batching).  With the graph driver (use_graph 1 or 3) the solves of all contexts are
   captured as parallel branches of ONE CUDA graph and launched once: each branch is one
   context's set-up, its device-resident WHILE loop over all its (instance, load) pairs with
   their per-pair convergence flags (a converged pair's blocks return at once) and its
   post-processing; each branch ends when its last pair converges.  The graph is kept for
   later calls with the same contexts and options (it is rebuilt after any change that
   invalidates a context's own graph, and dropped when a context is destroyed).  It runs after
   the work already enqueued on every context's stream, and their later work runs after it.
   The host-driven and persistent drivers run the contexts' solves concurrently on their own
   streams.  A context may appear once.  Blocks until all are done; infos may be NULL or hold
   n_ctx entries.                                                                           */
int unocg_batch_solve(int n_ctx, unocg_ctx* const* ctxs, const unocg_solve_opts* opts,
                      unocg_solve_info* infos);

/* Timing of the hot-path kernels: runs the first `reps` CG iterations of a fresh solve with the
   options `opts`, each kernel launched on its own between two CUDA events on the context stream,
   and writes the mean milliseconds per launch to ms_out[0..3]: UNO: [axis-1 pass with block
   multiply, inverse plane pass, K d, residual update + forward plane pass]; Jacobi / none:
   [direction update, (unused, 0), K d, residual update].  Invalidates the last solution.     */
int unocg_profile_iteration(unocg_ctx* ctx, const unocg_solve_opts* opts, int reps, double* ms_out, int n_out);

/* ---------------------------------------------------------------- standalone UNO operator
   P = T^H Q T on a batch of fields, for training (Sec. 5.3, Algorithm 3).                  */
typedef struct unocg_uno unocg_uno;
/* Grid rules as unocg_create; the backward pass holds four line buffers, which bounds
   n1 <= 218 (c = 1) and n1 <= 145 (c = 3).                                                 */
int unocg_uno_create(unocg_uno** out, int c, int n1, int n2, int n3);
void unocg_uno_destroy(unocg_uno* op);
const char* unocg_uno_last_error(const unocg_uno* op);
/* theta_dev: device float [N1][N2][N3/2+1][C], mapped through psi on every call.            */
int unocg_uno_set_theta_dev(unocg_uno* op, const float* theta_dev, void* stream);
/* The paper's layout instead (see unocg_set_uno_modes): w_dev device float
   [1 + n_modes][C]; the backward then returns dL/dw in the same layout.  The operator keeps
   the pointer: w_dev must stay valid until the next set call.                              */
int unocg_uno_set_modes_dev(unocg_uno* op, int M, const float* w_dev, void* stream);
/* s = P r for a batch: r_dev, s_dev device float [batch][c][N1][N2][N3].                    */
int unocg_uno_apply_dev(unocg_uno* op, int batch, const float* r_dev, float* s_dev, void* stream);
/* Backward of s = P r: gr = P gs (P is self-adjoint) and gtheta = dL/dtheta (device float,
   [N1][N2][N3/2+1][C], or [1 + n_modes][C] after unocg_uno_set_modes_dev; overwritten) from
   dL/dQ(k) = sum_b w_k Re(conj(T gs_b) (T r_b)^T).                                         */
int unocg_uno_backward_dev(unocg_uno* op, int batch, const float* r_dev, const float* gs_dev,
                           float* gr_dev, float* gtheta_dev, void* stream);
/* Features of the second-order training (Sec. 5.4, Eq. (features-c-1), Eq. (features-c-2) and
   the c = 3 features of App. C): for a batch of right-hand sides f_dev and solutions u_dev
   (device float [batch][c][N1][N2][N3]) adds, per half-grid mode k and unique entry (i, j) of
   the paper's order (C = 1 or 6),
     sum_b w_k Re(conj(F_i) F_j) [+ Re(conj(F_j) F_i) for i != j]   to ab_dev[0 .. nh*C) and
     sum_b w_k Re(conj(U_i) F_j) [+ Re(conj(U_j) F_i) for i != j]   to ab_dev[nh*C .. 2 nh*C)
   (layout [nh][C] each; F = T f_b, U = T u_b unitary; w_k the half-grid multiplicity;
   nh = N1 N2 (N3/2+1)); accumulate = 0 zeroes ab_dev first.  The features of the paper are
   a = first / n_samples and b = 2 second / n_samples.  The weights set on the operator are
   not used.                                                                                */
int unocg_uno_features_dev(unocg_uno* op, int batch, const float* f_dev, const float* u_dev, float* ab_dev,
                           int accumulate, void* stream);

/* ---------------------------------------------------------------- second-order training
   Algorithm 4 (Sec. 5.4; c = 3: App. C) on the device for the paper's bypass-plus-modes weights
   w = [w_0; w_1 .. w_n] (psi(w) = w^2 for c = 1; L L^T with L lower triangular holding the
   parameters for c = 2 (Eq. (local-param-2)) and c = 3 (App. B.1); entries in the paper's
   order).  Per learned mode k the loss is (1/2) v^T H_k v - b_k . v in the unique block
   entries v = psi(w_0) + psi(w_k), H_k[e][f] = sum_m a_{k,m} (E_e E_f + E_f E_e)_m from the
   features a_k (Eq. (features-c-1), Eq. (features-c-2), App. C); all other modes see psi(w_0)
   and enter through the sums a_rest, b_rest of their features.  Each Newton-Raphson step
   solves the arrow-shaped Hessian (bypass row / column plus one P x P block per mode, P =
   c(c+1)/2) by its Schur complement in O(n), with Levenberg-Marquardt damping when a step
   does not lower the loss.  The object owns its device buffers and its stream.             */
typedef struct unocg_newton unocg_newton;
/* c in {1, 2, 3}; n_modes >= 0 learned modes.                                              */
int unocg_newton_create(unocg_newton** out, int c, int n_modes);
void unocg_newton_destroy(unocg_newton* op);
const char* unocg_newton_last_error(const unocg_newton* op);
/* Host arrays: a_k, b_k [n_modes][C] (the features at the learned modes, multiplicities of
   the conjugate modes included), a_rest, b_rest [C] (their sums over all other modes).
   Non-finite values return UNOCG_ERR_INVALID_ARG.                                           */
int unocg_newton_set_features(unocg_newton* op, const double* a_k, const double* b_k, const double* a_rest,
                              const double* b_rest);
/* Runs up to max_steps steps from w0 [1 + n_modes][C] (host), stopping when the loss changes by
   at most tol * max(1, |loss|); writes the weights to w_out and the loss history (without the
   constant delta; first entry the loss of w0) to hist, of capacity *n_hist on entry and
   length on return (hist may be NULL).                                                     */
int unocg_newton_run(unocg_newton* op, const double* w0, int max_steps, double tol, double* w_out, double* hist,
                     int* n_hist);

/* ---------------------------------------------------------------- operator-level entry points
   Device-pointer access to single steps of the hot path, on a context's microstructure and
   properties (instance 0 .. B-1 via `instance`).  Fields are double [c][N1][N2][N3].        */
/* p = K d (Sec. 4.1, matrix-free), in FP64.                                                 */
int unocg_apply_K_dev(unocg_ctx* ctx, int instance, const double* d_dev, double* p_dev, void* stream);
/* p = K d (Sec. 4.1, matrix-free) in FP32 with the kernel of the mixed-precision loop: for
   thermal problems the kernel of unocg_set_ku_tile where the grid allows it.
   Fields are float [c][N1][N2][N3], caller-owned device memory, enqueued on `stream`.         */
int unocg_apply_K32_dev(unocg_ctx* ctx, int instance, const float* d_dev, float* p_dev, void* stream);
/* s = P r with the context's current UNO weights (Algorithm 2, transform / block multiply /
   inverse transform), in FP64.                                                             */
int unocg_apply_uno_dev(unocg_ctx* ctx, int instance, const double* r_dev, double* s_dev, void* stream);
/* s = P r as unocg_apply_uno_dev, without allocating: the two spectra live in a static device
   scratch of the library (2 x 8 MiB), not in memory from cudaMallocAsync.  The paper has no
   counterpart; this serves callers that cannot allocate when they apply the preconditioner
   (device memory held by another allocator, latency-bound loops, fixed footprints).
   Limit: c*N1*N2*(N3/2+1) <= 524288 (e.g. 64^3 elastic); larger grids return
   UNOCG_ERR_INVALID_ARG and launch nothing.  The UNO weights must already be prepared on the
   device (unocg_set_uno_weights after unocg_set_phase_properties), else UNOCG_ERR_STATE.
   The first call in a CUDA context of a device looks up the scratch address
   (cudaGetSymbolAddress) and caches it under that context's id; a context created again
   (e.g. after cudaDeviceReset) is looked up anew.  Make the first call of each context before
   any stream capture.  No part of the scratch needs to start at zero.
   Every call on a device uses the same scratch: calls whose work overlaps in time (different
   streams, contexts or host threads without ordering between them) race and corrupt each
   other's results; order them on one stream or with events.                               */
int unocg_apply_uno_dev_noalloc(unocg_ctx* ctx, int instance, const double* r_dev, double* s_dev, void* stream);
/* Right-hand side f of load `load` (Sec. 6): double [c][N1][N2][N3].                        */
int unocg_rhs_dev(unocg_ctx* ctx, int instance, int load, double* f_dev, void* stream);

/* ---------------------------------------------------------------- Dirichlet boundary conditions
   The fluctuation vanishes on the boundary of the cell (Sec. 6.1 / 6.2, "Dirichlet BC"; also
   called kinematic uniform BC): on an N1 x N2 x N3 voxel grid only the M_a = N_a - 1 interior
   nodes per axis are free (Sec. 4.1), and the unitary transform of the UNO preconditioner is
   the orthonormal sine transform (DST-I) on every component, real, with no conjugate modes
   (Dirichlet row of Table (fnocg-mode-selection-2d)).  Mode k = (k1, k2, k3), 0 <= k_a < M_a,
   is the sine basis vector sqrt(2/N_a) sin(pi (j+1)(k_a+1)/N_a) per axis.
   Same conventions as the periodic context: voxel edge h = L0 / N1, phase labels per voxel
   [B][N1][N2][N3], loads, properties, status codes, unocg_solve_opts / unocg_solve_info.
   Fields on the free nodes: device layout [c][M1][M2][M3] (double); host I/O interleaved
   [M1*M2*M3*c].  No zero-mean projection (the Dirichlet fluctuation is unique).
   Limits: 2 <= N_a <= 512, each N_a of the form 2^a 3^b 5^c.  use_graph: 0 host-driven
   loop (one residual check read back per iteration), any other value one CUDA graph with
   conditional nodes; flexible CG is not available (UNOCG_ERR_INVALID_ARG).
   MIXED precision: FP32 fields, transforms, K.u and FP32 weights; FP64 solution, reductions
   and residual replacement r = f - K u, with the triggers of unocg_solve_opts.             */
typedef struct unocg_dir unocg_dir;

int unocg_dir_create(unocg_dir** out, int physics, int batch, int n1, int n2, int n3, double L0);
/* Mixed boundary conditions (Sec. 6.2; Table (fnocg-mode-selection-2d), mixed row): bc[a] = 1
   gives axis a Dirichlet faces, bc[a] = 0 makes the fluctuation periodic across them (at least
   one axis Dirichlet; all periodic is unocg_create).  A periodic axis has N_a free nodes and
   the Fourier transform as the UNO's transform along it, the paper's FFT^x o DST^y; the library
   applies it through Hartley passes, which give the same operator T^H Q T for real blocks with
   Q(-k) = Q(k) (k negated on every periodic axis): BLOCKS / THETA weights are made even that
   way when set, and with two periodic axes a pass converts the separable Hartley spectrum to
   the two-dimensional one around the block multiply.  unocg_dir_create is bc = {1, 1, 1}.
   Reference weights: Q(k) = (t_k^H K_ref t_k)^-1 with t_k the Fourier x sine basis vector.
   The mode layout (unocg_dir_set_uno_modes) needs bc = {1, 1, 1}.                          */
int unocg_dir_create_bc(unocg_dir** out, int physics, int batch, int n1, int n2, int n3, double L0,
                        const int* bc);
void unocg_dir_destroy(unocg_dir* ctx);
const char* unocg_dir_last_error(const unocg_dir* ctx);
int unocg_dir_set_stream(unocg_dir* ctx, void* stream);
int unocg_dir_set_microstructure(unocg_dir* ctx, const uint8_t* phase, int n_phases);
int unocg_dir_set_phase_properties(unocg_dir* ctx, const double* props);
int unocg_dir_set_macro_load(unocg_dir* ctx, int n_loads, const double* loads);
/* UNO weights on the sine modes.  UNOCG_W_REFERENCE_MEDIUM (per instance, `w` unused):
   Q(k) = (t_k^T K_ref t_k)^-1, the inverse of the c x c diagonal block of the sine-transformed
   stiffness of the homogeneous medium with the arithmetic-mean conductivity / Lame constants
   (exact inverse of that operator for c = 1; for c = 3 the transform does not decouple the
   components and the off-diagonal blocks vanish on the diagonal k).  UNOCG_W_BLOCKS /
   UNOCG_W_THETA: [M1][M2][M3][C] unique entries / psi parameters (shared by all instances).
   Safety check lambda_min(Q(k)) > spd_eps on every mode (also after rounding to FP32 for the
   mixed path), else UNOCG_ERR_NOT_SPD.                                                      */
int unocg_dir_set_uno_weights(unocg_dir* ctx, int kind, const void* w, int dtype, double spd_eps);
/* The paper's Dirichlet layout: Q(k) = psi(w_0) + psi(w_i) for the i-th mode of
   [0, 2M]^3 (k1 slowest, then k2, then k3), psi(w_0) elsewhere; w: [1 + (2M+1)^3][C].
   Requires 2M + 1 <= M_a on every axis.                                                    */
int unocg_dir_set_uno_modes(unocg_dir* ctx, int M, const void* w, int dtype, double spd_eps);
/* Q of `instance` (unscaled unique entries [M1][M2][M3][C], FP64) to host memory `out`.      */
int unocg_dir_get_uno_weights(unocg_dir* ctx, int instance, double* out);
int unocg_dir_solve(unocg_dir* ctx, const unocg_solve_opts* opts, unocg_solve_info* info);
int unocg_dir_solve_async(unocg_dir* ctx, const unocg_solve_opts* opts);
int unocg_dir_solve_wait(unocg_dir* ctx, unocg_solve_info* info);
/* Fluctuation on the free nodes: host interleaved [M1*M2*M3*c] / device [c][M1][M2][M3].    */
int unocg_dir_get_fluctuation(unocg_dir* ctx, int instance, int load, double* out);
int unocg_dir_get_fluctuation_dev(unocg_dir* ctx, int instance, int load, double* out_dev, void* stream);
/* Averaged flux / stress [B][dim][n_loads] over all voxels, as unocg_get_effective_tensor.  */
int unocg_dir_get_effective_tensor(unocg_dir* ctx, double* out);
/* q = K p and s = T^T Q T r (FP64, device [c][M1][M2][M3]) for one instance.                 */
int unocg_dir_apply_K_dev(unocg_dir* ctx, int instance, const double* p_dev, double* q_dev, void* stream);
int unocg_dir_apply_uno_dev(unocg_dir* ctx, int instance, const double* r_dev, double* s_dev, void* stream);
/* Pass engines of one precision (UNOCG_FP64 / UNOCG_MIXED): plane_engine 0 register plane
   passes (Dirichlet faces everywhere, N2 = N3 a power of two <= 128), 1 shared-memory plane
   passes (the plane fits a block), 2 separate axis-3 and axis-2 passes; line_engine 0 register
   axis-1 pass with the block multiply (Dirichlet faces everywhere, c = 1, N1 a power of two
   <= 128), 1 shared-memory pass.  UNOCG_ERR_INVALID_ARG when not applicable.  Defaults at
   creation: the register engines where they apply, else shared-memory planes up to 110 KB.  */
int unocg_dir_set_tuning(unocg_dir* ctx, int precision, int plane_engine, int line_engine);
/* Autotuner: times `reps` solves of `opts` (after one warm-up solve each) for every applicable
   engine pair of opts->precision, writes the mean ms to times[plane_engine * 2 + line_engine]
   (double[6]; NaN where not applicable) and keeps the fastest pair.  Needs the inputs set.   */
int unocg_dir_autotune(unocg_dir* ctx, const unocg_solve_opts* opts, int reps, double* times);

#ifdef __cplusplus
}
#endif

#endif /* UNOCG_H */
