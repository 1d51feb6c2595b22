/*
 * bhem.h - C ABI of the GB300 (sm_103a) BHEM shell library (libbhem.so).
 *
 * Bicubic Hermite element method for Kirchhoff-Love thin shells (arXiv 2312.14839): per-patch
 * 4x4 Gauss-point evaluation of the membrane + bending energy, its 48-DOF gradient and 48x48
 * Hessian, assembly into a 12x12-block sparse (BSR) matrix, and implicit-Euler Newton steps
 * whose linear systems are solved by block-Jacobi PCG. All compute runs in CUDA kernels of
 * this library; there is no CPU fallback.
 *
 * Conventions used by every entry point
 *  - Node arrays hold 12 doubles per node, [x, x_,1, x_,2, x_,12] (each in R^3), the
 *    generalised coordinates of Sec. 4.1 (Eq. hermite): derivative DOFs are derivatives with
 *    respect to the global parameters xi^1, xi^2. Node (i, j) has id j * n1 + i, i along xi^1,
 *    n1 = nu + 1 (nu when periodic in u), n2 = nv + 1 (nv when periodic in v).
 *  - Patch (pu, pv) has id pv * nu + pu; its corners 00, 10, 01, 11 are nodes (pu+p, pv+q)
 *    (indices wrap when periodic, Sec. 4.2). Patch-local DOF order is corner * 12 + kind * 3 +
 *    component, kind in {x, x_,1, x_,2, x_,12}.
 *  - "device" pointers are CUDA device (or managed) memory owned by the caller. Entry points
 *    that accept "host or device" detect the kind with cudaPointerGetAttributes and stage host
 *    buffers through library-owned device memory.
 *  - All GPU work is enqueued on the stream given to shell_create (a cudaStream_t passed as
 *    void*; NULL means the legacy default stream). Entry points that return host values
 *    (stats, flags) synchronise that stream; the others are asynchronous.
 *  - Errors are returned as shell_status codes, never thrown. shell_last_error() gives a
 *    thread-local message for the last failing call. Outputs are unspecified after an error,
 *    except where stated.
 */
#ifndef BHEM_H
#define BHEM_H

#if defined(__GNUC__)
#define SHELL_API __attribute__((visibility("default")))
#else
#define SHELL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct shell_s shell_t;

typedef enum {
  SHELL_OK = 0,
  SHELL_ERR_ARG = 1,            /* invalid argument (NULL, size, enum value)                   */
  SHELL_ERR_CUDA = 2,           /* a CUDA runtime call failed                                   */
  SHELL_ERR_OOM = 3,            /* device allocation failed                                     */
  SHELL_ERR_DEGENERATE = 4,     /* |a_1 x a_2| <= 1e-300 at a Gauss point (no normal, Sec. 3.1) */
  SHELL_ERR_NONFINITE = 5,      /* a non-finite energy, gradient or residual was produced      */
  SHELL_ERR_NOT_CONVERGED = 6,  /* Newton hit newton_max; q, v hold the last iterate            */
  SHELL_ERR_LINESEARCH = 7,     /* no step satisfied the Armijo test in 20 trials               */
  SHELL_ERR_INDEFINITE = 8,     /* negative curvature persisted beyond tau = 1e4                */
  SHELL_ERR_TIMEOUT = 9         /* a bounded device-side wait expired (results of the call are void) */
} shell_status;

/* Patch grid (Sec. 4.1, Fig. regular; periodic boundary conditions of Sec. 4.2). dxi1, dxi2
   are the parameter extents of one patch (uniform grid). */
typedef struct {
  int nu, nv;
  int periodic_u, periodic_v;
  double dxi1, dxi2;
} shell_grid;

/* Material (Sec. 3.3): Young's modulus Y, Poisson ratio nu, thickness h, density rho.
   lambda = Y nu / (1 - nu^2), mu = Y / (2 (1 + nu)). */
typedef struct {
  double young, poisson, thickness, density;
} shell_material;

enum { SHELL_PREC_FP64 = 0, SHELL_PREC_MIXED = 1 };
enum { SHELL_HESS_EXACT = 0, SHELL_HESS_PSEUDO = 1 };
enum { SHELL_ASM_ATOMIC = 0, SHELL_ASM_COLOR = 1 };
enum { SHELL_SPMV_AUTO = 0, SHELL_SPMV_PLAIN = 1, SHELL_SPMV_TMA = 2 };
enum { SHELL_SOLVER_PCG = 0, SHELL_SOLVER_DIRECT = 1 };

/* precision: SHELL_PREC_FP64 = every quantity in FP64; SHELL_PREC_MIXED = element Hessian,
   BSR values, SpMV and block-Jacobi in FP32, while the energy, gradient/residual, line-search
   energy differences and PCG dot products stay FP64.
   hessian: exact (App. B.2) or the pseudo Hessian of App. B.2 without the second derivative of
   beta. assembly: atomic scatter or colour-ordered scatter of the element blocks (shell_grid_colours).
   spmv (SHELL_PREC_MIXED only): the FP32 BSR SpMV of shell_spmv and of PCG. SHELL_SPMV_PLAIN:
   one CTA per 8 block rows, blocks loaded straight into registers. SHELL_SPMV_TMA: a persistent
   kernel that streams each CTA's row groups into a shared-memory ring with bulk asynchronous
   copies (cp.async.bulk + mbarrier); rejected when 8 block rows of the longest row do not fit.
   SHELL_SPMV_AUTO: plain (the faster of the two on GB300). Both give bit-identical results.
   Batches ignore this field.
   solver: the linear solver of shell_newton_step. SHELL_SOLVER_PCG: block-Jacobi PCG (the
   default). SHELL_SOLVER_DIRECT: a comparator for the paper's direct LDL^T solve (Sec. 6.1): the
   assembled matrix plus the regulariser, prescribed DOFs as identity rows, is factorised in FP64
   by a banded Cholesky over the node rows of the grid (the matrix is block tridiagonal over the
   rows of one grid direction, so the factor has no fill-in outside those bands), with hand-
   written kernels; a pivot that is not positive multiplies the regulariser by 10 as negative
   curvature does for PCG. The rows run along a direction that is not periodic (shells periodic in
   both directions are rejected) and hold at most 4096 unknowns; the first direct step allocates
   16 rows B^2 bytes (B unknowns per row) for the factor. The pcg_* fields of shell_step_params
   are ignored. Batches ignore this field. */
typedef struct {
  int precision;
  int hessian;
  int assembly;
  int spmv;
  int solver;
} shell_options;

/* One implicit-Euler step (Eq. implicit, Sec. 6.1). Newton stops when |g_free| <= newton_rtol *
   |g_free(zero guess)|; PCG stops when |r| <= pcg_rtol |b| or after pcg_max iterations, or
   runs exactly pcg_fixed_iters iterations when that is > 0. tau_carry (>= 0) is the regulariser
   level carried into the step: its first Newton iteration starts at tau_carry / 10, as later
   iterations start at a tenth of the previous one's (pass the previous step's
   shell_step_stats.tau_final to carry it across steps, 0 for none). */
typedef struct {
  double dt;
  double gravity[3];
  double newton_rtol;
  int newton_max;
  double pcg_rtol;
  int pcg_max;
  int pcg_fixed_iters;
  double tau_carry;
} shell_step_params;

typedef struct {
  int newton_iters;       /* Newton updates applied                                         */
  int pcg_iters_total;    /* PCG iterations over all solves (regularised restarts included) */
  int ls_backtracks;      /* rejected line-search trials                                    */
  int regularizations;    /* solves with a diagonal shift tau D > 0 (Sec. 6.1 regulariser)  */
  int status;             /* shell_status of the step                                       */
  int diag_fixes;         /* free diagonal entries A_ii <= 0 replaced (regulariser, local)  */
  double res0;            /* |g_free| at the zero guess                                     */
  double res_final;       /* |g_free| at the returned state                                 */
  double tau_final;       /* regulariser level of the last accepted solve (0: none)         */
} shell_step_stats;

typedef struct {
  int n_nodes, n_patches, n_blocks, n_dof;
} shell_info_t;

/* Creates a shell on the current CUDA device. rest_dofs: host or device, [n_nodes * 12] FP64,
   the reference configuration (copied). Builds the BSR pattern (Sec. 4.3 "Properties of the mass
   matrix": two nodes couple iff they share a patch), the consistent mass M (Eq. mass) and the
   gravity load factors (Sec. 4.3), all with the 4x4 Gauss rule of App. A.2. *out receives an
   opaque handle owned by the caller (release with shell_destroy). stream: cudaStream_t. */
SHELL_API shell_status shell_create(const shell_grid* grid, const shell_material* material,
                          const double* rest_dofs, const shell_options* options, void* stream,
                          shell_t** out);

/* Frees every device buffer of the shell (synchronises its stream first). NULL is allowed. */
SHELL_API shell_status shell_destroy(shell_t* shell);

/* Sizes of the shell (host output). */
SHELL_API shell_status shell_info(const shell_t* shell, shell_info_t* info);

/* Budget of the library's bounded device-side waits on this shell: the grid barriers of the
   persistent mixed-precision PCG (one cooperative launch per solve; selected by the environment
   variable BHEM_PCG_LOOP=persistent when the shell is created), the mbarrier waits of
   the bulk-copy SpMV (SHELL_SPMV_TMA) and those of the tensor-core element pass (mixed
   precision; each CTA waits for the MMAs it commits) poll at most `polls` times before the
   waiting CTA gives up. The call then returns SHELL_ERR_TIMEOUT (its results are void): a CTA
   that gave up at a barrier leaves the kernel, the others give up at their next barrier, and the
   bulk-copy SpMV and the tensor-core element pass still wait, with the default budget, for the
   copies or MMAs they have issued (then free their tensor memory), so that the device stays
   usable.
   polls < 0 restores the default (2^20 polls); 0 makes every such wait expire at once (a test
   of the timeout path). Synchronises the shell's stream and drops its cached PCG graphs. No paper
   counterpart (a watchdog of this implementation). */
SHELL_API shell_status shell_set_wait_budget(shell_t* shell, int polls);

/* Colour classes of the colour-ordered assembly (SHELL_ASM_COLOR, Sec. 4.3 "Properties of the
   mass matrix": two patches add into the same block iff they share a node). colour: host
   [nu * nv], receives colour[pv * nu + pu] in [0, 9): pu % 2 + 3 (pv % 2), except that along a
   periodic direction with an odd patch count the seam patch (index n - 1) takes colour 2 there,
   so that it does not share the colour of patch 0 across the wrap. Patches of one colour share
   no node, and their element blocks are added with plain (non-atomic) writes, one launch per
   colour. Host computation only: needs no GPU. */
SHELL_API shell_status shell_grid_colours(const shell_grid* grid, int* colour);

/* Element-by-element evaluation, unassembled (App. B): for every patch p, energy_p[p] (FP64),
   grad_p[p * 48 + l] (FP64) and hess_p[p * 2304 + l * 48 + m] (FP32 when precision is
   SHELL_PREC_MIXED, FP64 when SHELL_PREC_FP64), l, m patch-local DOF indices. q: device
   [n_nodes * 12]. Any output may be NULL. Asynchronous. The FP32 Hessian's contraction
   K = sum_g Phi_g^T M_g Phi_g (App. B.2) runs on the tensor cores (TF32 head-and-tail products,
   FP32 accuracy) unless the environment variable BHEM_ELEMENT=ffma was set when the shell was
   created (then on the FP32 FMA pipe); this applies to every FP32 Hessian of the shell. */
SHELL_API shell_status shell_element_egh(shell_t* shell, const double* q, int precision, double* energy_p,
                               double* grad_p, void* hess_p);

/* Assembled elastic energy V_e (device, 1 double), elastic gradient dV_e/dq (device
   [n_nodes * 12], App. B.1) and, when want_hessian != 0, the BSR matrix K + mass_scale * M
   (App. B.2 Hessian, Eq. mass) into the shell's internal BSR (read with shell_get_bsr).
   energy or grad may be NULL. Asynchronous. */
SHELL_API shell_status shell_energy_grad_hess(shell_t* shell, const double* q, double mass_scale,
                                    double* energy, double* grad, int want_hessian);

/* Internal BSR arrays (device, valid until the next call that assembles or shell_destroy):
   row_ptr[n_nodes + 1], col[n_blocks] (sorted per row), val[n_blocks * 144] 12x12 row-major
   blocks, FP32 (*val_is_fp64 = 0) or FP64 (*val_is_fp64 = 1). Both triangles are stored. */
SHELL_API shell_status shell_get_bsr(shell_t* shell, const int** row_ptr, const int** col,
                           const void** val, int* val_is_fp64);

/* Consistent mass as 4x4 scalar blocks on the same pattern (device, [n_blocks * 16], M =
   mass (x) I3 per node pair, Eq. mass) and gravity load factors (device, [n_nodes * 4],
   F = factors (x) g, Sec. 4.3). */
SHELL_API shell_status shell_get_mass(shell_t* shell, const double** mass_blocks,
                            const double** gravity_factors);

/* Block-Jacobi PCG on the currently assembled BSR A: solves (A + tau D) x = rhs, D diagonal with
   D_ii = mean of |A_jj| over the free DOFs j of DOF i's kind (x, x_,1, x_,2 or x_,12), with
   fixed DOFs (mask != 0) held at zero (identity rows/columns). rhs, x: device [n_dof];
   fixed_mask: device [n_dof] or NULL. Runs until |r| <= rtol |rhs| or max_iter, or exactly
   fixed_iters (> 0) iterations. *iters receives the iterations done, *neg_curv 1 when
   p^T A p <= 0 stopped it. Synchronises. */
SHELL_API shell_status shell_pcg_solve(shell_t* shell, const unsigned char* fixed_mask, double tau,
                             const double* rhs, double* x, double rtol, int max_iter,
                             int fixed_iters, int* iters, int* neg_curv);

/* y = A x with the currently assembled BSR A (the product inside every PCG iteration of
   Sec. 6.1's linear solve; FP32 arithmetic with FP32 accumulation per row chunk when the shell
   is SHELL_PREC_MIXED, FP64 otherwise). x, y: device [n_dof], x 16-byte (SHELL_ERR_ARG
   otherwise) and y 8-byte aligned.
   x_is_fp32 != 0 (SHELL_PREC_MIXED shells only): x and y are FP32 and the call is one launch of
   the kernel every PCG iteration runs. Otherwise x and y are FP64 (a mixed shell converts
   through its own FP32 vectors: three launches). No mask, no regulariser. Asynchronous. */
SHELL_API shell_status shell_spmv(shell_t* shell, const void* x, int x_is_fp32, void* y);

/* One implicit-Euler step (Eq. implicit) by Newton with line search (Sec. 6.1):
   minimises Pi(q) = (q - y)^T M (q - y) / (2 dt^2) + V_e(q) - F^T q, y = q^n + dt v^n, over the
   free DOFs; fixed DOFs (fixed_mask[k] != 0) take q_fixed[k] (Sec. 4.2 positional constraints).
   Each Newton direction solves (A' + tau D) d = -g, A = M / dt^2 + K (Sec. 6.1's diagonal
   regulariser): A' replaces every free diagonal entry A_ii <= 0 of DOF kind k by
   max(-A_ii, 1e-8 D_k) (D_k = mean |A_ii| over the free DOFs of kind k; the assembled matrix
   read by shell_get_bsr afterwards holds A'); tau starts at a tenth of the previous iteration's
   tau (at the first iteration, of params->tau_carry; 0 when a tenth is below 1e-8); negative curvature
   met by the solve multiplies tau by 10 (at least 1e-8) and restarts it; beyond tau = 1e4 the
   step returns SHELL_ERR_INDEFINITE. The line search is Armijo (c1 = 1e-4) from alpha = 1 with
   the quadratic, then cubic, interpolant's minimiser clamped to [0.1, 0.5] of the last trial.
   q, v: [n_dof] FP64 in/out (host or device); fixed_mask [n_dof] uint8 and q_fixed [n_dof]
   (host or device, may be NULL together); warm_start [n_dof] or NULL: initial Newton iterate
   (the residual reference stays the zero guess q^n). stats: host. Returns stats->status. On
   SHELL_ERR_NOT_CONVERGED q and v hold the last iterate; on other errors they are unchanged. */
SHELL_API shell_status shell_newton_step(shell_t* shell, const shell_step_params* params,
                               const unsigned char* fixed_mask, const double* q_fixed,
                               double* q, double* v, const double* warm_start,
                               shell_step_stats* stats);

/* Elastic energy and gradient without any device allocation. This is an interface addition of
   this library; the paper has no counterpart. It computes the same quantities as the energy
   and grad outputs of shell_energy_grad_hess (Sec. 3.3 energy, App. B.1 gradient), for
   callers that must not allocate device memory while they run: applications whose device
   memory belongs entirely to their own pool allocator (cudaMalloc would fail or escape its
   accounting), latency-bound loops that cannot afford the device-wide synchronisation a
   cudaMalloc/cudaFree may cause, and plug-ins that receive a fixed memory budget from their
   host. No shell object is needed: the patch topology comes from grid, the shape table and the
   rest geometry are computed from rest_dofs on every call.
   Arguments: grid, material (host); rest_dofs, q: device [n_nodes * 12] FP64 (caller-owned,
   read only); energy: device, 1 double (overwritten); grad: device [n_nodes * 12] FP64 or NULL
   (overwritten); stream: cudaStream_t or NULL. Asynchronous: enqueues a memset of the ticket
   (and of grad) and two kernels on stream, calls no cudaMalloc, cudaFree or allocating library
   routine.
   Scratch: one file-scope device array of about 141 KB (per-CTA energy sums, the shape table and
   a counter), present on every GPU that loads the library until the process exits. Grids of
   more than 131072 patches are rejected with SHELL_ERR_ARG. The first call on a device looks up
   the array's device address (cudaGetSymbolAddress) with that device current; make that first
   call before any stream capture. The address is kept for the life of the process: after
   cudaDeviceReset on a device (which unloads the library's module there) this entry point must
   not be called on that device again. All calls share the array and each call resets the counter it
   needs: calls whose work overlaps on the GPU (other streams, other host threads on the same
   device) race on it and must be serialised by the caller. A degenerate geometry gives a
   non-finite energy instead of an error code. */
SHELL_API shell_status shell_energy_grad_noalloc(const shell_grid* grid, const shell_material* material,
                                                 const double* rest_dofs, const double* q,
                                                 double* energy, double* grad, void* stream);

/* ---------------------------------------------------------------------------------------------
   Batches: many independent shells of uneven sizes and materials stepped together (every shell
   runs its own Newton to its own residual tolerance, with the same policies as
   shell_newton_step). Shells are concatenated: node k of shell s is node node_offsets[s] + k of
   the batch, and q, v, masks are the shells' arrays one after the other. Precision is
   SHELL_PREC_MIXED. Each phase of a Newton iteration is one launch over all shells; PCG
   iterations are replayed from a CUDA graph.
   --------------------------------------------------------------------------------------------- */
typedef struct shell_batch_s shell_batch_t;

typedef struct {
  int n_shells, n_nodes, n_patches, n_blocks, n_dof;
  int patches_per_item;   /* patches per element work item (set by shell_batch_autotune)   */
  int assembly;           /* SHELL_ASM_ATOMIC or SHELL_ASM_COLOR                           */
  long long kernel_launches;
} shell_batch_info_t;

/* Creates a batch of n_shells shells (grids[s], materials[s]; rest_dofs: host or device, the
   shells' rest DOFs concatenated). options may be NULL (mixed precision, atomic assembly); a
   precision other than SHELL_PREC_MIXED is rejected. Every shell needs at least 16 nodes.
   stream: cudaStream_t (NULL: the batch creates its own blocking stream). */
SHELL_API shell_status shell_batch_create(int n_shells, const shell_grid* grids,
                                          const shell_material* materials, const double* rest_dofs,
                                          const shell_options* options, void* stream,
                                          shell_batch_t** out);
SHELL_API shell_status shell_batch_destroy(shell_batch_t* batch);
/* Sizes and the current tuning; node_offsets (host, [n_shells + 1]) may be NULL. */
SHELL_API shell_status shell_batch_info(const shell_batch_t* batch, shell_batch_info_t* info,
                                        int* node_offsets);
/* Times the element Hessian assembly at the state q (device [n_dof]) for patches-per-item
   4, 8, 16, 32 and atomic / colour-ordered scatter (repeats timed runs each, CUDA events) and
   keeps the fastest. Synchronises. */
SHELL_API shell_status shell_batch_autotune(shell_batch_t* batch, const double* q, int repeats);
/* One implicit-Euler step of every shell (same contract as shell_newton_step, on the
   concatenated arrays; host or device). stats: host [n_shells]. Returns SHELL_OK when every
   shell succeeded, else the status of the first shell that did not (stats[s].status holds
   each shell's). */
SHELL_API shell_status shell_batch_newton_step(shell_batch_t* batch, const shell_step_params* params,
                                               const unsigned char* fixed_mask, const double* q_fixed,
                                               double* q, double* v, const double* warm_start,
                                               shell_step_stats* stats);

/* ---------------------------------------------------------------------------------------------
   Learned Newton warm start. The paper has no learning component: this is an extension that
   predicts the initial Newton iterate of an implicit-Euler step (Sec. 6.1) per node. The
   network is a per-node MLP 28 -> 256 -> 256 -> 256 -> 12 with GELU after each hidden layer;
   weights and activations are BF16, products accumulate in FP32 on the fifth-generation tensor
   cores (tcgen05.mma into tensor memory, operands and outputs moved by TMA); FP32 master weights
   are trained with an MSE loss and Adam (beta1 0.9, beta2 0.999, eps 1e-8).
   Node features (28 floats, written by shell_node_features): u = q - q_rest (12), v (12), the
   mean over the node's present edge neighbours of u_nb - u for the position DOFs (3), and the
   mean over the same neighbours of their position speed |v_nb| (1). Target and output (12 floats): the update
   beyond the inertial predictor, q^{n+1} - q^n - dt v^n (shell_warm_targets). Inputs and
   targets are normalised per column by shell_mlp_set_normalization (x' = (x - mean) / std;
   a std of 0 is taken as 1); the loss is the mean of squared normalised errors.
   The Newton step that consumes the warm start still measures convergence against the residual
   at q^n (the zero-guess start), so the network changes the starting point, never the answer.
   Parameters are exchanged as one packed FP32 host array: for each layer l = 1..4 the weight
   matrix [fan_out x fan_in] row-major, then the bias [fan_out] (shell_mlp_param_count floats).
   All GPU work runs on the stream given to shell_mlp_create, except shell_mlp_warm_start, which
   runs on the shell's stream; a network's buffers are shared by its calls, so calls on one
   network must not overlap.
   --------------------------------------------------------------------------------------------- */
typedef struct shell_mlp_s shell_mlp_t;

/* Creates a network with zero parameters for batches of up to max_rows rows (1 .. 2^24) of
   features; stream: cudaStream_t or NULL. Device memory: about 12.7 KB per row plus 2.9 MB.
   Fails with SHELL_ERR_CUDA when the driver cannot encode the network's TMA tensor maps. */
SHELL_API shell_status shell_mlp_create(int max_rows, void* stream, shell_mlp_t** out);
SHELL_API shell_status shell_mlp_destroy(shell_mlp_t* mlp);
/* Number of floats of the packed parameter array (142,092). */
SHELL_API shell_status shell_mlp_param_count(long long* count);
/* Uploads packed FP32 parameters (host) and resets the Adam moments and step count. Synchronises. */
SHELL_API shell_status shell_mlp_set_params(shell_mlp_t* mlp, const float* params);
/* Downloads the packed parameters and/or the packed gradients of the last shell_mlp_gradients or
   shell_mlp_train_step (host buffers, either may be NULL). Synchronises. */
SHELL_API shell_status shell_mlp_get_params(shell_mlp_t* mlp, float* params, float* grads);
/* Per-column normalisation (host arrays: in_mean, in_std [28]; out_mean, out_std [12]). */
SHELL_API shell_status shell_mlp_set_normalization(shell_mlp_t* mlp, const float* in_mean, const float* in_std,
                                                   const float* out_mean, const float* out_std);
/* Mean and population standard deviation (FP64 sums) of each column of X (device [rows x cols]
   FP32, cols <= 28); mean, std: host [cols]. Synchronises. */
SHELL_API shell_status shell_mlp_column_stats(shell_mlp_t* mlp, const float* X, long long rows, int cols,
                                              double* mean, double* std);
/* Y (device [rows x 12] FP32, de-normalised) = network(X) for X device [rows x 28] FP32. */
SHELL_API shell_status shell_mlp_forward(shell_mlp_t* mlp, const float* X, int rows, float* Y);
/* Loss and parameter gradients on a batch of rows rows of a data set of data_rows rows (X device
   [data_rows x 28], T device [data_rows x 12], FP32). idx: device [rows] int row indices, or NULL
   for rows 0 .. rows-1. loss: host, may be NULL (then the call is asynchronous). An index outside
   [0, data_rows) contributes a zero row and makes the next synchronising call of this network
   return SHELL_ERR_ARG. */
SHELL_API shell_status shell_mlp_gradients(shell_mlp_t* mlp, const float* X, const float* T, long long data_rows,
                                           const int* idx, int rows, double* loss);
/* shell_mlp_gradients followed by one Adam update with learning rate lr; loss as above (the loss
   before the update). */
SHELL_API shell_status shell_mlp_train_step(shell_mlp_t* mlp, const float* X, const float* T, long long data_rows,
                                            const int* idx, int rows, float lr, double* loss);
/* Number of CUDA kernels this network has launched (host counter). */
SHELL_API shell_status shell_mlp_kernel_launches(const shell_mlp_t* mlp, long long* count);
/* Bound of the network's device-side waits: every mbarrier wait of its tensor-core kernels (TMA
   stage arrivals, MMA completion) gives up after `polls` polls (< 0: the default, 2^20; 0: every
   such wait expires at once). A kernel whose wait expires waits for the copies it issued itself,
   frees its tensor memory, skips its output and raises an error bit that the next synchronising
   call of this network (shell_mlp_gradients or shell_mlp_train_step with a loss pointer) returns
   as SHELL_ERR_TIMEOUT. Synchronises the network's stream. */
SHELL_API shell_status shell_mlp_set_wait_budget(shell_mlp_t* mlp, int polls);
/* Node features of a shell state: q, v device [n_dof] FP64; X device [n_nodes x 28] FP32. Runs on
   the shell's stream. */
SHELL_API shell_status shell_node_features(shell_t* shell, const double* q, const double* v, float* X);
/* Training targets T[k] = q_next[k] - q[k] - dt v[k] (device arrays of n_dof entries; T FP32). */
SHELL_API shell_status shell_warm_targets(long long n_dof, const double* q_next, const double* q, const double* v,
                                          double dt, float* T, void* stream);
/* warm = q + dt v + network(features(q, v)) (device [n_dof] FP64), ready to pass as warm_start to
   shell_newton_step with the same dt: one fused launch of 128 nodes per CTA, whose output equals
   that of shell_node_features followed by shell_mlp_forward. mlp may be NULL: then warm = q + dt v,
   the inertial predictor alone. An expired device-side wait (shell_mlp_set_wait_budget) leaves
   warm unwritten and is reported by the network's next synchronising call. */
SHELL_API shell_status shell_mlp_warm_start(shell_mlp_t* mlp, shell_t* shell, const double* q, const double* v,
                                            double dt, double* warm);

/* Measured arithmetic peak of the current device (no paper counterpart: a measurement aid for
   the element kernel, bound by FP32 FMA, and the FP64 energy/gradient kernel, bound by the FP64
   pipe). Times one launch of 8 independent FMA chains per thread, `iters` FMAs each, over 8 CTAs
   of 256 threads per SM (after one warm-up launch), FP64 when fp64 != 0 else FP32; stream:
   cudaStream_t or NULL. *flops_per_s receives 2 x FMAs / elapsed seconds. Synchronises; allocates
   and frees a small device buffer. */
SHELL_API shell_status shell_measure_fma_peak(int fp64, int iters, void* stream, double* flops_per_s);

/* Measured warp-level tensor-core throughput of the current device (no paper counterpart; the
   rate a TF32 tensor-core split of the element Hessian contraction of App. B.2 would run at).
   kind 0: mma.sync m16n8k8 TF32 with FP32 accumulation, kind 1: mma.sync m16n8k16 BF16. Times one
   launch of four independent accumulator tiles per warp, `iters` MMAs each, register operands,
   4 CTAs of 8 warps per SM (after one warm-up launch). *flops_per_s receives 2 x MACs / elapsed
   seconds. Synchronises; allocates and frees a small device buffer. */
SHELL_API shell_status shell_measure_mma_peak(int kind, int iters, void* stream, double* flops_per_s);

/* ------------------------------------------------------------------------------------------ */
/* Static ray-patch intersection (Sec. 5, Eq. ray, Eq. ineqray)                                */
/* ------------------------------------------------------------------------------------------ */
typedef enum { SHELL_RAY_MIDPOINT = 0, SHELL_RAY_NEWTON = 1 } shell_ray_variant;
#define SHELL_RAY_HIT 1      /* flags bit: the ray meets the shell; tau, patch, uv are written  */
#define SHELL_RAY_LIMIT 2    /* flags bit: 65536 candidates were split and the search stopped  */
#define SHELL_RAY_OVERFLOW 4 /* flags bit: the candidate heap was full even in the second pass
                                (8192 entries) or more than 65536 rays of the call needed that
                                pass; the ray is reported as a miss and its result is void    */
#define SHELL_RAY_HEAP 256   /* candidate heap entries per ray in the first pass                */

/* Nearest intersection of each ray x(tau) = o + tau d (tau >= 0, d a unit vector) with the shell
   at configuration q, by the subdivision search of Sec. 5: every patch in Bezier form (Hermite
   data b1 = a + a'/3, b2 = b - b'/3 per direction), ray-box tests of the control points' boxes
   (Eq. ineqray), a min-heap of candidate sub-patches keyed by the box's entry time, and
   De Casteljau sub-patches. variant SHELL_RAY_MIDPOINT splits every candidate at its parameter
   midpoint (Fig. submid); SHELL_RAY_NEWTON first runs Newton's method on x(u, v) = o + tau d
   from the candidate's centre (at most 12 iterations) and, on a root inside it, abandons the
   root's neighbourhood (1e-3 of the candidate's parameter extent) and splits the rest into four
   rectangles (Fig. subany). A candidate whose control-point box is at most 1e-9 on every side is
   an intersection at the midpoint of its tau interval. All arithmetic is FP64.
     q        device [n_dof] nodal DOFs (12 per node)
     origins  device [n_rays][3], dirs device [n_rays][3] (unit length; a zero component is fine)
     tau      device [n_rays]: nearest tau on a hit, +infinity on a miss
     patch    device [n_rays]: patch id of the hit, -1 on a miss
     uv       device [n_rays][2]: local patch parameters in [0, 1]^2 of the hit, 0 on a miss
     flags    device [n_rays]: SHELL_RAY_* bits
     stats    device [n_rays][4] or NULL: candidates split, largest heap size, candidate boxes
              formed (one per patch for the roots included), Newton iterations run
   A ray whose candidates outgrow the SHELL_RAY_HEAP-entry first-pass heap continues in one of 128
   library-owned 8192-entry heaps; rays beyond those 128 are traced again from the start by a
   second kernel with such a heap, so every result is that of an unbounded heap unless
   SHELL_RAY_OVERFLOW is set. n_rays in [0, 2^31 - 1]; 0 does nothing. Asynchronous
   on the shell's stream (four kernel launches and an 8-byte memset). The first call on a shell
   allocates 450 bytes per patch plus 64.3 MB of library-owned device memory (Bezier nets and
   boxes, the second pass's heaps), kept until shell_destroy; calls on one shell must not
   overlap on the GPU. */
SHELL_API shell_status shell_trace_rays(shell_t* shell, const double* q, long long n_rays, const double* origins,
                                        const double* dirs, int variant, double* tau, int* patch, double* uv,
                                        int* flags, int* stats);

/* Earliest contact of each moving point with the moving shell over one time step (Sec. 5, dynamic
   ray-patch intersection, Eq. ineqccd). The shell moves linearly from q to q + dq (its Bezier
   control points p_ij + s dp_ij, s = t / dt in [0, 1]); point k moves from x0[k] to
   x0[k] + dx[k]. Patches whose swept box misses the point's segment box are skipped; the others
   enter the subdivision search of shell_trace_rays with time in place of distance: feasible
   times of a (sub)net are [0, 1] minus, per axis and box face, the open interval outside the
   union of the control points' half-lines; candidates are keyed by their earliest feasible time;
   a candidate whose start-box side plus displacement-box side is at most 1e-9 on every axis is a
   contact at that time; variant SHELL_RAY_NEWTON splits around Newton roots in (u, v, s)
   (Fig. subany), SHELL_RAY_MIDPOINT at the midpoint (Fig. submid). All arithmetic is FP64.
     q, dq    device [n_dof]: DOFs at the start of the step and their change over the step
     x0, dx   device [n_points][3]: point positions at the start, displacements over the step
     s        device [n_points]: earliest contact time in [0, 1], +infinity when none
     patch    device [n_points]: patch id, -1 when none; uv device [n_points][2]: local (u, v)
     flags    device [n_points]: SHELL_RAY_HIT (contact), SHELL_RAY_LIMIT, SHELL_RAY_OVERFLOW
     stats    device [n_points][4] or NULL: splits, largest heap size, feasibility tests (patches
              that passed the swept-box test included), Newton iterations
   Heaps, second pass and flags as in shell_trace_rays. n_points in [0, 2^31 - 1]; 0 does
   nothing. Asynchronous on the shell's stream (four kernel launches and an 8-byte memset). The
   first call allocates 834 bytes per patch (nets and swept boxes), and the first of this call
   and shell_trace_rays the 64.3 MB search scratch they share, kept until shell_destroy; calls on
   one shell must not overlap on the GPU. */
SHELL_API shell_status shell_ccd_points(shell_t* shell, const double* q, const double* dq, long long n_points,
                                        const double* x0, const double* dx, int variant, double* s, int* patch,
                                        double* uv, int* flags, int* stats);

/* Number of CUDA kernels this shell has launched since shell_create (host counter; counts the
   launches of the library's own kernels, not memset/memcpy operations). */
SHELL_API shell_status shell_kernel_launches(const shell_t* shell, long long* count);

/* Thread-local message describing the last error ("" if none). */
SHELL_API const char* shell_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BHEM_H */
