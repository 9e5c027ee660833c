/*
 * festung.h -- C ABI of the GB300 (sm_103a) LDG diffusion solver.
 *
 * The library discretises  dt c - div(d grad c) = f  on a triangle mesh with the
 * local discontinuous Galerkin (LDG) method of FESTUNG Part I (arXiv:1408.3877):
 * orthonormal modal bases of order p = 0..4 (Sec. 2.4.1), the flux unknown
 * z = -grad c (Sec. 2.2), central fluxes with the 1/|E| penalty (Sec. 2.4.4) and
 * implicit Euler in time (Sec. 2.5).  The flux unknown is eliminated element by
 * element through the block-diagonal mass matrix, M = 2|T_k| I (Sec. 3.6.1), so a
 * step solves, for the coefficients C^{n+1},
 *
 *   S C = M C + tau (eta (S + S_D) C - sum_m A_m M^{-1} B_m C)                 (E1)
 *       = M C^n + tau (eta K_D - K_N + L + sum_m A_m M^{-1} J_D^m)  =: b       (E2)
 *
 * with B_m = -H^m + Q^m + Q_N^m and A_m = -G^m + R^m + R_D^m the block rows of the
 * system matrix of eq. timeDepSystem.  S is applied matrix-free by CUDA kernels and
 * the step is solved by BiCGStab (CG when S is symmetric, i.e. when d_h is
 * elementwise constant).
 *
 * Conventions for every call:
 *  - Return value 0 (FESTUNG_OK) on success, a negative FESTUNG_E* code otherwise;
 *    festung_last_error() then returns a message.  A failed call leaves the
 *    context's state (C, coefficients, boundary data) unchanged.
 *  - Host arrays are read (or written) during the call only; the caller keeps
 *    ownership.  Arrays flagged FESTUNG_DEVICE are device pointers of the current
 *    CUDA device, read in stream order on the context's stream.
 *  - Indices are 0-based.  Local edge n of triangle k lies opposite its vertex n
 *    and runs from vertex n+1 to vertex n+2 (mod 3), counter-clockwise.
 *  - "Samples" are values of a function at the physical quadrature points that
 *    festung_quad_points() returns, in the same order.
 *  - Coefficient arrays of the public state are K x N row-major (element-major,
 *    the paper's global ordering (k-1)N + i) in the caller's triangle order.
 *  - Internally triangles are renumbered along a Morton curve of their centroids, so
 *    that neighbours sit close in memory.  Vectors handed to festung_apply() use the
 *    library's device layout: N x K (row j holds coefficient j of all triangles) with
 *    the triangles in this internal order; festung_element_order() returns it.
 *  - All calls on one context must come from one host thread at a time.
 */
#ifndef FESTUNG_H
#define FESTUNG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FESTUNG_OK        0
#define FESTUNG_EINVAL   -1   /* bad argument (range, NULL, unsupported order)           */
#define FESTUNG_EMESH    -2   /* invalid mesh: orientation, non-manifold edge, markers    */
#define FESTUNG_ENOMEM   -3   /* device or host allocation failed                        */
#define FESTUNG_ECUDA    -4   /* CUDA runtime error                                      */
#define FESTUNG_ENOCONV  -5   /* Krylov solve did not reach the tolerance in max_iter    */
#define FESTUNG_ESTATE   -6   /* call out of order (e.g. apply before setup)              */
#define FESTUNG_EDATA    -7   /* NaN/Inf in inputs or a non-positive diffusion sample     */

#define FESTUNG_HOST      0
#define FESTUNG_DEVICE    1

#define FESTUNG_FP64      0   /* operator and Krylov iterations in FP64                   */
#define FESTUNG_FP32      1   /* FP32 operator (FP32 copies of geometry, tables, D)       */
#define FESTUNG_MIXED     2   /* step only: FP32 inner Krylov, refinement on residuals
                                 evaluated in double-float arithmetic (FESTUNG_DFLOAT)    */
#define FESTUNG_DFLOAT    3   /* apply only: FP64 arrays; the operator is evaluated in
                                 double-float arithmetic (value = hi + lo, two FP32
                                 numbers, about 48 significant bits) from double-float
                                 copies of D, the geometry and the tables               */
#define FESTUNG_BF16TAB   4   /* apply: FP32 arrays, the FP32 operator with its reference
                                 tables (basis values, weighted gradients, H^, edge
                                 traces) rounded to BF16, FP32 accumulation; step: FP32
                                 inner Krylov with that operator, refinement on residuals
                                 evaluated in FP64 (the FESTUNG_FP64 operator)          */
#define FESTUNG_MIXED64   5   /* step only: FP32 inner Krylov, refinement on residuals
                                 evaluated in FP64 (the FESTUNG_FP64 operator)          */

#define FESTUNG_BDR_INTERIOR  0
#define FESTUNG_BDR_DIRICHLET 1
#define FESTUNG_BDR_NEUMANN   2

#define FESTUNG_SOLVER_CG        1
#define FESTUNG_SOLVER_BICGSTAB  2

#define FESTUNG_BATCH_UNION       0   /* one joined mesh per group                          */
#define FESTUNG_BATCH_CONCURRENT  1   /* every problem its own step, several at a time (the
                                         default)                                           */

typedef struct festung_ctx festung_ctx;

typedef struct festung_step_opts {
    double tol;          /* stop when ||b - S C||_2 <= tol ||b||_2 (unpreconditioned, over K x N) */
    int    max_iter;     /* bound on Krylov iterations (all inner iterations in FESTUNG_MIXED)  */
    int    prec;         /* FESTUNG_FP64, FESTUNG_MIXED, FESTUNG_MIXED64 or FESTUNG_BF16TAB     */
    double inner_tol;    /* FESTUNG_MIXED: relative reduction per inner FP32 solve (e.g. 1e-2)   */
    int    max_outer;    /* FESTUNG_MIXED: bound on refinement sweeps                          */
    int    solver;       /* 0: choose (CG iff S is symmetric); else FESTUNG_SOLVER_*            */
} festung_step_opts;

typedef struct festung_step_info {
    int    iterations;   /* Krylov iterations (summed over refinement sweeps)                  */
    int    outer;        /* refinement sweeps (1 for FESTUNG_FP64)                              */
    double rel_residual; /* final ||b - S C||_2 / ||b||_2 (FESTUNG_MIXED: S C in double-float;
                            the other modes: in FP64)                                        */
    int    solver;       /* FESTUNG_SOLVER_CG or FESTUNG_SOLVER_BICGSTAB                        */
    int    symmetric;    /* 1 if d_h is elementwise constant (S symmetric, Sec. 2.4.3-2.4.4)   */
    int    fp64_iterations; /* mixed modes: iterations of the FP64 solve that finished the step
                               after an FP32 sweep failed to lower the residual (else 0)            */
    double initial_rel_residual; /* ||b - S C0||_2 / ||b||_2 of the initial guess C0               */
    int    coarse_iterations;    /* Krylov iterations of the coarse (p = 1) solves, festung_set_coarse */
    int    precond_built;        /* 1 if this step built its block-Jacobi blocks, 0 if it reused
                                    earlier ones (festung_set_precond_reuse)                        */
} festung_step_info;

/* Build the grid lists of Tab. 1 (Sec. 3.1, routine generateGridData): edges,
 * neighbours, the affine maps F_k(x^) = B_k x^ + a_k1 (eq. affinemappings) and edge
 * normals, and upload them to the current device.
 *   coordV   numV x 2 vertex coordinates, row-major (host).
 *   V0T      numT x 3 vertex indices of each triangle, counter-clockwise (host).
 *   bdr_type numT x 3 type of local edge n of triangle k: FESTUNG_BDR_* (host).
 *            Interior edges must be 0; every boundary edge must be 1 or 2.
 *   out      receives the new context (owns all device memory it allocates).
 * Errors: EINVAL (NULL, sizes), EMESH (det B_k <= 0, an edge shared by more than
 * two triangles or traversed twice in one direction, marker mismatch, bad index),
 * EDATA (non-finite coordinates), ENOMEM, ECUDA. */
int festung_mesh_create(const double *coordV, int64_t numV,
                        const int32_t *V0T, int64_t numT,
                        const int8_t *bdr_type, festung_ctx **out);

/* Choose the order and quadrature (Sec. 3.3) and build the basis/quadrature tables.
 *   p          polynomial degree 0..4, N = (p+1)(p+2)/2 (Sec. 2.4.1).
 *   quad_order exactness degree of the triangle rule: 0 selects 2p (the paper's
 *              choice); otherwise 2p or 2p+1 (degree 3 is served by the degree-4
 *              rule, degrees >= 7 by a collapsed Gauss rule).  Edges use
 *              Gauss-Legendre exact to degree max(quad_order, 2p+1).
 *   eta        penalty coefficient > 0 (Sec. 2.4, eta = 1 in the paper).
 * Resets C to zero and D to the constant 1.  Errors: EINVAL, ENOMEM, ECUDA. */
int festung_setup(festung_ctx *ctx, int p, int quad_order, double eta);

/* Sizes after setup: K triangles, N local DOFs, R2 triangle and R1 edge quadrature
 * points (any pointer may be NULL). */
int festung_sizes(const festung_ctx *ctx, int64_t *K, int *N, int *R2, int *R1);

/* Physical quadrature points F_k(q_r) (host outputs, either may be NULL):
 *   xy   K x R2 x 2 triangle points;   exy  K x 3 x R1 x 2 Gauss points of every
 *   local edge n, ordered along gamma_n (eq. gammaMap). */
int festung_quad_points(const festung_ctx *ctx, double *xy, double *exy);

/* L2 projection of d(t^{n+1}) (Sec. 3.4): d_samples is K x R2 at the triangle
 * points.  Every sample must be finite and > 0 (else EDATA).  loc: FESTUNG_HOST or
 * FESTUNG_DEVICE (FP64).  Decides whether S is symmetric (d_h elementwise constant). */
int festung_set_coeff(festung_ctx *ctx, const double *d_samples, int loc);

/* L2 projection of the source f(t^{n+1}) (K x R2 samples); NULL sets f = 0. */
int festung_set_source(festung_ctx *ctx, const double *f_samples, int loc);

/* Boundary data at t^{n+1} at the edge Gauss points, each K x 3 x R1: c_D is read
 * on Dirichlet edges, g_N = -grad c . nu on Neumann edges (Sec. 1.1); other
 * entries are ignored.  NULL means zero. */
int festung_set_bc(festung_ctx *ctx, const double *cD, const double *gN, int loc);

/* Set C: K x N coefficients (is_samples = 0), or K x R2 samples of c^0 that are
 * L2-projected (is_samples = 1, Sec. 3.4). */
int festung_set_state(festung_ctx *ctx, const double *C, int is_samples, int loc);

/* Copy C (K x N, FP64) out to host or device memory. */
int festung_get_state(const festung_ctx *ctx, double *C, int loc);

/* y = S x of (E1) with the current D and time step dt (dt = 0 gives y = M x).
 *   x, y  device arrays in the N x K layout, FP64 (prec = FESTUNG_FP64 or
 *         FESTUNG_DFLOAT) or FP32 (prec = FESTUNG_FP32 or FESTUNG_BF16TAB); x and y
 *         must not overlap;
 *         16-byte aligned.
 * FESTUNG_DFLOAT evaluates the operator in double-float arithmetic (the residual of
 * FESTUNG_MIXED steps): x is split into pairs of FP32 values, the result is rounded
 * back to FP64; error a few units of 2^-48 times |S| |x| (elementwise magnitudes).
 * Boundary data does not enter (S is the homogeneous operator). Runs on the
 * context's stream and returns without synchronising. */
int festung_apply(festung_ctx *ctx, const void *x, void *y, int prec, double dt);

/* Same result as festung_apply(), for callers that cannot allocate device memory:
 * code running under an external memory manager that owns the device's memory (a
 * framework pool or a fixed budget, where an extra cudaMalloc fails or escapes the
 * accounting) and latency-critical loops where cudaMalloc/cudaFree would synchronise
 * the device.  The paper has no counterpart; it is a deployment variant of the apply.
 * The flux unknowns go to a fixed 32 MiB array inside the library instead of
 * context scratch, so the call allocates and frees nothing.  Limit: 2 x N x K values
 * of the chosen precision must fit in 32 MiB (N*K <= 2,097,152 for FP64, 4,194,304
 * for FP32); larger meshes get FESTUNG_EINVAL.  The array exists once per device
 * for the life of the process and is shared by all contexts and calls: calls whose
 * kernels overlap on the GPU (other streams or threads) race on it and must be
 * ordered by the caller.  Every call made outside stream capture looks up the array's
 * device address (it changes when cudaDeviceReset replaces the device's context); a call
 * on a stream being captured reuses the last address found, so make the first call on a
 * device before any stream capture (ESTATE otherwise).  Arguments, layout and errors as
 * festung_apply(). */
int festung_apply_noalloc(festung_ctx *ctx, const void *x, void *y, int prec, double dt);

/* One implicit-Euler step of size dt (Sec. 2.5): forms b of (E2) from the current
 * C, D, f and boundary data, solves (E1) and, only on success, replaces C by C^{n+1}.
 * The initial guess extrapolates the previous states in time: quadratically through
 * C^{n-2}, C^{n-1}, C^n after two successful steps, linearly after one, else C^n;
 * festung_set_state and festung_setup reset this history.  Preconditioner: inverse N x N
 * diagonal blocks of S.  opts may be NULL (tol 1e-10, max_iter 20000, FESTUNG_MIXED,
 * inner_tol 1e-2, max_outer 50).  opts->prec: FESTUNG_FP64 (FP64 Krylov), FESTUNG_MIXED
 * (FP32 inner Krylov sweeps, refinement residual in double-float), FESTUNG_MIXED64 (the
 * same with the refinement residual in FP64), FESTUNG_BF16TAB (FP32 inner Krylov on the
 * BF16-table operator, FP64 residual).  Every mode meets tol on its own residual
 * and falls back to FP64 Krylov sweeps when the inner sweeps stop lowering it.  info may
 * be NULL.  Synchronises the context's stream.  Errors: ENOCONV (C unchanged), EINVAL,
 * ESTATE, ECUDA. */
int festung_step(festung_ctx *ctx, double dt, const festung_step_opts *opts,
                 festung_step_info *info);

/* The stationary problem of Sec. 3.9 (the code-verification setting): solves
 *   (eta (S + S_D) - sum_m A_m M^{-1} B_m) C = eta K_D - K_N + L + sum_m A_m M^{-1} J_D^m
 * with the current D, f and boundary data, starting from the current C, and replaces C
 * on success.  Options and info as festung_step (info->rel_residual relative to the
 * right-hand side).  Needs at least one Dirichlet edge (EINVAL otherwise: with
 * zero-flux data alone the operator is singular).  Resets the time extrapolation. */
int festung_solve_stationary(festung_ctx *ctx, const festung_step_opts *opts, festung_step_info *info);

/* Discretisation error ||c_h - c||_{L2} (Sec. 3.5) of the current C from samples of the
 * exact c at the triangle points (K x R2, host), with the context's triangle rule;
 * evaluated on the device. */
int festung_l2_error(const festung_ctx *ctx, const double *c_samples, double *err);

/* Recover the flux unknown z_h = -grad c_h in the mixed form (Sec. 2.2) from the
 * current C: Z^m = -M^{-1} (B_m C + J_D^m), block rows 1-2 of eq. timeDepSystem, with
 * the Dirichlet data last given to festung_set_bc.  Z: 2 x K x N (Z^1 then Z^2, each
 * K x N in the caller's order like the state), host or device (loc).  Synchronises the
 * context's stream. */
int festung_get_flux(const festung_ctx *ctx, double *Z, int loc);

/* Tile size by measurement: times the FP32 operator apply for tiles of 96..256
 * triangles (multiples of 32) and keeps the fastest (festung_setup picks the tiles from
 * an occupancy model, deterministically; batches run this for every group).  Results do
 * not depend on the tiling beyond rounding.  tile may be NULL.  Synchronises the
 * context's stream. */
int festung_autotune(festung_ctx *ctx, int *tile);

/* ---- Learned warm start -----------------------------------------------------------
 * A small network proposes the correction C^{n+1} - C^n of the next step from local
 * features; the Krylov solve then starts from C^n plus that correction and is converged
 * to the same tolerance as always, so the answer does not depend on the network.  The
 * paper has no counterpart.
 *
 * festung_warmstart_features: with the current D, f, boundary data and C (= C^n), the
 * residual r = b - S C^n of (E1)-(E2) for step dt (S C^n in double-float arithmetic), and
 * per triangle k of the internal order row k of X (device, K x F FP32, F = 3 + 4 N):
 * d_h modes 0..2 over the mean of mode 0, then M^{-1} r of k and of its neighbours across
 * local edges 0, 1, 2 (zeros on the boundary), divided by rs = RMS of M^{-1} r over all
 * coefficients; *scale = rs.  A network output y (K x N rows) then means the correction
 * rs y.  Wt (device, K x N FP32, or NULL): loss weights sqrt(S_kk[j][j] / 2|T_k|) from the
 * diagonal blocks of S, large for the stiff modes that a wrong correction turns into
 * residual.  Synchronises the context's stream.
 * festung_set_guess: the next festung_step starts from C^n + delta (delta K x N in the
 * caller's order like the state, host or device; NULL clears it).  Used once; set_state
 * and setup clear it. */
int festung_warmstart_features(festung_ctx *ctx, double dt, float *X, float *Wt, double *scale);
int festung_set_guess(festung_ctx *ctx, const double *delta, int loc);

/* The network: in -> 64 -> 64 -> out, ReLU after the hidden layers, BF16 weights with an
 * FP32 master copy, FP32 biases and accumulation.  Parameters: W1 (64 x in, row-major),
 * b1 (64), W2 (64 x 64), b2, W3 (out x 64), b3 (out).  Weights start Glorot-uniform from
 * a seeded generator, biases at 0.  in <= 96, out <= 32.
 *   forward: Y = net(X) for rows x in inputs (device FP32, row-major; Y rows x out);
 *   grad:    gradient of (1 / 2 rows) sum (Wt (net(X) - T))^2 over the rows into the
 *            net's gradient buffer (replacing it), the loss into *loss (may be NULL); Wt:
 *            rows x out weights (device) or NULL for 1;
 *   adam:    one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on the
 *            FP32 master, then the BF16 copy;
 *   get/set: the FP32 master parameters (and the last gradient) on the host.
 * Errors: EINVAL, ENOMEM, ECUDA (festung_mlp_last_error). */
typedef struct festung_mlp festung_mlp;
int festung_mlp_create(int n_in, int n_out, uint64_t seed, festung_mlp **out);
int festung_mlp_sizes(const festung_mlp *net, int *n_in, int *n_out, int *n_params);
int festung_mlp_set_stream(festung_mlp *net, void *cuda_stream);
int festung_mlp_forward(festung_mlp *net, const float *X, float *Y, int64_t rows);
int festung_mlp_grad(festung_mlp *net, const float *X, const float *T, const float *Wt, int64_t rows, double *loss);
int festung_mlp_adam(festung_mlp *net, double lr);
int festung_mlp_get(const festung_mlp *net, float *params, float *grad);
int festung_mlp_set(festung_mlp *net, const float *params);
const char *festung_mlp_last_error(void);
void festung_mlp_destroy(festung_mlp *net);

/* Multiply-add throughput of the current device in TFLOP/s (FP32 or FP64 by prec): 8
 * independent chains per thread, 8 blocks of 256 threads per SM, best of 5 launches.
 * The ALU ceiling the operator kernels are compared with; the paper has no counterpart. */
int festung_fma_peak(int prec, double *tflops);

/* ---- Batches of independent problems -------------------------------------------
 * Many problems (each its own context, set up, with its own mesh, order, coefficient,
 * source and boundary data) advance by one implicit-Euler step together.  The paper has
 * no counterpart: it solves one problem at a time.  Two modes:
 *
 * FESTUNG_BATCH_CONCURRENT (the default): each problem takes its own single-problem step
 * (festung_step with opts, FP64 fallback included), `workers` problems at a time, each
 * worker on a CUDA stream and host thread of its own, so that the kernels of small
 * problems share the GPU.  A problem's step runs after the work queued on its own stream
 * and on the batch's stream; the problems' own streams are left as they were.
 *
 * FESTUNG_BATCH_UNION: problems of the same p, quadrature and eta form a group whose
 * meshes are joined into one internal mesh, and each kernel of the step runs over all
 * problems of the group at once.  Every problem runs its own BiCGStab iteration (its own
 * scalars, reductions summed per problem) and its own refinement, and reaches tol on its
 * own residual; tiles of problems that have finished do no work.  A problem the group
 * cannot finish is stepped on its own (the single-problem path).  The groups run
 * concurrently, each on a stream and host thread of its own.  The joined meshes are built
 * at the first union-mode step, which then also reports the errors of building them
 * (EINVAL for a group with K N >= 2^31, ENOMEM).  The extrapolated initial
 * guess of a group restarts when one of its problems' state was set from outside since
 * the last batch step.
 *
 * festung_batch_create: problems[0..nprob) stay owned by the caller and must outlive the
 * batch; they must not be set up again while in it.  Their data are set with the usual
 * calls (festung_set_coeff, _source, _bc, _state) before each festung_batch_step, which
 * reads them, steps all problems (FESTUNG_MIXED only; opts as festung_step) and writes
 * every C back (festung_get_state reads it).  infos: nprob entries or NULL.  The step
 * starts after the work queued on the batch's stream (festung_batch_set_stream; default
 * the legacy default stream), which then waits for all of it; the call returns once every
 * problem is done.  On an error the failing problems keep their C, the others complete
 * their step, and the code of the first failure (by problem, or by group) is returned.
 * festung_batch_set_mode: mode and workers (0: the default, 16 or the host's thread count
 * if lower; at most 64; the union mode ignores it).
 * festung_batch_launch_count: kernels launched by the batch's steps, those on the
 * problems' own contexts included. */
typedef struct festung_batch festung_batch;
int festung_batch_create(festung_ctx *const *problems, int nprob, festung_batch **out);
int festung_batch_set_stream(festung_batch *batch, void *cuda_stream);
int festung_batch_set_mode(festung_batch *batch, int mode, int workers);
int festung_batch_step(festung_batch *batch, double dt, const festung_step_opts *opts, festung_step_info *infos);
int festung_batch_launch_count(const festung_batch *batch, int64_t *n);
/* Message of the last failed batch call (batch = NULL: of the last failed create). */
const char *festung_batch_last_error(const festung_batch *batch);
void festung_batch_destroy(festung_batch *batch);

/* The internal triangle order of the device layout: order[i] is the caller's index of
 * the triangle stored at position i (order holds K entries, host memory). */
int festung_element_order(const festung_ctx *ctx, int64_t *order);

/* The block-Jacobi preconditioner of a step with time step dt, for inspection: blocks
 * gets the N x N diagonal blocks S_kk of (E1) as the FP32 build computes them (from the
 * FP32 copies of geometry, tables and D, with the context's current D), inverse the
 * BF16 inverses the Krylov kernels apply (converted to FP64).  Each K x N x N, host
 * memory, triangle k in the caller's order, row-major blocks (row i, column j at
 * (k N + i) N + j); either may be NULL, not both.  The context's preconditioner is
 * replaced (every step builds its own).  EDATA if a block is singular (the blocks are
 * still written).  The paper has no counterpart: it solves directly. */
int festung_precond_blocks(festung_ctx *ctx, double dt, double *blocks, double *inverse);

/* Number of CUDA kernels this context has launched so far (kernels inside a replayed
 * CUDA graph count one each per replay, including those that exit early because the
 * Krylov iteration already converged).  For instrumentation; *count must not be NULL. */
int festung_launch_count(const festung_ctx *ctx, int64_t *count);

/* Use this CUDA stream (cudaStream_t) for all later work; NULL = legacy default. */
int festung_set_stream(festung_ctx *ctx, void *stream);

/* Message of the last failed call on ctx (or of the last failed festung_mesh_create
 * when ctx is NULL).  Valid until the next call on the context. */
const char *festung_last_error(const festung_ctx *ctx);

/* Coarse correction of the FP32 sweeps (p >= 2; FESTUNG_MIXED, _MIXED64 and _BF16TAB
 * steps and the stationary solve).  The basis is hierarchical, so the coefficients of
 * phi_1..phi_3 of every triangle span the P1 subspace.  With enable = 1 each sweep first
 * solves the p = 1 problem on the same mesh (the method of Sec. 2 at p = 1, d_h replaced by
 * its P1 part, the same tau and mass term) for the P1 part of the sweep's right-hand side,
 * to a relative residual of 1e-2 (FP32 Krylov, block Jacobi, started from the previous
 * coarse solution), and starts the sweep from that correction instead of from zero.  The smooth error components, which block-Jacobi
 * Krylov removes slowest, are handled by the small problem.  The result does not depend on
 * it beyond the tolerance.  The p = 1 problem is built at the first step that needs it
 * (device memory of a p = 1 context).  enable = 0 (the default) turns it off.  The paper has
 * no counterpart: it solves directly. */
int festung_set_coarse(festung_ctx *ctx, int enable);

/* How the BiCGStab iterations of the FP32 solves run at p <= 1 (the inner sweeps of a
 * p <= 1 context, and the coarse problem of festung_set_coarse).  enable = 1 (the
 * default): one persistent cooperative kernel per solve, whose blocks each keep their
 * tiles of the mesh and meet at grid-wide barriers between the four phases of an
 * iteration; its reductions are summed in double-float arithmetic by every block in the
 * same order.  enable = 0: the CUDA graph of four kernels per iteration (the form used at
 * p >= 2).  Both iterate the same method; their sums are rounded differently.  A device
 * that cannot hold the persistent grid falls back to the graph.  EINVAL unless enable is
 * 0 or 1. */
int festung_set_persistent(festung_ctx *ctx, int enable);

/* Testing hook for the failure path of the persistent kernel: with enable = 1 every grid
 * barrier of the context's persistent solves waits for one block more than the grid has,
 * so that each wait runs out (after about a second) and the solve fails with
 * FESTUNG_ECUDA ("a grid barrier wait gave up"); the context stays usable, and enable = 0
 * restores normal solves.  EINVAL unless enable is 0 or 1. */
int festung_test_barrier_timeout(festung_ctx *ctx, int enable);

/* Reuse of the block-Jacobi preconditioner over time steps.  Every step solves with the
 * inverse diagonal blocks of S; they depend on d_h, dt and the mass term and cost about as
 * much to build as a few Krylov iterations.  With max_steps = m > 1 one build serves up
 * to m consecutive steps (festung_step, the FP32 sweeps and the FP64 solves alike, and the
 * coarse problem's blocks with them) while dt and the mass term stay the same: the blocks
 * then belong to d_h of the step that built them (a lagged preconditioner).  A step whose
 * Krylov iterations exceed 1.5 times those of the building step plus 4 ends the reuse
 * (the next step builds).  The answer does not depend on it beyond the tolerance;
 * festung_step_info.precond_built tells which steps built.  max_steps = 1 (the default):
 * every step builds its own.  EINVAL if max_steps < 1.  The paper has no counterpart: it
 * solves directly. */
int festung_set_precond_reuse(festung_ctx *ctx, int max_steps);

/* Free the context and all its device memory.  NULL is a no-op. */
void festung_destroy(festung_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* FESTUNG_H */
