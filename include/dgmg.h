/*
 * dgmg.h -- C ABI of libdgmg: matrix-free SIPG discontinuous Galerkin with
 * hp-multigrid on one NVIDIA GB300 GPU (sm_103a).
 *
 * Method: Baccas, Belozerov, Mueller, Weinzierl, "Implementation techniques for
 * multigrid solvers for high-order Discontinuous Galerkin methods" (arXiv
 * 2510.00998). Section / algorithm / equation numbers below refer to that paper.
 *
 * Problem: -div(kappa grad u) = f on the unit box [0,1]^d (d = 2 or 3),
 * homogeneous Dirichlet, uniform mesh of n[0] x n[1] (x n[2]) cells,
 * tensor-product GLL Lagrange basis of degree p per axis (q = p+1 nodes per
 * axis, q^d DoFs per cell), cellwise-constant kappa > 0. Bilinear form: Eq.
 * weak_form_IP (Sec. 2.3.1) with theta = -1 (symmetric interior penalty),
 * penalty gamma_F = 2 p (p+1) / h on every facet, every interior facet term
 * scaled by the harmonic mean 2 k- k+ / (k- + k+), boundary facet terms and
 * the volume term by the cell's kappa.
 *
 * Vector layout (every DG vector argument): double[ncell * q^d], cell-major,
 * cell = ix + n0 * (iy + n1 * iz), node = i + q * (j + q * k) within the cell
 * (x fastest), nodes at the GLL points of the cell. CG (Q1) vectors live on the
 * interior vertices, (vx-1) + (n0-1) * ((vy-1) + (n1-1) * (vz-1)).
 *
 * Memory: unless stated otherwise, vector arguments are DEVICE pointers owned by
 * the caller; the library keeps no reference to them after the call returns its
 * work to the stream. All device work of a call is queued on `stream` (a
 * cudaStream_t passed as void*, NULL = the legacy default stream); calls return
 * without a host synchronisation unless stated. The library owns everything
 * inside a dgmg_ctx. A ctx may be used from one host thread at a time.
 *
 * Errors: every int-returning call returns DGMG_OK (0) or a negative code; the
 * thread-local message of the last failure is returned by dgmg_last_error().
 * Arguments are validated before any device work is queued.
 */
#ifndef DGMG_H
#define DGMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGMG_OK 0
#define DGMG_EINVAL (-1)          /* invalid argument (message says which)            */
#define DGMG_ENOMEM (-2)          /* device or host allocation failed                 */
#define DGMG_EBUDGET (-3)         /* request cannot fit the server's HBM budget       */
#define DGMG_ENOTCONVERGED (-4)   /* maxit reached; x holds the last iterate          */
#define DGMG_ENONFINITE (-5)      /* a NaN/Inf was detected in an input or residual   */
#define DGMG_ECUDA (-6)           /* a CUDA runtime call failed                       */
#define DGMG_ETIMEOUT (-7)        /* a bounded device-side wait ran out during the    */
                                  /* call (see dgmg_wait_timeouts): its result is not */
                                  /* to be trusted                                    */

/* precision of the V-cycle used as preconditioner */
#define DGMG_FP64 0               /* every stage in FP64                               */
#define DGMG_MIXED_FP32 1         /* V-cycle in FP32 inside FP64 CG (Sec. 5 cycle,     */
                                  /* outer residual/update/coarsest solve in FP64)     */

/* outer iteration of dgmg_solve */
#define DGMG_OUTER_AUTO 0         /* RELIABLE with DGMG_MIXED_FP32, PCG with DGMG_FP64  */
#define DGMG_OUTER_PCG 1          /* FP64 CG: one FP64 apply per iteration (flexible   */
                                  /* Polak-Ribiere form with the FP32 V-cycle)         */
#define DGMG_OUTER_RELIABLE 2     /* DGMG_MIXED_FP32 only: CG in FP32 (FP32 apply and  */
                                  /* V-cycle, FP64-accumulated dot products), solution */
                                  /* accumulated in FP64, true residual recomputed in  */
                                  /* FP64 whenever the FP32 residual fell by `delta`   */
                                  /* (reliable updates) and for the stopping test      */
#define DGMG_OUTER_MGMULT 3       /* DGMG_FP64 only: the stationary hp-multigrid       */
                                  /* iteration (Alg. 7, MGMult): per cycle nu_pre      */
                                  /* block-Jacobi steps and one coarse-grid correction */
                                  /* (Alg. 6); stops when ||b - A x|| <= rtol ||b||    */
#define DGMG_OUTER_MGMULT_PREC 4  /* as DGMG_OUTER_MGMULT, but stops on the            */
                                  /* preconditioned residual: ||x_k - x_(k-1)|| <=     */
                                  /* rtol ||x_1 - x_0||                                */

/* block inverse used by the block-Jacobi smoother (Eq. block-Jacobi-IP) */
#define DGMG_BASIS_GLL 0          /* Gauss-Lobatto-Legendre nodes (Sec. 2.2): the end  */
                                  /* nodes carry the traces, non-diagonal mass matrix  */
#define DGMG_BASIS_GL 1           /* Gauss-Legendre nodes (Sec. 6.4): diagonal mass    */
                                  /* matrix, every node contributes to a trace (dense  */
                                  /* cell-to-facet projection, Sec. 4.1). The same     */
                                  /* discrete problem in another basis; solves run the */
                                  /* sum-factorised per-pencil smoother (the           */
                                  /* one-thread-per-cell smoother is GLL-only), and    */
                                  /* batched solves take GLL only                      */

#define DGMG_BLOCK_EXACT 0        /* exact diagonal block A_KK of every cell           */
#define DGMG_BLOCK_INTERIOR_ONLY 1/* Technique 4: the block of an interior cell, with  */
                                  /* the cell's own kappa, for every cell              */

typedef struct {
    int dim;                      /* 2 or 3                                            */
    int n[3];                     /* cells per axis, each >= 1 (n[2] ignored for d=2)  */
} dgmg_mesh;

typedef struct {
    double omega_dg;              /* block-Jacobi damping, 0 < omega < 2 (default 0.8) */
    double omega_cg;              /* point-Jacobi damping on Q1 levels (default 0.8)   */
    int nu_pre, nu_post;          /* smoothing steps per level (default 2, 2)          */
    int precision;                /* DGMG_FP64 (default) or DGMG_MIXED_FP32            */
    int block_inverse;            /* DGMG_BLOCK_EXACT (default) | _INTERIOR_ONLY       */
    int coarsening;               /* h-coarsening factor 2 (default) or 3              */
    double rtol;                  /* dgmg_solve: stop at ||b-Ax||_2 <= rtol ||b||_2    */
                                  /* (default 1e-10)                                   */
    int maxit;                    /* dgmg_solve iteration cap (default 200)            */
    int outer;                    /* DGMG_OUTER_* (default AUTO)                       */
    double delta;                 /* reliable-update factor, 0 < delta < 1 (0.01)      */
    int autotune;                 /* 1: dgmg_create times the candidate tile shapes of */
                                  /* the DG-level kernels on this mesh and keeps the   */
                                  /* fastest (cached per mesh shape in the process);   */
                                  /* 0 (default): fixed heuristic                      */
    int p_coarsening;             /* 0 (default): DG degree p straight to continuous   */
                                  /* Q1 (Sec. 5.2); 1: gradual, DG p, p-1, ..., 1, then */
                                  /* Q1 (the nested sequence of the outlook of Sec.    */
                                  /* 6.4), every DG level the Galerkin product of the  */
                                  /* one above (finest penalty) with its own           */
                                  /* block-Jacobi smoother and nu_pre/nu_post steps    */
    int basis;                    /* nodes of the 1D Lagrange basis of the DG space:   */
                                  /* DGMG_BASIS_GLL (default) or DGMG_BASIS_GL         */
    int recompute_block;          /* 0 (default): the per-cell factors of the block    */
                                  /* inverses A_KK^-1 are computed once at set-up      */
                                  /* (Technique 3, precomputed); 1: recomputed on the  */
                                  /* device before every smoothing step (the paper's   */
                                  /* "recompute" variant of Table 6, Sec. 7.1); same   */
                                  /* results. Batched solves take 0 (DGMG_EINVAL)      */
} dgmg_opts;

typedef struct {
    int dim, p, q;                /* dimension, degree, nodes per axis                 */
    int n[3];                     /* cells per axis                                    */
    int64_t ncell, ndof;          /* cells, DG unknowns                                */
    int nlevels_cg;               /* Q1 levels below the DG level (>= 1)               */
    int64_t nvert0;               /* unknowns of the first Q1 level                    */
    int64_t ncoarse;              /* unknowns of the coarsest level (dense solve)      */
    double omega_dg, omega_cg;    /* damping actually used                             */
    int nu_pre, nu_post, precision, block_inverse, coarsening;
    size_t device_bytes;          /* device memory held by the ctx                     */
    int outer;                    /* DGMG_OUTER_* in use (AUTO resolved)               */
    int dg_levels;                /* DG levels of the V-cycle (1, or p with gradual    */
                                  /* p-coarsening)                                     */
    int tiles[6];                 /* cells per CTA of the DG-level kernels in use:     */
                                  /* FP64 projection, smoothing, residual, then FP32   */
                                  /* (mixed precision only, else 0); a smoothing entry */
                                  /* of 0 = the one-thread-per-cell kernel where it    */
                                  /* applies (3D, exact blocks, FP32 q <= 5, FP64      */
                                  /* q <= 4), else the default pencil tile             */
} dgmg_info_t;

typedef struct {
    int iterations;               /* outer CG iterations                               */
    double rel_residual;          /* ||b - A x||_2 / ||b||_2 of the returned x, recomputed */
    double rel_residual_recursive;/* the CG recurrence's last estimate                 */
    double prec_residual;         /* ||z||_2 / ||z_0||_2 of the last preconditioned    */
                                  /* residual z = V(r) (Eq. preconditioned_residual)   */
    double seconds;               /* wall time of the call                             */
    int fp64_applies;             /* FP64 applications of A (residuals b - A x and, in */
                                  /* DGMG_OUTER_PCG, the products A p)                 */
    double queue_seconds;         /* served requests: submit -> admission (else 0);   */
                                  /* `seconds` is then submit -> completion            */
} dgmg_stats;

typedef struct dgmg_ctx dgmg_ctx;
typedef struct dgmg_server dgmg_server;

/* request states reported by dgmg_poll */
#define DGMG_PENDING 0            /* queued, not yet admitted                          */
#define DGMG_RUNNING 1            /* admitted, solve in progress on the GPU            */
#define DGMG_DONE 2               /* converged; x holds the solution                   */
#define DGMG_FAILED 3             /* see dgmg_poll's return code and dgmg_last_error   */

typedef struct {
    int pending, active;          /* queued / admitted requests                        */
    long long done, failed, admitted;
    int cache_entries;            /* resident hierarchies (busy or idle)               */
    long long cache_hits, cache_misses, evictions;
    size_t bytes_in_use, budget;  /* device bytes held by resident hierarchies         */
} dgmg_server_info_t;

/* Library version string. */
const char *dgmg_version(void);

/* Message of the last failed call on this host thread ("" if none). */
const char *dgmg_last_error(void);

/* Fill *opts with the defaults listed in dgmg_opts. */
void dgmg_default_opts(dgmg_opts *opts);

/*
 * Build the hierarchy for `mesh`, degree p (1..6) and kappa (HOST array of
 * ncell positive finite doubles, cell-major; NULL = kappa 1 everywhere):
 * 1D reference matrices (Sec. 2.2), per-cell fast-diagonalisation factors of
 * the exact diagonal blocks A_KK (Sec. 4.1, Technique 3), the Q1 operator
 * P^T A P (Sec. 2.4) and its Galerkin coarsenings (Sec. 5.2), the dense inverse
 * of the coarsest operator, and all device work buffers. opts NULL = defaults.
 * Synchronous. On failure *out is NULL and nothing is leaked.
 */
int dgmg_create(const dgmg_mesh *mesh, int p, const double *kappa, const dgmg_opts *opts,
                dgmg_ctx **out);

/* Free every resource of ctx (waits for its device work). NULL is accepted. */
int dgmg_destroy(dgmg_ctx *ctx);

/* Describe ctx (host struct, filled synchronously). */
int dgmg_info(const dgmg_ctx *ctx, dgmg_info_t *info);

/* The 1D node coordinates on [-1,1] of ctx's basis (GLL, or GL with
 * opts.basis = DGMG_BASIS_GL; Sec. 2.2.1, 6.4): HOST array of q doubles,
 * ascending. */
int dgmg_gll_nodes(const dgmg_ctx *ctx, double *nodes_host);

/*
 * Replace ctx's coefficient field by kappa_host (HOST array of ncell doubles,
 * each positive and finite, layout as for dgmg_create) without rebuilding the
 * hierarchy: the Q1 operators P^T A P, their Galerkin coarsenings and the
 * coarsest inverse are recomputed on the host into the existing device
 * buffers, and the per-cell fast-diagonalisation factors of every DG level
 * on the device (the exact diagonal blocks A_KK of Sec. 4.1 for the new
 * kappa: the paper's independent per-cell inversion tasks, Technique 6, for
 * coefficients that change between solves). No allocation; captured solver
 * graphs stay valid. Blocking: returns when the device data are updated. No
 * work of ctx may be in flight on other streams. DGMG_EINVAL for an invalid
 * kappa (ctx unchanged).
 */
int dgmg_update_kappa(dgmg_ctx *ctx, const double *kappa_host);

/*
 * y = A u (the SIPG operator, Eq. matrix_form_IP), FP64, DG layout. Runs the
 * warm-up projection (Alg. 4 preamble) and the cell equation of Alg. 2 stage 3
 * on the stored projections. u and y must not overlap.
 */
int dgmg_apply(dgmg_ctx *ctx, const double *u, double *y, void *stream);

/* r = b - A u, FP64 (Alg. 6 residual without the restriction). */
int dgmg_residual(dgmg_ctx *ctx, const double *u, const double *b, double *r, void *stream);

/*
 * nsteps >= 0 damped block-Jacobi steps u <- u + omega_dg A_KK^{-1} (b - A u)
 * in the single-touch order of Alg. 4 (one warm-up projection, then one fused
 * traversal per step reading the neighbours' stored projections, updating the
 * cell, re-projecting it). FP64, u in/out, b input.
 */
int dgmg_smooth(dgmg_ctx *ctx, double *u, const double *b, int nsteps, void *stream);

/*
 * e = V(r): one hp V(nu_pre, nu_post) cycle with zero initial guess (Alg. 6 /
 * Alg. 7 building blocks, Sec. 5.2): nu_pre smoothing steps, residual and
 * p-restriction to Q1, the h-multigrid V-cycle with point Jacobi on the Q1
 * levels and the dense coarsest solve, p-prolongation fused into the next
 * projection, nu_post smoothing steps. In DGMG_MIXED_FP32 precision the cycle
 * runs in FP32 (r rounded on entry, e widened on exit); the coarsest solve is
 * FP64 in both. r and e are FP64 and must not overlap. The Q1 part is one
 * cooperative kernel launch (all its blocks co-resident, steps separated by a
 * bounded grid barrier; see dgmg_wait_timeouts) where the device supports it
 * and the launch can be captured into a CUDA graph, else one launch per step;
 * the results agree to rounding.
 */
int dgmg_vcycle(dgmg_ctx *ctx, const double *r, double *e, void *stream);

/*
 * Solve A x = b with conjugate gradients preconditioned by dgmg_vcycle (one
 * multigrid cycle as the preconditioner P^-1, Sec. 5.1 "Exit criterion"),
 * starting from the x passed in. DGMG_OUTER_PCG: FP64 residual, update and dot
 * products every iteration (flexible Polak-Ribiere form with the FP32 V-cycle).
 * DGMG_OUTER_RELIABLE (mixed precision): the CG recurrences run in FP32 with
 * FP64-accumulated dot products; the solution is accumulated in FP64 and the
 * true residual b - A x is recomputed in FP64 whenever the FP32 residual has
 * dropped by `delta` and before stopping (outer residual, solution update and
 * coarsest solve stay FP64). Stops when ||b - A x||_2 <= rtol ||b||_2 (PCG: on
 * the recursive residual, then verified), reports the recomputed residual in
 * stats (HOST struct, may be NULL). DGMG_OUTER_MGMULT / _PREC run the stationary
 * iteration of Alg. 7 instead (iterations = cycles; prec_residual = ||x_k - x_(k-1)|| /
 * ||x_1 - x_0|| of the last cycle; rel_residual the true residual of the last
 * cycle). Blocks until done (it reads one scalar per
 * iteration). Returns DGMG_ENOTCONVERGED after maxit iterations,
 * DGMG_ENONFINITE if a residual norm is not finite, DGMG_ETIMEOUT (which
 * takes precedence) if a bounded device-side wait of the library ran out on
 * this device while the solve ran (read from the wait counters at its start
 * and end; see dgmg_wait_timeouts).
 */
int dgmg_solve(dgmg_ctx *ctx, const double *b, double *x, dgmg_stats *stats, void *stream);

/*
 * dgmg_solve (same method) with HOST vectors: copies b and x (initial guess)
 * to the ctx's device buffers, solves, copies x back. b_host, x_host: ndof doubles each
 * (pinned memory gives the fastest copies). Blocks until x_host is written.
 */
int dgmg_solve_host(dgmg_ctx *ctx, const double *b_host, double *x_host, dgmg_stats *stats,
                    void *stream);

/*
 * b_i = (f, phi_i) (Sec. 2.3.1 right-hand side) from f sampled at the (p+2)^d
 * Gauss-Legendre points of every cell: fq is a DEVICE array [ncell][(p+2)^d]
 * (x fastest within a cell), b a DEVICE DG vector. dgmg_quad_points writes the
 * physical coordinates of those points, DEVICE array [ncell][(p+2)^d][dim].
 */
int dgmg_quad_points(dgmg_ctx *ctx, double *xq, void *stream);
int dgmg_load_vector(dgmg_ctx *ctx, const double *fq, double *b, void *stream);

/*
 * Sizing for the server's admission (no counterpart in the paper).
 * Device bytes dgmg_create would hold for this problem (exact byte count of its
 * allocations, before allocator rounding). HOST output.
 */
int dgmg_estimate_bytes(const dgmg_mesh *mesh, int p, const dgmg_opts *opts, size_t *bytes);

/* ---- serving: continuous batching of independent solves ---- */

/*
 * Serving (the paper has no counterpart: independent solves of the method,
 * as dgmg_solve, scheduled together).
 * Start a solve server on the current device: at most `max_active` solves run
 * at once (each on its own stream, advanced one CG iteration at a time by a
 * scheduler thread, so their kernels overlap), and the hierarchies it keeps
 * resident (busy or idle, reused for repeated problems, least recently used
 * idle ones evicted first) never exceed `hbm_budget_bytes`. opts (NULL =
 * defaults) apply to every request.
 * The scheduler captures repeated CG iterations into CUDA graphs on its own
 * streams. Meanwhile other threads of the process should synchronise streams
 * or events, not the whole device: a device-wide synchronisation during a
 * capture fails in the caller (cudaErrorStreamCaptureUnsupported); the server
 * then finishes the affected solves without graphs, with the same results.
 */
int dgmg_server_create(size_t hbm_budget_bytes, int max_active, const dgmg_opts *opts, dgmg_server **out);

/*
 * Queue a solve of A x = b for (mesh, p, kappa_host) and return at once with a
 * ticket. kappa_host (HOST, ncell values, NULL = 1) is copied. b_dev, x_dev:
 * caller-owned DEVICE vectors (x_dev holds the initial guess and receives the
 * solution); they must be ready when dgmg_submit is called and stay alive
 * until dgmg_poll reports DGMG_DONE or DGMG_FAILED. Requests that can never
 * fit the budget fail with DGMG_EBUDGET. Thread-safe.
 */
int dgmg_submit(dgmg_server *server, const dgmg_mesh *mesh, int p, const double *kappa_host,
                const double *b_dev, double *x_dev, uint64_t *ticket);

/*
 * State of a ticket (DGMG_PENDING / RUNNING / DONE / FAILED) and, once finished,
 * its stats (HOST, may be NULL; `seconds` = submit to completion, `queue_seconds`
 * = submit to admission). Returns the request's error code when it FAILED.
 * DONE or FAILED is reported once: that poll releases the request's record, and
 * later polls of the ticket return DGMG_EINVAL (unknown ticket). Thread-safe.
 */
int dgmg_poll(dgmg_server *server, uint64_t ticket, int *status, dgmg_stats *stats);

/* Counters of the server (HOST struct). */
int dgmg_server_info(dgmg_server *server, dgmg_server_info_t *info);

/* Fail the queued requests, finish the running ones, free everything. */
int dgmg_server_destroy(dgmg_server *server);

/* ---- batched solves: independent problems sharing one launch per stage ---- */

typedef struct dgmg_batch dgmg_batch;

typedef struct {
    int count;                    /* problems in the batch                             */
    int groups;                   /* DG launch groups (one per polynomial degree)      */
    int64_t ndof;                 /* length of the batch vectors (with padding)        */
    size_t device_bytes;          /* device memory of the problems' hierarchies        */
    int max_levels;               /* deepest Q1 hierarchy of the batch                 */
    long long kernels_per_iteration; /* kernels in one CG iteration of the whole batch */
                                  /* (0 before the first solve); independent of count  */
    int group_q[4];               /* nodes per axis of the first four groups           */
    int group_tiles[4][3];        /* their cells per CTA: projection, smoothing (0 =   */
                                  /* one thread per cell), residual                    */
} dgmg_batch_info_t;

/*
 * Batching (the paper has no counterpart: independent problems, each solved
 * as dgmg_solve, sharing launches).
 * Build `count` independent problems (meshes[i], degree p[i] in 1..6,
 * kappa[i]: HOST array of the mesh's ncell positive values or NULL = 1; kappa
 * itself may be NULL) for batched solving: each problem gets its own hierarchy
 * (as dgmg_create), and the problems of equal degree share one launch per
 * DG-level stage (projection, smoothing step, residual + p-restriction), all
 * problems share one launch per Q1-level stage (point Jacobi, residual,
 * h-restriction, h-prolongation, vertex gather, dense coarsest solve). All
 * meshes have the same dimension. opts (NULL = defaults) apply to every
 * problem; nu_pre >= 1 (DGMG_EINVAL otherwise). precision DGMG_FP64, or
 * DGMG_MIXED_FP32: reliable-update CG as in dgmg_solve, batched: the CG
 * recurrences, V-cycle and operator in FP32 (the dense coarsest solve stays
 * FP64; flexible Polak-Ribiere beta, FP64 dot products), the FP64 solution and
 * true residuals refreshed for the whole batch at reliable updates (`delta`).
 * With opts->autotune the cells per CTA of each group's launches are timed and
 * chosen on the batch itself. Synchronous.
 */
int dgmg_batch_create(int count, const dgmg_mesh *meshes, const int *p, const double *const *kappa,
                      const dgmg_opts *opts, dgmg_batch **out);

int dgmg_batch_info(const dgmg_batch *batch, dgmg_batch_info_t *info);

/*
 * Solve A_i x_i = b_i for every problem: preconditioned conjugate gradients
 * (FP64, or the mixed-precision reliable-update form) with the problem's own
 * hp V-cycle, one CG recurrence per problem (its own alpha and beta), all
 * problems advanced by the same batched launches; a problem that met
 * ||b_i - A_i x_i||_2 <= rtol ||b_i||_2 (FP64 true residual) stops changing
 * while the others continue. b[i], x[i]: DEVICE vectors of problem i
 * (x[i] holds the initial guess and receives the solution). stats: HOST array
 * of `count` (may be NULL): each problem's iterations and recomputed true
 * residual. Blocks until done. DGMG_ENOTCONVERGED after maxit iterations.
 */
int dgmg_batch_solve(dgmg_batch *batch, const double *const *b, double *const *x, dgmg_stats *stats,
                     void *stream);

int dgmg_batch_destroy(dgmg_batch *batch);

/* ---- stage entry points: the individual steps of the path, for testing ---- */

/*
 * Warm-up projection (Alg. 4 preamble, Eq. solution_projection /
 * gradient_projection), optionally fused with the p-prolongation u += P e
 * (Eq. prolongation, Sec. 5.1 "Prolongation"): e is a DEVICE Q1 vector of
 * level 0 or NULL; u (in/out when e != NULL). traces: DEVICE output
 * [ncell][2d faces][2][q^(d-1)] doubles, face = 2*axis + (0 low, 1 high end),
 * component 0 = value, 1 = derivative along +axis; face node index = the
 * remaining axes, lowest axis fastest. FP64.
 */
int dgmg_project(dgmg_ctx *ctx, double *u, const double *e, double *traces, void *stream);

/*
 * Residual r = b - A u and p-restriction rc = P^T r (Alg. 6, the restriction
 * fused into the residual traversal), given the projections `traces` of u
 * (layout of dgmg_project). r may be NULL (not written); rc (DEVICE Q1 vector
 * of level 0) may be NULL. FP64.
 */
int dgmg_residual_restrict(dgmg_ctx *ctx, const double *u, const double *b,
                           const double *traces, double *r, double *rc, void *stream);

/*
 * Same result as dgmg_residual_restrict, without allocating anything: for
 * callers that cannot allocate device memory when they call (loops that
 * forbid allocation after start-up, fixed memory budgets that leave no room
 * for a per-context scratch, hosts whose allocator is not available at the
 * point of the call). The paper has no counterpart; this is an interface
 * variant of the residual + p-restriction stage.
 * The 2^d corner partial sums per cell go to one fixed device array of 2^21
 * doubles (16 MiB) that every GPU loading the library keeps until exit;
 * meshes needing more (more than 262,144 hexahedra or 524,288 quadrilaterals)
 * are rejected with DGMG_EINVAL. The first call on a device looks up that
 * array's device address (a one-time set-up per device, made with that device
 * current). All calls share
 * the array: calls whose GPU work overlaps in time (other streams, other
 * threads, other contexts on the same device) race and must be serialised
 * by the caller. Every call overwrites the sums it reads, so no clearing is
 * needed between calls.
 */
int dgmg_residual_restrict_noalloc(dgmg_ctx *ctx, const double *u, const double *b,
                                   const double *traces, double *r, double *rc, void *stream);

/* Q1 level `level` (0 = first Q1 level): `nsteps` damped point-Jacobi steps
 * u <- u + omega_cg D^{-1}(b - A_l u) (Sec. 2.4), FP64, u in/out. */
int dgmg_cg_smooth(dgmg_ctx *ctx, int level, double *u, const double *b, int nsteps,
                   void *stream);

/* Q1 level `level`: r = b - A_l u (A_l the Galerkin operator, Sec. 2.4, 5.2). */
int dgmg_cg_residual(dgmg_ctx *ctx, int level, const double *u, const double *b, double *r,
                     void *stream);

/* h-restriction rc = P_h^T rf from level `level` to level+1 (Sec. 5.2). */
int dgmg_h_restrict(dgmg_ctx *ctx, int level, const double *rf, double *rc, void *stream);

/* h-prolongation uf += P_h ec from level+1 to level `level` (Sec. 5.2). */
int dgmg_h_prolong(dgmg_ctx *ctx, int level, const double *ec, double *uf, void *stream);

/* Coarsest-level solve e = A_c^{-1} r (dense, FP64; Alg. 6 coarse solve). */
int dgmg_coarse_solve(dgmg_ctx *ctx, const double *r, double *e, void *stream);

/* Unknowns of Q1 level `level` (HOST query); -1 if out of range. */
int64_t dgmg_cg_size(const dgmg_ctx *ctx, int level);

/*
 * The volume term of the operator on its own, r = b - kappa_K E u_K for every
 * cell, where E is the element stiffness matrix of a unit coefficient, the
 * cell integral (grad u, grad v)_K of Eq. weak_form_IP, one dense q^3 x q^3
 * matrix shared by all cells of the uniform mesh (Sec. 4.1: the dense local
 * mat-vecs): the cell contraction that could run on the tensor cores, exposed
 * to measure that choice. 3D, p = 4 (q = 5) only. u, b, r: DEVICE FP32 DG
 * vectors (layout as above, 16-byte aligned, r aliasing neither u nor b);
 * kappa is ctx's coefficient. method 0: sum factorisation on the CUDA cores
 * (FP32; the shared generalised eigenvectors of the 1D stiffness and mass
 * factor E into six passes of q x q matrices); method 1: a dense contraction
 * D = U E^T on the tensor cores (tcgen05, TF32 operands, FP32 accumulation,
 * tiles of 128 cells; results to TF32 accuracy, about 1e-3 relative). The
 * first call builds E and the factors (a one-time device allocation in ctx).
 * DGMG_EINVAL for another dimension or degree, or misaligned vectors.
 */
int dgmg_volume_residual_f32(dgmg_ctx *ctx, const float *u, const float *b, float *r, int method, void *stream);

/*
 * y = A u in FP32 on the finest level of a DGMG_MIXED_FP32 ctx: the operator of
 * the FP32 CG recurrences of the reliable-update solver (Eq. matrix_form_IP,
 * the cell equation of Alg. 2 stage 3 with b = 0), exposed to test and time its
 * forms. u, y: DEVICE FP32 DG vectors (layout as above, 16-byte aligned for the
 * one-thread-per-cell forms), y not aliasing u; ctx's FP32 traces are scratch.
 * form 0: the solver's choice (form 1 or the one-thread-per-cell kernel with
 * A_KK u in the direct sum-factorised form sum_a Kt_a (x) M (x) M, which keeps
 * the rounding of form 1); form 1: the per-pencil kernel; form 2: one thread per
 * cell with A_KK u through the fast-diagonalisation factors (the V-cycle's
 * residual; its FP32 rounding costs the CG recurrences iterations). All forms
 * agree to FP32 rounding. DGMG_EINVAL for an FP64 ctx, NULL or aliasing vectors,
 * another form, or form 2 on a ctx with interior-only blocks
 * (DGMG_BLOCK_INTERIOR_ONLY, whose factors are not those of A_KK).
 */
int dgmg_apply_f32(dgmg_ctx *ctx, const float *u, float *y, int form, void *stream);

/* ---- instrumentation ---- */

/*
 * Per-stage device time: while enabled, every stage launch of ctx is bracketed
 * by CUDA events recorded on the launching stream. Stages (index into the
 * arrays of dgmg_profile_read): 0 projection, 1 smoothing step, 2 residual
 * (apply / residual / residual+restriction), 3 Q1 levels (vertex gather,
 * h-cycle, coarsest solve), 4 vector kernels of the outer CG loop.
 * dgmg_profile(ctx, on) enables or disables it and clears the accumulators.
 */
int dgmg_profile(dgmg_ctx *ctx, int enable);

/* Waits for the recorded events and writes, for the first nstage stages, the
 * summed milliseconds and the number of timed launches since the last read
 * (HOST arrays); then clears the accumulators. */
int dgmg_profile_read(dgmg_ctx *ctx, double *ms, long long *launches, int nstage);

/* Number of CUDA kernels this library has launched in this process. */
long long dgmg_kernel_launches(void);

/*
 * Arithmetic peak of the current device, measured: a kernel in which every
 * thread runs 8 independent chains of fused multiply-adds, launched with 1, 2,
 * 4, ... resident 256-thread blocks per SM up to the occupancy limit (a few
 * tens of milliseconds each), timed with CUDA events on `stream`; the best
 * launch shape gives the result. kind: 0 = FP64 FMA, 1 = FP32 FMA, 2 = FP32 FMA on packed pairs
 * (two lanes of one instruction). *tflops (HOST) receives 2 x FMAs / time in
 * TFLOP/s: the denominator of the roofline fraction of the FP64 kernels, which
 * are bound by the FP64 pipe on this chip. Synchronous; allocates nothing.
 * DGMG_EINVAL for another kind or a NULL pointer.
 */
int dgmg_fma_peak(int kind, double *tflops, void *stream);

/* Bounded device-side waits that ran out of iterations on the CURRENT device
 * since the library was loaded: the mbarrier phases of the bulk copies in the
 * one-thread-per-cell kernels, and the grid barrier of the Q1 cycle run as one
 * cooperative launch. 0 in every healthy run. A smoothing kernel whose wait
 * runs out abandons its cells for that launch (their u and traces keep the old
 * values); after a grid-barrier wait ran out, every later Q1 cycle launch
 * returns without work. A nonzero count means the results are not to be trusted.
 * Solves (dgmg_solve, dgmg_solve_host, served requests through dgmg_poll)
 * check the counters themselves and return DGMG_ETIMEOUT. Recovery: after a
 * grid-barrier time-out every context of the process switches to the launch
 * per step of the Q1 levels (their CUDA graphs are captured again), so later
 * solves are correct; after a bulk-copy time-out nothing is switched off, and
 * the next solve runs normally.
 * Synchronous (reads device memory); *count (HOST) receives the number.
 * Returns DGMG_EINVAL for a NULL pointer, DGMG_ECUDA if the read fails. */
int dgmg_wait_timeouts(unsigned long long *count);

#ifdef __cplusplus
}
#endif
#endif /* DGMG_H */
