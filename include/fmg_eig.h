/*
 * fmg_eig.h - C ABI of the GB300 full-multigrid solver for the Gross-Pitaevskii ground state.
 *
 * Method: Jia, Xie, Xie, Xu, "A Full Multigrid Method for Nonlinear Eigenvalue Problems"
 * (arXiv:1502.04657).  The problem is Example 4.1 (Section 4):
 *
 *     -Lap u + W u + zeta u^3 = lambda u  in [0, L]^d,  u = 0 on the boundary,  int u^2 = 1,
 *
 * with W(x) = w_const + sum_d w_quad[d] x_d^2, discretised by P1 finite elements (Section 2)
 * on nested, regularly refined structured meshes (Section 3: beta = 2): 2D squares split by
 * their (1,1) diagonal, 3D cubes split into 6 Kuhn tetrahedra.  fmg_eig_solve runs the full
 * multigrid scheme (Algorithm 3.2): a direct nonlinear solve on the coarsest level, then on
 * every finer level p correction steps (Algorithm 3.1), each = m multigrid V-cycles on the
 * auxiliary linear problem followed by the nonlinear eigenproblem on V_H + span{u~}.
 *
 * Conventions (every entry point):
 *   - Return 0 (FMG_OK) or a negative FMG_E* code; nothing is thrown across the ABI.
 *   - Vectors u on level k are FP64, interior nodes only, lexicographic with x fastest:
 *     (n_k - 1)^d entries, n_k = coarse_cells << (k - 1) cells per side.  Dirichlet values
 *     are zero and are not stored.
 *   - The library owns every device buffer it allocates; the caller owns the buffers it
 *     passes.  "_dev" pointers are device memory on the handle's device, other pointers are
 *     host memory (pinned or pageable).
 *   - A handle is not thread-safe: use one handle per host thread.  All work of a handle is
 *     ordered on the stream passed to the call (NULL = the handle's own stream).
 *   - Every device-side loop (SCF/Newton iterations) is bounded; a bound that is hit is
 *     reported as FMG_ENOCONV with the partial result still written.  Every device-side wait
 *     (the mbarrier waits of the TMA-fed sweeps) is bounded too; one that gives up is
 *     reported as FMG_ETIMEOUT for its instance (it outranks FMG_ENOCONV), and that
 *     instance's results are not meaningful.
 */
#ifndef FMG_EIG_H
#define FMG_EIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FMG_OK 0
#define FMG_EINVAL (-1)   /* invalid argument or size */
#define FMG_ENOMEM (-2)   /* device allocation failed */
#define FMG_ENOCONV (-3)  /* a nonlinear solve hit its iteration cap */
#define FMG_ECUDA (-4)    /* a CUDA runtime call failed */
#define FMG_ETIMEOUT (-5) /* a bounded device wait gave up */
#define FMG_ENOTSUP (-6)  /* combination of options not built */

#define FMG_SMOOTH_JACOBI 0    /* damped Jacobi, omega, nu_pre / nu_post sweeps            */
/* Chebyshev semi-iteration of degree nu_pre / nu_post on [0.3, 2] for the spectrum of
 * D^{-1} L (2 = Gershgorin's bound for these operators; omega is not used); FMG_FP64 only */
#define FMG_SMOOTH_CHEBYSHEV 1
/* nu_pre / nu_post steps of the conjugate gradient method (no preconditioner) on L_j x = f
 * from the current x: the smoother of the paper's experiments (Section 4, 3 + 3 steps);
 * omega is not used; FMG_FP64 only                                                          */
#define FMG_SMOOTH_CG 2
#define FMG_FP64 0
#define FMG_MIXED_FP32 1
/* the same FP64 defect correction with the V-cycle's vectors and coefficients stored in
 * bfloat16 (arithmetic in FP32): a storage ablation of FMG_MIXED_FP32                      */
#define FMG_MIXED_BF16 2
#define FMG_W_LEFT 0        /* (A + W) u^ = lambda M u - N(u)              */
#define FMG_PAPER_LITERAL 1 /*  A u^      = lambda M u - W u - N(u)        */
/* flags: keep the default 32 x 8 thread blocks instead of timing the candidate block shapes
 * of every level when the handle is created (results do not depend on the shapes).        */
#define FMG_FLAG_NO_AUTOTUNE 1
/* flags (with FMG_MIXED_FP32 / FMG_MIXED_BF16 only): evaluate the auxiliary right-hand side lambda M u - N(u)
 * of Algorithm 3.1 step 1 in FP32 as well.  Faster (the FP64 evaluation is a large share of
 * a mixed solve) but its rounding, ~1e-7 of |f|, enters u~ directly: measured |d lambda| up
 * to 7.6e-9 relative against FP64 (3D, W = 100(x^2 + y^2 + 4z^2), zeta = 100), against
 * 1.9e-9 with the default FP64 right-hand side.                                            */
#define FMG_FLAG_FP32_RHS 2
/* flags (with FMG_MIXED_FP32 / FMG_MIXED_BF16): run every single-precision Jacobi sweep and
 * residual with the register-blocked kernels instead of the TMA-fed ones that the levels
 * with at least 512 (2D) or 128 (3D) cells per side use by default.  Both compute every node with the same
 * expression, so the results are bit-identical; the flag exists for comparison and for
 * drivers where tensor maps cannot be encoded (the library also falls back by itself).     */
#define FMG_FLAG_NO_TMA 4
/* flags: evaluate the FP64 cubic load, auxiliary right-hand side and density stencil as
 * column (2D) or plane (3D) walks on every level.  The walks form each mesh edge's (2D) or
 * tetrahedron's (3D) share of the exact integrals of Section 2 once, for all the nodes that
 * need it; by default they are taken only where the launch gives them at least two blocks
 * per SM, and smaller launches run node by node.  Both evaluate the same closed forms, so
 * results agree to rounding; the flag exists for comparison and testing.                   */
#define FMG_FLAG_STAR_WALKS 8
/* flags (test hook, no counterpart in the paper): every bounded device wait of the solve's
 * TMA-fed sweeps (FMG_MIXED_FP32 / FMG_MIXED_BF16 levels with at least 512 (2D) or 128 (3D)
 * cells per side) gives up at once instead of after its normal bound.  The sweep then takes
 * the path of a wait that ran out: it records the instance in the solve's status word,
 * writes NaN over its tile, waits (with the normal bound) for its own loads in flight and
 * returns, and the solve reports FMG_ETIMEOUT for that instance.  This exercises the timeout
 * path without a fault or a hang; results of such a solve are not meaningful.               */
#define FMG_FLAG_EXPIRE_WAITS 32
/* flags: run the fused levels of V-cycles as separate kernels, one per sweep and transfer:
 * the 2D FP64 levels of at most 32 cells per side (damped Jacobi; otherwise one kernel per
 * V-cycle with one CTA per instance) and the single-precision levels below the TMA-fed ones
 * of at most 256 cells (2D) or 32 cells (3D) per side (mixed modes; otherwise two kernels per
 * level on 32 x 32 or 8 x 8 x 8 tiles).  Both evaluate the same expressions in the same
 * order, so the results are bit-identical; the flag exists for comparison and testing.      */
#define FMG_FLAG_SEPARATE_VCYCLE 16

/* Problem and method parameters.  Example 4.1 fixes the PDE; Algorithm 3.1 fixes m (vcycles)
 * and Algorithm 3.2 fixes p (corrections) and the level count n.                            */
typedef struct fmg_eig_problem {
  int32_t dim;          /* 2 or 3                                                          */
  int32_t coarse_cells; /* cells per side of T_H = T_{h_1}; >= 2                           */
  int32_t levels;       /* n >= 1; finest cells per side = coarse_cells << (levels - 1)    */
  int32_t nu_pre;       /* damped-Jacobi pre-smoothing sweeps per V-cycle level (>= 0)     */
  int32_t nu_post;      /* post-smoothing sweeps (>= 0)                                    */
  int32_t vcycles;      /* m of Algorithm 3.1 (>= 1)                                       */
  int32_t corrections;  /* p of Algorithm 3.2 (>= 1)                                       */
  int32_t smoother;     /* FMG_SMOOTH_JACOBI | FMG_SMOOTH_CHEBYSHEV | FMG_SMOOTH_CG        */
  int32_t precision;    /* FMG_FP64 | FMG_MIXED_FP32 | FMG_MIXED_BF16                      */
  int32_t operator_form;/* FMG_W_LEFT | FMG_PAPER_LITERAL                                  */
  int32_t scf_max_iter; /* cap on nonlinear iterations per small solve (e.g. 100)          */
  int32_t flags;        /* FMG_FLAG_* bits (0 = defaults)                                  */
  double box_len;       /* L > 0                                                           */
  double w_const;       /* W(x) = w_const + sum_d w_quad[d] x_d^2                          */
  double w_quad[3];
  double zeta;          /* >= 0                                                            */
  double omega;         /* Jacobi damping, 0 < omega <= 1 (2/3)                            */
  double scf_tol;       /* relative residual tolerance of the small nonlinear solves       */
} fmg_eig_problem;

#define FMG_MAX_LEVELS 16

typedef struct fmg_eig_stats {
  double lambda;                        /* final eigenvalue                                */
  double solve_ms;                      /* device time of the solve (CUDA events)          */
  double norm_defect;                   /* b(u,u) - 1 on the finest level                  */
  double identity_defect;               /* lambda - a(u,u) - (Wu,u) - zeta int u^4         */
  double lambda_levels[FMG_MAX_LEVELS]; /* lambda_{h_k} after level k                      */
  int32_t scf_iters[FMG_MAX_LEVELS];    /* nonlinear iterations of the last small solve    */
  int32_t levels;
  int32_t status;                       /* FMG_OK or FMG_ENOCONV                           */
} fmg_eig_stats;

typedef struct fmg_eig_handle fmg_eig_handle;

/* Validate *prob, allocate the level hierarchy on the current CUDA device and record the
 * solve as a CUDA graph.  Returns FMG_EINVAL for a bad parameter, FMG_ENOMEM if device
 * memory runs out (nothing stays allocated then), FMG_ECUDA for other CUDA failures.      */
int fmg_eig_create(const fmg_eig_problem* prob, fmg_eig_handle** out);

/* Number of interior unknowns of level k (1-based) of this handle, 0 for a bad k.          */
size_t fmg_eig_level_size(const fmg_eig_handle* h, int32_t level);

/* Algorithm 3.2 end to end with host buffers: writes lambda_{h_n} to *lambda and, when
 * u_host is not NULL, u_{h_n} (u_len must equal fmg_eig_level_size(h, levels)).  stats may
 * be NULL.  Synchronous.                                                                    */
int fmg_eig_solve(fmg_eig_handle* h, double* lambda, double* u_host, size_t u_len,
                  fmg_eig_stats* stats);

/* Same solve with device outputs and no host synchronisation: lambda_dev (1 double) and
 * u_dev (nullable, u_len doubles) are written in stream order on `stream` (a cudaStream_t,
 * NULL for the handle's stream).                                                            */
int fmg_eig_solve_dev(fmg_eig_handle* h, double* lambda_dev, double* u_dev, size_t u_len,
                      void* stream);

/* Release every device buffer, graph and stream of the handle.  NULL is ignored.           */
void fmg_eig_destroy(fmg_eig_handle* h);

/* Change the potential (w_const, w_quad), zeta and omega of an existing handle: the PDE of
 * Example 4.1 with new coefficients on the same mesh hierarchy.  Every other field of *prob
 * must equal the handle's (FMG_EINVAL otherwise).  Synchronises the handle's stream; the
 * next solve uses the new values (they are uploaded from pinned host memory per solve).   */
int fmg_eig_set_params(fmg_eig_handle* h, const fmg_eig_problem* prob);

/* Instrumentation (no counterpart in the paper).  fmg_eig_kernel_count: kernel launches
 * per solve (nodes of the solve's CUDA graph).  fmg_eig_profile: device time in ms of the
 * finest-level launch of each step in the most recent solve, in the order
 * [Jacobi sweep, residual, restriction, prolongation, auxiliary RHS, cubic load + density
 * stencil of u~, augmented nonlinear solve, one whole V-cycle, T3 moments, operator setup];
 * writes min(count, 10) entries and returns that number (FMG_EINVAL for bad arguments).
 * Entries a solve does not contain read -1.  Synchronises the handle's stream.             */
int fmg_eig_kernel_count(const fmg_eig_handle* h);
int fmg_eig_profile(fmg_eig_handle* h, double* ms, int32_t count);

/* Arithmetic-throughput probe (instrumentation, no counterpart in the paper): the rate of
 * fused multiply-adds this GPU sustains, the denominator of the roofline of the FP64-bound
 * kernels of this library.  Launches ctas_per_sm (1..8) blocks per SM of 256 threads, each
 * thread running 4 (fp64 != 0: FP64) or 8 (FP32) independent chains of `iters`
 * multiply-adds in registers, once to warm up and once timed with CUDA events on `stream`
 * (NULL = legacy default stream).  Writes the timed launch's duration in ms to *ms_out and its flop
 * count (2 per multiply-add) to *flops_out.  Allocates nothing; synchronous.               */
int fmg_eig_probe_fma(int32_t fp64, int32_t ctas_per_sm, int32_t iters, void* stream,
                      double* ms_out, double* flops_out);

/* Fault injection for tests (no counterpart in the paper): after `after` more device
 * allocations by the library in this process succeed, the next one fails as if the device
 * were out of memory, once; later allocations succeed again.  A negative value cancels a
 * pending injection.  The failed call reports FMG_ENOMEM and releases what it had allocated
 * (fmg_eig_create, fmg_eig_batch_create); fmg_eig_serve retries or rejects the cohort whose
 * allocation failed and serves the others.  Returns FMG_OK.                                 */
int fmg_eig_inject_alloc_failure(int64_t after);

/* Static description of a return code.                                                    */
const char* fmg_eig_strerror(int code);

/* ------------------------------------------------------------------------------------------
 * Batches: many independent instances of Example 4.1 solved together (no counterpart in the
 * paper, whose algorithms solve one problem).  The instances may differ in the level count
 * (mesh size), w_const, w_quad, zeta and omega; every other field must be equal (FMG_EINVAL
 * otherwise).  Every step of Algorithm 3.2 on level k runs as one launch over all instances
 * that have a level k, and the whole batch is one CUDA graph.
 * ---------------------------------------------------------------------------------------- */

/* Create a batch handle for probs[0 .. count-1] (count >= 1).  Errors as fmg_eig_create,
 * plus FMG_ENOTSUP when a 3D level holds more instances than one launch can address.       */
int fmg_eig_batch_create(const fmg_eig_problem* probs, int32_t count, fmg_eig_handle** out);

/* Instances of a handle (1 for fmg_eig_create).                                           */
int32_t fmg_eig_batch_count(const fmg_eig_handle* h);

/* Solve every instance of a batch handle.  lambdas: count doubles (host).  u_hosts
 * (nullable): count host pointers, each NULL or a buffer of u_lens[i] doubles, u_lens[i]
 * equal to instance i's finest level size.  stats (nullable): count records; statuses
 * (nullable): count codes.  Returns FMG_OK when every instance converged, FMG_ENOCONV when
 * some did not (their partial results are written), or an error code.  Synchronous.      */
int fmg_eig_batch_solve(fmg_eig_handle* h, double* lambdas, double* const* u_hosts,
                        const size_t* u_lens, fmg_eig_stats* stats, int32_t* statuses);

/* Device-side batch solve without host synchronisation: lambdas_dev (count doubles, device,
 * caller's order) is written in stream order on `stream` (NULL = the handle's stream).    */
int fmg_eig_batch_solve_dev(fmg_eig_handle* h, double* lambdas_dev, void* stream);

/* One-shot batch: groups probs by the fields that must agree, creates one batch handle per
 * group, runs the groups concurrently on their own streams, writes the outputs as
 * fmg_eig_batch_solve does (in the caller's order) and releases everything.              */
int fmg_eig_solve_batch(const fmg_eig_problem* probs, int32_t count, double* lambdas,
                        double* const* u_hosts, const size_t* u_lens, fmg_eig_stats* stats,
                        int32_t* statuses);

/* ------------------------------------------------------------------------------------------
 * Serving (no counterpart in the paper): a stream of independent solve requests, each with an
 * arrival time, served with continuous batching on one GPU.  Requests that have arrived are
 * admitted as a cohort (one batch handle: every step of each level one launch for all of
 * them) as soon as fewer than max_inflight cohorts are in flight and the cohort's hierarchy
 * fits the device-memory budget; each cohort runs on its own stream, so newly admitted
 * cohorts overlap with the ones already on the GPU.  Hierarchies stay resident in device
 * memory: a finished cohort's hierarchy (with its recorded CUDA graph) is pooled and replayed
 * by a later cohort with the same level counts and settings, and pooled hierarchies are
 * released (stream-ordered, oldest first) when an admission needs their memory.
 * ---------------------------------------------------------------------------------------- */
typedef struct fmg_eig_serve_config {
  double hbm_budget_bytes; /* device bytes for resident hierarchies; <= 0: 80% of free    */
  double batch_window_s;   /* a queued request waits at most this long for others to join */
  int32_t max_batch;       /* instances per cohort (>= 1)                                 */
  int32_t max_inflight;    /* cohorts resident at once (>= 1)                             */
} fmg_eig_serve_config;

typedef struct fmg_eig_request {
  fmg_eig_problem problem;
  double arrival_s; /* seconds after the start of the fmg_eig_serve call (non-decreasing)  */
  double* u;        /* nullable host buffer for u (u_len doubles, the finest level size)   */
  size_t u_len;
} fmg_eig_request;

typedef struct fmg_eig_result {
  double lambda;
  double latency_s; /* arrival -> lambda copied to host memory (GPU clock of that copy)    */
  double admit_s;   /* when its cohort was admitted, seconds after the start              */
  double done_s;    /* arrival_s + latency_s                                              */
  int32_t status;   /* FMG_OK, FMG_ENOCONV, or an error code of its cohort                */
  int32_t cohort;   /* index of the cohort it ran in                                      */
} fmg_eig_result;

typedef struct fmg_eig_serve_stats {
  double p50_s, p99_s, mean_s, max_s; /* latency percentiles (nearest rank)               */
  double solves_per_s;                /* requests / (last done - first arrival)           */
  double makespan_s;                  /* last done - first arrival                        */
  double peak_bytes;                  /* most device bytes held by resident hierarchies   */
  double budget_bytes;                /* the budget admission used                        */
  int32_t cohorts;                    /* cohorts admitted                                 */
  int32_t max_cohort;                 /* largest cohort                                   */
  int32_t max_inflight_seen;          /* most cohorts resident at once                    */
  int32_t completed;                  /* requests with a result                           */
  int32_t reused;                     /* cohorts that replayed a pooled hierarchy's graph */
  int32_t evicted;                    /* pooled hierarchies released to admit others      */
} fmg_eig_serve_stats;

/* Device bytes a batch handle for probs[0 .. count-1] allocates (an upper bound; 0 for bad
 * arguments).  The server admits cohorts against its budget with these figures.          */
size_t fmg_eig_estimate_bytes(const fmg_eig_problem* probs, int32_t count);

/* Serve reqs[0 .. n-1] (arrival order) and return when every request has a result.  Each
 * result is the request's solve alone (a cohort changes which launches an instance shares,
 * not its arithmetic).  Returns FMG_OK, FMG_ENOCONV when some request did not converge,
 * FMG_EINVAL for bad arguments (a request that can never fit the budget included).         */
int fmg_eig_serve(const fmg_eig_serve_config* cfg, const fmg_eig_request* reqs, int32_t n,
                  fmg_eig_result* results, fmg_eig_serve_stats* stats);

/* Thread-block shape (x, y threads) the handle uses for the stencil kernels of level k,
 * as chosen by the autotuner when the handle was created.                                 */
int fmg_eig_level_tile(const fmg_eig_handle* h, int32_t level, int32_t* bx, int32_t* by);

/* ------------------------------------------------------------------------------------------
 * Component entry points: the steps of the hot path, one call each, on device vectors in the
 * interior layout above.  Each call is asynchronous on `stream` (NULL = handle's stream) and
 * uses the handle's level buffers as scratch, so calls on one handle must not overlap.
 * ---------------------------------------------------------------------------------------- */

/* y = L_k x with L = A + W (FMG_W_LEFT) or A (FMG_PAPER_LITERAL): the operator of the
 * auxiliary problem of Algorithm 3.1 step 1 (Section 2, the forms a^ and (W u, v)).          */
int fmg_eig_apply_operator(fmg_eig_handle* h, int32_t level, const double* x_dev,
                           double* y_dev, void* stream);

/* y = M_k x, the mass matrix of b(u, v) = int u v (Section 2).                             */
int fmg_eig_apply_mass(fmg_eig_handle* h, int32_t level, const double* x_dev, double* y_dev,
                       void* stream);

/* One damped Jacobi sweep x_out = x_in + omega D^{-1} (f - L_k x_in) (the smoother of the
 * multigrid iteration of Algorithm 3.1 step 1); omega = 1 on a handle whose smoother is
 * FMG_SMOOTH_CHEBYSHEV.                                                                     */
int fmg_eig_jacobi(fmg_eig_handle* h, int32_t level, const double* f_dev,
                   const double* x_in_dev, double* x_out_dev, void* stream);

/* r_c = P_k^T (f - L_k x): fine residual restricted to level k-1 (k >= 2).                 */
int fmg_eig_residual_restrict(fmg_eig_handle* h, int32_t level, const double* f_dev,
                              const double* x_dev, double* rc_dev, void* stream);

/* x += P_k e_c: coarse correction of level k-1 prolonged to level k (k >= 2); the nested
 * space embedding of Section 3.                                                             */
int fmg_eig_prolong_add(fmg_eig_handle* h, int32_t level, const double* ec_dev, double* x_dev,
                        void* stream);

/* n_i = int u^3 phi_i on level k (the cubic part of f(x, u) of Example 4.1, without zeta). */
int fmg_eig_nonlinear_load(fmg_eig_handle* h, int32_t level, const double* u_dev,
                           double* n_dev, void* stream);

/* f = lambda M_k u - zeta N(u) [- W_k u for FMG_PAPER_LITERAL]: the right-hand side of the
 * auxiliary problem (Algorithm 3.1 step 1).  lambda is read from host memory.               */
int fmg_eig_aux_rhs(fmg_eig_handle* h, int32_t level, double lambda, const double* u_dev,
                    double* f_dev, void* stream);

/* x <- MG(V_{h_k}, f, x, m): m V-cycles in place (Algorithm 3.1 step 1).                    */
int fmg_eig_multigrid(fmg_eig_handle* h, int32_t level, const double* f_dev, double* x_dev,
                      void* stream);

/* One correction step EigenMG(V_H, lambda, u, V_{h_k}, m) (Algorithm 3.1) on level k >= 2:
 * reads (lambda_in, u_in), writes the new pair and, if u_tilde_dev is not NULL, the
 * auxiliary iterate u~.  *iters receives the nonlinear iteration count.  Synchronous.       */
int fmg_eig_correction(fmg_eig_handle* h, int32_t level, double lambda_in,
                       const double* u_in_dev, double* lambda_out, double* u_out_dev,
                       double* u_tilde_dev, int32_t* iters);

/* The small system of Algorithm 3.1 step 2 on level k >= 2 for a given u~ (u_tilde_dev, level
 * k interior layout): with the basis psi = (phi^H_1..phi^H_N, u~), N = interior nodes of
 * level 1, writes the n x n row-major host matrices (n = N + 1)
 *   K[i][j] = a^(psi_i, psi_j) + (W psi_i, psi_j),  M[i][j] = b(psi_i, psi_j),
 *   G[i][j] = int w^2 psi_i psi_j  with w = sum_j c_host[j] psi_j,
 * as the small nonlinear solve assembles them from one fine pass.  FMG_EINVAL if n != N + 1.
 * Synchronous.                                                                              */
int fmg_eig_augmented_system(fmg_eig_handle* h, int32_t level, const double* u_tilde_dev,
                             const double* c_host, int32_t n, double* K_host, double* M_host,
                             double* G_host);

/* Algorithm 3.2 step 1: the nonlinear eigenproblem directly on V_{h_1}.  Synchronous.       */
int fmg_eig_coarse_solve(fmg_eig_handle* h, double* lambda_out, double* u_dev,
                         int32_t* iters);

/* The same coarsest-level solve as fmg_eig_coarse_solve, for callers that must not allocate
 * device memory (the paper has no counterpart: this is a library service).  Examples are
 * frameworks that own every byte of the GPU through their own pool (an allocation from
 * outside can fail or fragment it) and services that may not allocate once they serve
 * (cudaMalloc / cudaFree can synchronise the device and stall the work in flight).  No
 * handle is needed and nothing is allocated: the caller passes the problem (only dim,
 * coarse_cells, box_len, w_const, w_quad, zeta, omega, scf_tol and scf_max_iter are read)
 * and u_dev, a device buffer of (coarse_cells - 1)^2 doubles that receives u_{h_1} in the
 * interior layout.  *lambda_out (host) receives lambda_{h_1}; iters (host, nullable) the
 * nonlinear iteration count.  All intermediates live in one fixed 256 KiB device array inside
 * the library, which every GPU that loads the library keeps until the process exits.
 * Limits: dim = 2, FMG_FP64, FMG_W_LEFT (else FMG_ENOTSUP); 2 <= coarse_cells <= 9 (else
 * FMG_EINVAL, the array's capacity).  The first call on a device looks up the array's device
 * address and keeps it for the process (a device reset invalidates it: do not call again on
 * a device after cudaDeviceReset).  The call copies small tables from host memory, runs on
 * `stream` (NULL = legacy default stream) and synchronises it before returning.  Calls share
 * the array; calls that overlap on the GPU, from several host threads or streams, race and
 * must be serialised by the caller.  Returns FMG_OK, FMG_ENOCONV (cap hit, partial result
 * written), FMG_ECUDA (a launch or copy failed, or the solve kernel never ran) or another
 * error code.                                                                                */
int fmg_eig_coarse_solve_noalloc(const fmg_eig_problem* prob, double* lambda_out, double* u_dev,
                                 int32_t* iters, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FMG_EIG_H */
