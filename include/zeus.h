/*
 * zeus.h -- C ABI of the GB300 (sm_103a) implementation of the Zeus method
 * (arXiv 2603.28770): a short particle-swarm phase seeds N start points, one
 * BFGS run per start takes forward-mode dual-number gradients (or a
 * reverse-mode adjoint), a backtracking Armijo line search and the dense
 * inverse-Hessian rank-two update, and a best-of-swarm reduction picks the
 * result.
 *
 * Conventions for every entry point:
 *  - Return value: ZEUS_OK (0) or a negative zeus_status code.  No entry
 *    point aborts, throws or prints; zeus_strerror() names a code.
 *  - "device" pointers are CUDA global-memory addresses on the current
 *    device, "host" pointers are ordinary CPU memory.  The caller owns every
 *    buffer it passes; the library keeps no pointer after a call returns.
 *  - Arrays of points are row-major [n][dim] (the paper's N x dim swarm
 *    layout, Alg. 7), contiguous, dim elements per row.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued on it and the call returns without
 *    waiting, except where a function says it synchronizes.
 *  - Entry points that take `workspace` allocate nothing: the caller
 *    provides `workspace_bytes` >= zeus_workspace_size() bytes of device
 *    memory, 256-byte aligned.  Its contents need no initialisation and are
 *    undefined afterwards.  Two calls in flight must not share a workspace.
 *  - Validation errors (ZEUS_EINVAL, ZEUS_EWORKSPACE, ZEUS_EUNSUPPORTED) are
 *    reported before any work is enqueued.
 *  - Host threads: every entry point may be called from several host
 *    threads at once, on one device or several, provided that no two calls
 *    in flight share a workspace, a zeus_context, a batch plan's device
 *    tables or an output buffer (one context per host thread for
 *    zeus_solve_host).  The library's process-wide state is small and
 *    guarded: the bounded-wait limit (an atomic, zeus_set_wait_limit), the
 *    two streams of the batched form on each device (created once, under
 *    a lock, by zeus_batch_prepare) and the scratch array of
 *    zeus_solve_from_noalloc (its enqueue is serialised under a lock, but
 *    overlapping calls share the array: see there).  Kernel attributes are
 *    set before each launch, with the same value every time.
 */
#ifndef ZEUS_H
#define ZEUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ZEUS_ABI_VERSION 2

typedef enum {
    ZEUS_OK = 0,
    ZEUS_EINVAL = -1,          /* an argument is out of range */
    ZEUS_ENOMEM = -2,          /* a handle could not allocate device memory */
    ZEUS_ECUDA = -3,           /* a CUDA call failed (launch, copy, ...) */
    ZEUS_ETIMEOUT = -4,        /* a bounded device-side wait expired */
    ZEUS_EUNSUPPORTED = -5,    /* combination of options not built */
    ZEUS_EWORKSPACE = -6       /* workspace missing, too small or misaligned */
} zeus_status;

/* Test functions of Section V-B.  QUADRATIC is a test objective
 * f = 0.5 * sum_i (i+1) x_i^2 (minimum 0 at x = 0). */
typedef enum {
    ZEUS_OBJ_ROSENBROCK = 0,       /* sum_{i<d-1} (1-x_i)^2 + 100 (x_{i+1}-x_i^2)^2, d >= 2 */
    ZEUS_OBJ_RASTRIGIN = 1,        /* 10 d + sum (x_i^2 - 10 cos(2 pi x_i)) */
    ZEUS_OBJ_ACKLEY = 2,           /* -20 e^{-0.2 sqrt(mean x^2)} - e^{mean cos 2 pi x} + 20 + e */
    ZEUS_OBJ_GOLDSTEIN_PRICE = 3,  /* d == 2 */
    ZEUS_OBJ_QUADRATIC = 100
} zeus_objective;

/* User-defined objectives (Section IV-A: f is written once for any scalar
 * type and differentiated on dual numbers).  Objective ZEUS_OBJ_USER + k,
 * 0 <= k < zeus_user_objective_count(), is the k-th objective of the
 * plug-in header compiled into the library (contract and limits in
 * include/zeus_user.cuh): forward-mode gradients only, and H held in shared
 * memory (a plan that would stream it, or L-BFGS, returns
 * ZEUS_EUNSUPPORTED). */
#define ZEUS_OBJ_USER 200
#define ZEUS_USER_MAX 4

typedef enum {
    ZEUS_FP64 = 0,           /* every step in FP64 (the paper's precision) */
    ZEUS_FP32_GUARDED = 1    /* objective, gradient and H in FP32; y^T s, rho,
                                the Armijo test and the final f in FP64 */
} zeus_precision;

typedef enum {
    ZEUS_GRAD_FORWARD = 0,   /* dim dual-number passes (Alg. 5) */
    ZEUS_GRAD_ADJOINT = 1    /* one reverse sweep (hand-written adjoint) */
} zeus_grad_mode;

/* Per-start termination status (Alg. 4 result.status, extended). */
typedef enum {
    ZEUS_RUN_MAX_ITER = 0,   /* iteration cap reached (the paper's status 0) */
    ZEUS_RUN_CONVERGED = 1,  /* ||g|| < grad_tol, or f <= target_f */
    ZEUS_RUN_STOPPED = 2,    /* the shared stop flag was raised (Alg. 10) */
    ZEUS_RUN_NONFINITE = 3,  /* f or g became NaN or infinite */
    ZEUS_RUN_STALLED = 4     /* ZEUS_FP32_GUARDED only: the last iteration lowered f by no
                                more than FP32 can resolve, f_k - f_{k+1} <=
                                2^-23 max(|f_k|, |f_{k+1}|) (the gradient tolerance is
                                out of reach at FP32 resolution) */
} zeus_run_status;

/*
 * Arguments of the parallel Zeus procedure (Alg. 7:
 * Zeus(f, N, range, iter_bfgs, iter_pso, iter_ls, required_c, Theta, w, c1, c2)).
 * zeus_default_problem() fills the 2-D Rosenbrock workload.
 */
typedef struct {
    int32_t objective;          /* zeus_objective */
    int32_t dim;                /* d >= 1 (Rosenbrock >= 2, Goldstein-Price == 2), d <= 4096 */
    double lower, upper;        /* sampling box of Alg. 2, lower < upper (not enforced later) */
    int64_t n_starts;           /* N = particles = BFGS runs, 1 <= N <= 2^31 - 1 */
    int32_t pso_iters;          /* T >= 0 PSO updates (Alg. 3) */
    int32_t bfgs_max_iters;     /* K >= 0 (iter_bfgs) */
    int32_t ls_max_iters;       /* L >= 1 line-search trials (iter_ls, paper: 20) */
    int32_t required_converged; /* required_c of Alg. 10; 0 = off */
    double grad_tol;            /* Theta: converged when ||g||_2 < Theta */
    double w, c1, c2;           /* PSO inertia, cognitive, social (Section III-A) */
    double armijo_c;            /* Armijo constant c in (0,1) (Section III-D) */
    double backtrack;           /* step factor beta in (0,1) (paper: 0.5) */
    double target_f;            /* NaN = off; else a start with f <= target_f
                                   counts as converged and raises the stop flag */
    uint64_t seed;              /* Philox4x64-10 key word 0 */
    int32_t precision;          /* zeus_precision */
    int32_t grad_mode;          /* zeus_grad_mode */
    int32_t start_from_pbest;   /* 0: BFGS from current positions (Alg. 10), 1: from personal bests */
    int32_t threads_per_start;  /* 0 = automatic: one lane per start for small d, with the
                                   long-running starts handed to one 128-thread block
                                   each; H streamed from HBM when it does not fit on
                                   chip; 1 = one lane per start throughout;
                                   32 = one warp per start, four starts to a 128-thread
                                   block, H in shared memory;
                                   128 = one 128-thread block per start throughout;
                                   256 = one 256-thread block per start, H streamed */
    int32_t lbfgs_m;            /* 0 = the dense inverse-Hessian update of Alg. 4; m in 1..64 =
                                   L-BFGS (the paper's future work, Section VI): the m most
                                   recent pairs and the two-loop recursion, one 256-thread
                                   block per start, no H (threads_per_start 0 or 256;
                                   not for Goldstein-Price; not batched) */
    int32_t pad;
} zeus_problem;

/* Summary written on the device by zeus_solve / zeus_solve_from. */
typedef struct {
    double best_f;          /* min over starts of the final f (NaN counts as +inf) */
    int64_t best_index;     /* its start index, ties to the lowest index */
    int64_t n_converged;    /* starts with status ZEUS_RUN_CONVERGED */
    int64_t total_iters;    /* sum over starts of completed BFGS iterations */
    int64_t total_feval;    /* sum over starts of line-search objective evaluations */
    double gbest_f;         /* PSO global best value after the last update (zeus_solve) */
    int64_t gbest_index;    /* its particle index */
    int32_t error;          /* device-side error word, 0 = none */
    int32_t stop_flag;      /* 1 if the stop flag was raised */
    int64_t h_reads;        /* streamed H (zeus_plan_info().stream): passes over a start's
                               H that read it from device memory, summed over starts; the
                               pass is skipped while H = I, 0 for on-chip H */
    int64_t h_writes;       /* ... passes that wrote it back (an update was applied) */
} zeus_result;

/* Name of a zeus_status code (static string, never NULL). */
const char *zeus_strerror(int code);

/* ZEUS_ABI_VERSION of the built library. */
int zeus_abi_version(void);

/* Limit of the bounded device-side waits: the servers of the fused BFGS
 * launch poll the hand-over queue and the clustering kernel's blocks poll a
 * grid barrier (both the library's own; the paper's design has no such
 * waits).  Each poll sleeps about 256 ns; a wait that has not ended after
 * `polls` polls gives up: the kernel sets its error word
 * (zeus_result.error or zeus_cluster_result.error = 1), the outputs of the
 * starts it had not finished are undefined, and it returns, so the context
 * stays usable and the next call runs normally.  polls = 0 restores the
 * default, 2^23 polls (about two seconds).  The setting is process-wide
 * and is read when a call enqueues its kernels; thread-safe.  Meant for
 * tests of the error paths: a small limit makes correct runs report an
 * error.  Always ZEUS_OK. */
int zeus_set_wait_limit(uint32_t polls);

/* Fill *p with the defaults: 2-D Rosenbrock on [-5,5]^2, N = 128, T = 5,
 * w = 0.7, c1 = c2 = 1.5, K = 100, L = 20, c = 1e-4, beta = 0.5,
 * Theta = 1e-8, FP64, forward mode, seed 0.  Returns ZEUS_EINVAL if p is NULL. */
int zeus_default_problem(zeus_problem *p);

/* Check every field of *p; ZEUS_OK, ZEUS_EINVAL or ZEUS_EUNSUPPORTED. */
int zeus_validate(const zeus_problem *p);

/* Which kernels zeus_solve / zeus_solve_from run for problem *p. */
typedef struct {
    int32_t narrow;          /* 1: one lane per start (the bulk) */
    int32_t handover;        /* 1: long runs handed to one block per start */
    int32_t block;           /* 1: one 128-thread block per start, H in shared memory */
    int32_t stream;          /* 1: one 256-thread block per start, H streamed from HBM */
    int32_t blocks;          /* grid of the block-per-start / streaming kernel */
    int32_t lbfgs;           /* 1: L-BFGS (problem.lbfgs_m > 0), block per start, no H */
    int32_t warp;            /* 1: one warp per start, H in shared memory */
    int64_t h_bytes;         /* bytes of H per start in the chosen precision: d^2
                                elements; streamed FP32 H is held as the 32-column tiles
                                of its upper triangle, and h_bytes is then their size
                                (what one pass reads and writes) */
} zeus_plan;
int zeus_plan_info(const zeus_problem *p, zeus_plan *plan);

/* Device workspace needed by zeus_solve / zeus_solve_from / zeus_pso /
 * zeus_argmin for problem *p (host pointer), in bytes. */
int zeus_workspace_size(const zeus_problem *p, size_t *bytes);

/*
 * The whole method, Alg. 7: PSO initialisation (Alg. 2/8) and p->pso_iters
 * synchronous PSO updates (Alg. 3/9), one BFGS run per particle (Alg. 4/10)
 * started from its current position (or personal best), and the
 * best-of-swarm reduction.
 *   x_out      device double [N][dim]  final BFGS points (required)
 *   f_out      device double [N]       final f (may be NULL)
 *   gnorm_out  device double [N]       final ||g|| (may be NULL)
 *   status_out device int32  [N]       zeus_run_status (may be NULL)
 *   iters_out  device int32  [N]       completed iterations (may be NULL)
 *   result     device zeus_result      summary (may be NULL)
 * With required_converged = 0 and target_f = NaN the outputs depend only
 * on *p (bitwise reproducible run to run).
 */
int zeus_solve(const zeus_problem *p, void *workspace, size_t workspace_bytes,
               double *x_out, double *f_out, double *gnorm_out,
               int32_t *status_out, int32_t *iters_out, zeus_result *result,
               void *stream);

/* BFGS from caller-given starts (Alg. 10 without the PSO phase), then the
 * best-of-swarm reduction.  x0: device double [N][dim], may equal x_out.
 * Other arguments as zeus_solve; result->gbest_* are set to NaN / -1. */
int zeus_solve_from(const zeus_problem *p, const double *x0,
                    void *workspace, size_t workspace_bytes,
                    double *x_out, double *f_out, double *gnorm_out,
                    int32_t *status_out, int32_t *iters_out,
                    zeus_result *result, void *stream);

/* The PSO phase alone (Alg. 2 then Alg. 3 T times, synchronous global best).
 * All outputs device, required: x_out, v_out, px_out [N][dim] (positions,
 * velocities, personal-best positions), pf_out [N] (personal-best values),
 * gx_out [dim] (global-best position); result->gbest_f / gbest_index are
 * written if result is not NULL. */
int zeus_pso(const zeus_problem *p, void *workspace, size_t workspace_bytes,
             double *x_out, double *v_out, double *px_out, double *pf_out,
             double *gx_out, zeus_result *result, void *stream);

/* Objective values and gradients at n points (Section V-B objectives).
 *   x: device double [n][dim]; f_out: device double [n] (may be NULL);
 *   g_out: device double [n][dim] (may be NULL).
 *   grad_mode: ZEUS_GRAD_FORWARD (Alg. 5, dim dual passes) or
 *   ZEUS_GRAD_ADJOINT (reverse sweep).  FP64 throughout. */
int zeus_objective_eval(int32_t objective, int32_t dim, int64_t n,
                        const double *x, double *f_out, double *g_out,
                        int32_t grad_mode, void *stream);

/* The same in FP32 (x, f_out, g_out are float arrays). */
int zeus_objective_eval_f32(int32_t objective, int32_t dim, int64_t n,
                            const float *x, float *f_out, float *g_out,
                            int32_t grad_mode, void *stream);

/* Number of user objectives compiled into the library (0..ZEUS_USER_MAX).
 * Host only. */
int32_t zeus_user_objective_count(void);

/* Name and dimension range of user objective k (objective id
 * ZEUS_OBJ_USER + k).  name: host buffer of name_len bytes, written
 * NUL-terminated (truncated to fit; may be NULL); min_dim, max_dim: host
 * int32 (may be NULL; max_dim 0 = no limit beyond the library's).  Host
 * only.  ZEUS_EINVAL if k is out of range. */
int zeus_user_objective_info(int32_t k, char *name, int32_t name_len,
                             int32_t *min_dim, int32_t *max_dim);

/* Best-of-swarm reduction (Alg. 7 ParallelReduction): writes
 * result->best_f / best_index for device f[n] (NaN as +inf, ties to the
 * lowest index); the other result fields are zeroed.  Needs
 * zeus_argmin_workspace_size(n) bytes of workspace. */
int zeus_argmin(const double *f, int64_t n, void *workspace,
                size_t workspace_bytes, zeus_result *result, void *stream);
int zeus_argmin_workspace_size(int64_t n, size_t *bytes);

/* The uniform draws of the PSO phase (Philox4x64-10 per Section IV-A as
 * read here): out[i*dim + j] = draw (phase, particle i, dimension j) for
 * i < n, j < dim; device double [n][dim]. */
int zeus_uniform(uint64_t seed, uint64_t problem, uint64_t phase,
                 int64_t n, int32_t dim, double *out, void *stream);

/* The FP64 elementary functions the objectives use, for validation:
 *   fn 0: y0 = sin(2 pi x), y1 = cos(2 pi x)  (the library's own method)
 *   fn 1: y0 = e^x                             (the library's own method)
 *   fn 2: y0, y1 = CUDA sincospi(2x)           (CUDA math library)
 *   fn 3: y0 = CUDA exp(x)                     (CUDA math library)
 *   fn 4: y0 = cos(2 pi x) by the cosine-only evaluation the objectives
 *         use (bit for bit the y1 of fn 0)
 * x, y0: device double [n]; y1: device double [n] for fn 0 and 2, else
 * ignored (may be NULL). */
int zeus_math_eval(int32_t fn, int64_t n, const double *x, double *y0, double *y1,
                   void *stream);

/* ---- Batched form (the paper solves one problem per call) ----
 *
 * Many independent problems (any mix of objective, dim, N, T, K, seed)
 * solved by one fixed set of kernels: PSO updates of every problem in one
 * launch per update, BFGS of every start from a device work list
 * (persistent blocks; one launch per class of items that share a layout
 * and an occupancy), the hand-over launch, and one best-of-swarm reduction
 * per problem.  The lane-tile classes and the hand-over launch run on a
 * stream of the library's own, concurrently with the other classes, which
 * alternate between `stream` and a second stream of the library's own
 * (both forked from and joined back to `stream`, so the call stays
 * stream-ordered and graph-capturable).  Problem P's results equal those
 * of zeus_solve(&probs[P]) bit for bit.
 *
 * Every problem of a batch shares `precision` and `grad_mode`; problems
 * whose dense H must stream from HBM (zeus_plan_info().stream) are not
 * batched (ZEUS_EUNSUPPORTED); L-BFGS problems (lbfgs_m > 0) are, one
 * 256-thread block per start in classes of their own, beside dense ones.
 * A problem's n_starts must be below 2^30.
 *
 * Outputs are the problems' arrays concatenated in problem order:
 *   x_out      device double [sum_P N_P * dim_P]   final BFGS points (required)
 *   f_out      device double [sum_P N_P]           final f (required)
 *   gnorm_out  device double [sum_P N_P]           (may be NULL)
 *   status_out device int32  [sum_P N_P]           (may be NULL)
 *   iters_out  device int32  [sum_P N_P]           (may be NULL)
 *   results    device zeus_result [n_problems]     (may be NULL)
 * Problem P's rows start at the prefix sums of N_Q * dim_Q and N_Q, Q < P.
 */
#define ZEUS_BATCH_MAX_CLASSES 32

typedef struct {
    int32_t n_problems;
    int32_t pso_blocks;       /* blocks of each batched PSO launch */
    int32_t items;            /* BFGS work-list entries (lane tiles + block starts) */
    int32_t pso_iters_max;    /* PSO launches = pso_iters_max + 1 */
    int32_t q_cap;            /* hand-over queue entries */
    int32_t d_max_handover;   /* largest dim that can be handed over */
    int32_t precision, grad_mode;
    int32_t n_classes;        /* BFGS launches over the work list */
    int32_t handover_smem;    /* dynamic shared memory of the hand-over launch */
    int32_t n_user;           /* problems with a user objective (their kernels
                                 are compiled apart from the built-in ones) */
    int32_t pad;              /* 0 */
    int32_t class_first[ZEUS_BATCH_MAX_CLASSES];  /* work-list range and dynamic */
    int32_t class_count[ZEUS_BATCH_MAX_CLASSES];  /* shared memory of each BFGS */
    int32_t class_smem[ZEUS_BATCH_MAX_CLASSES];   /* launch */
    int32_t class_kind[ZEUS_BATCH_MAX_CLASSES];   /* 0: lane tiles, 1: one block per start,
                                                     2: one warp per start, 3: L-BFGS, one
                                                     256-thread block per start */
    int64_t total_starts;     /* sum_P N_P */
    int64_t total_coords;     /* sum_P N_P * dim_P */
    int64_t total_g;          /* sum_P dim_P */
    uint64_t workspace_bytes; /* device workspace the batch needs */
    uint64_t table_bytes;     /* bytes zeus_batch_prepare copies to the device */
} zeus_batch_plan;

/* Plans a batch (host only, no CUDA call).  probs: host array [n]. */
int zeus_batch_plan_make(const zeus_problem *probs, int32_t n, zeus_batch_plan *plan);

/* Writes the batch's tables (problem parameters, offsets, work list) into
 * the workspace: one host-to-device copy on `stream`, then synchronizes
 * `stream`.  On its first call on a device it also creates the library's
 * two streams and three events for that device (kept until exit), so call
 * it before any stream capture of zeus_batch_solve.  probs and plan must
 * be those given to zeus_batch_plan_make;
 * workspace: device, plan->workspace_bytes, 256-byte aligned.  The tables
 * stay valid for any number of zeus_batch_solve calls on this workspace. */
int zeus_batch_prepare(const zeus_problem *probs, int32_t n, const zeus_batch_plan *plan,
                       void *workspace, size_t workspace_bytes, void *stream);

/* Runs the prepared batch.  Enqueues kernels and one memset only (no copy,
 * no synchronization, no allocation), so a call can be recorded in a CUDA
 * graph and replayed; every replay recomputes the results from the tables. */
int zeus_batch_solve(const zeus_batch_plan *plan, void *workspace, size_t workspace_bytes,
                     double *x_out, double *f_out, double *gnorm_out, int32_t *status_out,
                     int32_t *iters_out, zeus_result *results, void *stream);

/* ---- No-allocation variant (the paper has no counterpart) ----
 *
 * zeus_solve_from without a workspace argument, for callers that cannot
 * call cudaMalloc: code that must stay inside a framework's own caching
 * allocator, plugins and embedded callers that are handed device buffers
 * but no allocation rights, and code that must not pay the device-wide
 * synchronisation that cudaMalloc and cudaFree can imply.  The library
 * allocates nothing in this call either: its scratch (control block,
 * reduction partials, hand-over queue) is one static device array of
 * ZEUS_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.
 *   - Limit: when the automatic mode runs one lane per start and hands
 *     long runs to the block-per-start kernel (dim <= 16 with
 *     threads_per_start 0), the hand-over queue holds as many entries as
 *     zeus_solve_from's would, at most as many as fit the array at
 *     16 + 8 * dim * dim bytes each (about 20000 at dim 10); a start that
 *     finds the queue full finishes in its lane, with the same result.
 *     The lane tiles and the queue's service run in one cooperative launch,
 *     as in zeus_solve_from.
 *   - Problems whose H must stream from HBM (zeus_plan_info().stream with
 *     lbfgs_m = 0) need more than the array and get ZEUS_EWORKSPACE;
 *     L-BFGS problems (no H) run.  Otherwise zeus_validate's limits apply.
 *   - f_out is required (device double [N]); the other arguments are those
 *     of zeus_solve_from.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture begins.  The address is kept for the life
 *     of the process: do not call this entry point on a device again after
 *     cudaDeviceReset (or anything else that destroys its primary context).
 *   - All calls share the one array and it keeps the previous call's
 *     contents (the call clears what must start at zero): calls that
 *     overlap on the GPU, on any streams, race and give undefined results.
 */
#define ZEUS_NOALLOC_SCRATCH_BYTES (16u << 20)

int zeus_solve_from_noalloc(const zeus_problem *p, const double *x0, double *x_out,
                            double *f_out, double *gnorm_out, int32_t *status_out,
                            int32_t *iters_out, zeus_result *result, void *stream);

/* ---- Host-buffer interface (owns device buffers; for callers without
 * CUDA memory of their own) ---- */
typedef struct zeus_context zeus_context;

/* Create a context on the current device.  *ctx receives the handle. */
int zeus_context_create(zeus_context **ctx);
/* Free the context and its device buffers (synchronizes the device). */
int zeus_context_destroy(zeus_context *ctx);

/* zeus_solve with HOST outputs: runs on `stream`, copies the outputs to
 * the host buffers (any of which may be NULL except x_out) and synchronizes
 * `stream` before returning.  Returns ZEUS_ETIMEOUT (outputs incomplete)
 * when the run's device error word is set (a bounded wait gave up).  Grows the context's device buffers on demand
 * (ZEUS_ENOMEM if that fails).  x_out: host double [N][dim]; f_out,
 * gnorm_out: host double [N]; status_out, iters_out: host int32 [N];
 * result: host zeus_result. */
int zeus_solve_host(zeus_context *ctx, const zeus_problem *p, double *x_out,
                    double *f_out, double *gnorm_out, int32_t *status_out,
                    int32_t *iters_out, zeus_result *result, void *stream);

/* ---- Solution clustering (Section VI names it as future work: cluster
 * the candidate solutions of the multistart by function value or by
 * coordinates, and take confidence in the region of the lowest f from the
 * number of starts that reached it) ----
 *
 * Candidates: starts whose f is finite (and, with only_converged, whose
 * status is ZEUS_RUN_CONVERGED).  Leader clustering in the order of
 * increasing (f, start index): each candidate joins the first existing
 * leader it is within tol of, else it becomes the next leader.  Cluster k
 * is the k-th leader's; cluster 0 holds the start of the lowest f.  "Within
 * tol" of leader L:
 *   ZEUS_CLUSTER_BY_F  |f_i - f_L| <= tol * max(1, |f_L|)
 *   ZEUS_CLUSTER_BY_X  sum_j (x_ij - x_Lj)^2 <= tol^2, the sum formed in
 *                      index order, one rounding per term (fused
 *                      multiply-add), in FP64
 * Only the first max_clusters clusters are formed; the candidates left then
 * are reported as unclustered. */
#define ZEUS_CLUSTER_BY_F 0
#define ZEUS_CLUSTER_BY_X 1
#define ZEUS_CLUSTER_MAX 4096     /* largest max_clusters */
#define ZEUS_LABEL_NONE (-1)      /* not a candidate */
#define ZEUS_LABEL_LEFT (-2)      /* candidate left after max_clusters clusters */

typedef struct {
    int32_t method;           /* ZEUS_CLUSTER_BY_F or ZEUS_CLUSTER_BY_X */
    int32_t max_clusters;     /* 1 .. ZEUS_CLUSTER_MAX */
    int32_t only_converged;   /* 0 or 1 (needs status) */
    int32_t pad;              /* 0 */
    double tol;               /* >= 0, finite */
} zeus_cluster_params;

typedef struct {
    int64_t n_candidates;
    int64_t n_clusters;       /* clusters formed */
    int64_t n_left;           /* candidates in no cluster (max_clusters reached) */
    int64_t best_count;       /* members of cluster 0, the region of the lowest f */
    int64_t best_leader;      /* start index of its leader (lowest f); -1 if none */
    double best_f;            /* f of that leader (NaN if none) */
    double best_spread;       /* largest distance (BY_X: sqrt of the sum above) or
                                 |f_i - f_L| (BY_F) of a member of cluster 0 */
    int32_t error;            /* 0 */
    int32_t pad;
} zeus_cluster_result;

/* Device workspace of zeus_cluster for this max_clusters (host only). */
int zeus_cluster_workspace_size(int32_t max_clusters, size_t *bytes);

/* Clusters the n final points of one problem (zeus_solve outputs).
 *   x: device double [n][dim]; f: device double [n]; status: device int32
 *   [n] (may be NULL unless only_converged); label_out: device int32 [n]
 *   (cluster id, ZEUS_LABEL_NONE or ZEUS_LABEL_LEFT); leader_out, count_out:
 *   device int32 [max_clusters] (leader start index and member count of
 *   each cluster formed, -1 / 0 past n_clusters; may be NULL); result:
 *   device zeus_cluster_result (may be NULL); workspace: device,
 *   zeus_cluster_workspace_size bytes, 256-byte aligned, not shared with a
 *   call in flight.
 * One memset and one cooperative launch on `stream` (graph-capturable);
 * n < 2^31.  ZEUS_EINVAL for bad parameters or pointers and
 * ZEUS_EWORKSPACE for a missing or small workspace, before any launch.  A
 * grid barrier that does not complete within about two seconds ends the
 * kernel with result->error = 1. */
int zeus_cluster(const zeus_cluster_params *cp, int64_t n, int32_t dim, const double *x,
                 const double *f, const int32_t *status, int32_t *label_out,
                 int32_t *leader_out, int32_t *count_out, zeus_cluster_result *result,
                 void *workspace, size_t workspace_bytes, void *stream);

/* Clusters the final points of every problem of a batch, each on its own
 * (the definition of zeus_cluster), one block per problem; needs no memory
 * beyond the batch's workspace.  plan, workspace: those of the
 * zeus_batch_solve that wrote x_out, f_out and status_out (status_out may
 * be NULL unless only_converged).  label_out: device int32 [total_starts],
 * in the order of f_out; leader_out, count_out: device int32
 * [n_problems][max_clusters] (may be NULL; leaders are start indices within
 * their problem); results: device zeus_cluster_result [n_problems] (may be
 * NULL).  ZEUS_EINVAL / ZEUS_EWORKSPACE before any launch. */
int zeus_batch_cluster(const zeus_batch_plan *plan, const void *workspace,
                       size_t workspace_bytes, const zeus_cluster_params *cp,
                       const double *x_out, const double *f_out, const int32_t *status_out,
                       int32_t *label_out, int32_t *leader_out, int32_t *count_out,
                       zeus_cluster_result *results, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ZEUS_H */
