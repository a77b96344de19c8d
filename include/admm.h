/*
 * admm.h -- C ABI of the GB300 (sm_103a) parallel ADMM solver for robust
 * quadratic resource allocation (Qureshi, East, Cannon, "Parallel ADMM for
 * robust quadratic optimal resource allocation problems").
 *
 * The problem is eq. (2) of Sec. II:
 *
 *   min_{x_1^(i), x_k^(i,j) in [lo_k^(i), hi_k^(i)]}  (1/q) sum_{j,i,k} f_k^(i,j)(x_k^(i,j))
 *   s.t.  sum_i x_k^(i,j) >= y_k^(j)              (demand, every k, j)
 *         sum_k g_k^(i,j)(x_k^(i,j)) <= c^(i)      (capacity, every i, j)
 *         x_1^(i,j) = x_1^(i)                      (shared first move)
 *
 * with quadratic f and g (Assumption 3):
 *   f_k^(i,j)(x) = f2 x^2 + f1 x + f0,  g_k^(i,j)(x) = g2 x^2 + g1 x + g0.
 * q = 1 is the nominal problem (1).  It is solved by the ADMM iteration
 * (a)-(i) of App. A, whose step (a) minimises one quartic per element with
 * Algorithm 1 (Sec. III-B), until the residuals r and sigma of App. A fall
 * below r_tol and s_tol (Alg. 2 step 3), checked every `check_every`
 * iterations (Sec. IV-B).
 *
 * Array layout (all row-major, k fastest; indices 0-based, so the paper's
 * k = 1 is k = 0 here):
 *   element arrays  f2 f1 f0 g2 g1 g0 x      [m][q][n]   index (i*q + j)*n + k
 *   bound arrays    x_lo x_hi                [m][n]      index i*n + k
 *   column arrays   y s mu                   [q][n]      index j*n + k
 *   pair arrays     lam zeta h p nu          [m][q]      index i*q + j
 *   source arrays   c x1                     [m]
 *
 * Errors: every call returns an admm_status; admm_last_error() gives a
 * thread-local message for the last failing call on the calling thread.
 * No call aborts the process.  Device waits inside the kernels are bounded:
 * a wait that runs out returns ADMM_ETIMEOUT instead of hanging.
 */
#ifndef ADMM_H
#define ADMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum admm_status {
    ADMM_OK = 0,
    ADMM_EINVAL = 1,         /* bad argument or problem data (see admm_create) */
    ADMM_ENOMEM = 2,         /* a device or pinned-host allocation failed */
    ADMM_ECUDA = 3,          /* a CUDA runtime call failed */
    ADMM_ETIMEOUT = 4,       /* a bounded device-side wait gave up */
    ADMM_ENOTCONVERGED = 5,  /* max_iter reached; the result is still filled */
    ADMM_EUNSUPPORTED = 6,   /* sizes beyond the compiled limits (ADMM_MAX_M, ...) */
    ADMM_EPENDING = 7,       /* a served request has not finished yet */
    ADMM_ECANCELLED = 8,     /* a served request was cancelled (admm_server_cancel) */
    ADMM_EBOUNDS = 9         /* bounds-checked build only: an element access of the mixed
                                element update fell outside its instance's arrays (it was
                                redirected inside them; the results are not valid) */
} admm_status;

/* Arithmetic of the per-element work (the stored state follows it). */
enum {
    ADMM_FP64 = 0,          /* everything in FP64 */
    ADMM_MIXED = 1,         /* FP32 storage and element work; FP64 k-sums, pair
                               scalars and residuals; the cubic's branch is
                               decided in FP64 whenever FP32 cannot certify it.
                               Mixed solves (this and the next) stop at
                               r < r_tol and sigma < 0.85 s_tol: the margin
                               on sigma, the binding residual, absorbs the
                               FP32 rounding of the stored x in the KKT
                               conditions of eq. (2) */
    ADMM_MIXED_FP64CUBIC = 2 /* as ADMM_MIXED, but the whole cubic step
                               (b, c, d, Q, R, Delta, roots, delta-f) in FP64 */
};
/* x-update of step (a) */
enum {
    ADMM_XMIN_EXACT = 0,    /* constrained minimiser: both local minima clamped, better kept */
    ADMM_XMIN_PAPER = 1     /* Pi(global unconstrained minimiser), as printed */
};
/* order of the sources in step (a) */
enum { ADMM_GAUSS_SEIDEL = 0, ADMM_JACOBI = 1 };

#define ADMM_MAX_M 8          /* sources per instance */
#define ADMM_MAX_PAIRS 1024   /* m*q per single instance */
#define ADMM_BATCH_MAX_PAIRS 256 /* m*q per instance of a batch or server */

typedef struct admm_problem {
    int32_t n, m, q;                 /* steps, sources, scenarios; all >= 1 */
    const double *f2, *f1, *f0;      /* alpha_{k,2..0}^(i,j)  [m][q][n]; f2 >= 0 */
    const double *g2, *g1, *g0;      /* beta_{k,2..0}^(i,j)   [m][q][n]; g2 >= 0 */
    const double *x_lo, *x_hi;       /* [m][n]; x_lo <= x_hi, finite */
    const double *y;                 /* [q][n] */
    const double *c;                 /* [m]; +INFINITY = no capacity limit */
    int32_t on_device;               /* 1: device pointers; 0: host pointers */
    int32_t coef_shared;             /* 1: f2..g0 are [m][n], the same maps for every scenario j
                                        (single-instance, batched and served solves; admm_solve_noalloc
                                        takes 0) */
} admm_problem;

typedef struct admm_params {
    double rho[4];                   /* rho_1..rho_4 > 0 (App. A) */
    double r_tol, s_tol;             /* stop when r < r_tol and sigma < s_tol */
    double tau;                      /* penalty factor of the adaptation (Sec. IV-A) */
    int32_t max_iter;                /* >= 1 */
    int32_t check_every;             /* >= 1; residuals at t % check_every == 0 and t == max_iter */
    int32_t precision;               /* ADMM_FP64 | ADMM_MIXED | ADMM_MIXED_FP64CUBIC */
    int32_t xmin_mode;               /* ADMM_XMIN_EXACT | ADMM_XMIN_PAPER */
    int32_t sweep;                   /* ADMM_GAUSS_SEIDEL | ADMM_JACOBI */
    int32_t adapt_rho;               /* 1: rho_i <- tau rho_i or rho_i / tau by r/sigma (Sec. IV-A) */
    int32_t rho2_over_n;             /* 1: each instance uses rho_2 = rho[1] / n (the capacity
                                        penalty acts on a sum of n terms) */
    int32_t adapt_start;             /* >= 0; with adapt_rho, the adaptation applies at the check
                                        iterations t >= adapt_start of a solve (0: from the first,
                                        as Sec. IV-A).  A warm-started re-solve starts close to its
                                        solution, and adapting only the ones still running after,
                                        say, 500 iterations keeps the warm start intact for the rest */
    int32_t reserved[2];             /* must be 0 */
} admm_params;

/* The solver state (the checkpoint).  z is not stored: after every
 * iteration z_k^(i,j) = g_k^(i,j)(x_k^(i,j)) + zeta^(i,j) and lambda is
 * constant over k (steps (b) and (g)), so (x, zeta, lam) determine z and
 * lambda.  cold = 1 marks the zero start of the paper's iteration, where
 * z = 0 instead. */
typedef struct admm_state {
    double *x;                       /* [m][q][n] */
    double *s, *mu;                  /* [q][n] */
    double *lam, *zeta, *h, *p, *nu; /* [m][q] */
    double *x1;                      /* [m] */
    double rho[4];                   /* penalties in force (they change with adapt_rho) */
    int32_t cold;
    int32_t on_device;               /* 1: the array pointers are device memory */
} admm_state;

typedef struct admm_result {
    double *x;                       /* out [m][q][n] or NULL */
    double *x1;                      /* out [m] or NULL */
    int32_t on_device;               /* 1: x, x1 are device pointers */
    int32_t iters;                   /* iterations run */
    int32_t converged;               /* 1 if the stop test passed */
    int32_t status;                  /* admm_status of the solve */
    double objective;                /* (1/q) sum f(x), eq. (2) */
    double r, sigma;                 /* residuals at the last check */
} admm_result;

typedef struct admm_handle admm_handle;

/* Defaults: rho = 1, r_tol = s_tol = 1e-6, max_iter = 5000,
 * check_every = 10 (Sec. IV-B), FP64, exact x-update, Gauss-Seidel,
 * no adaptation, tau = 1.1 (Sec. IV-A). */
void admm_default_params(admm_params *out);

/* Validates the problem (Assumptions 1 and 3: f2, g2 >= 0; finite data;
 * x_lo <= x_hi; c not NaN; sum_k min_{[lo,hi]} g > c is a sure
 * infeasibility), copies it into device memory owned by the handle in the
 * layout the kernels use, and sets the zero start.  The caller keeps its
 * buffers.  Returns ADMM_EINVAL, ADMM_EUNSUPPORTED (m > ADMM_MAX_M or
 * m*q > ADMM_MAX_PAIRS), ADMM_ENOMEM or ADMM_ECUDA on failure, with *out
 * set to NULL.  Runs on the current CUDA device and synchronises it. */
admm_status admm_create(const admm_problem *prob, const admm_params *params, admm_handle **out);

/* Replaces the settings used by later solves (same validation). */
admm_status admm_set_params(admm_handle *h, const admm_params *params);

/* Queues a solve from `warm` (NULL: continue from the handle's current
 * state; a fresh handle holds the zero start) until the stop test or
 * max_iter, with the whole loop on the device (one persistent launch), on
 * `stream` (a cudaStream_t; NULL = legacy default stream), and returns once
 * the work is queued: ADMM_OK, or ADMM_EINVAL / ADMM_ECUDA if it could not
 * be queued.  The solve's own outcome arrives later: `out` (may be NULL) is
 * filled by a host function queued behind the solve, so its fields,
 * out->status included (ADMM_OK, ADMM_ENOTCONVERGED with the result still
 * filled, ADMM_ETIMEOUT), are valid once the stream has been synchronised;
 * `out` and its x, x1 buffers must stay valid until then.  admm_wait waits
 * for the handle's last queued solve and returns that status.  The final
 * state stays in the handle.  A warm state is loaded before the call
 * returns (the call waits for that copy); with pageable host buffers for
 * out->x or out->x1 the call returns only after their copies.  One solve per
 * handle may be in flight at a time; solves of different handles on
 * different streams may overlap on the device. */
admm_status admm_solve(admm_handle *h, const admm_state *warm, admm_result *out, void *stream);

/* Waits until the handle's last queued solve has finished and returns its
 * status (ADMM_OK, ADMM_ENOTCONVERGED, ADMM_ETIMEOUT), filling `out` (may be
 * NULL) as admm_solve does. */
admm_status admm_wait(admm_handle *h, admm_result *out);

/* Resets the handle's state to the zero start. */
admm_status admm_reset(admm_handle *h);

/* Copies the handle's current state into `out` (host or device buffers as
 * out->on_device says; NULL array pointers are skipped).  Synchronous. */
admm_status admm_get_state(admm_handle *h, admm_state *out, void *stream);

/* Copies the per-solve record of the last admm_solve on this handle (valid
 * after admm_wait or a sync of its stream) into info_out[0 .. count-1]
 * (count <= 16): 0 iterations, 1 converged, 2 r,
 * 3 sigma, 4..7 the four terms of r, 8..10 the three terms of sigma,
 * 11 objective, 12 status, 13 cubic branch decisions that FP32 could not
 * certify and FP64 took (ADMM_MIXED).  Host-only; no device work. */
admm_status admm_get_info(admm_handle *h, double *info_out, int count);

/* Frees everything the handle owns.  NULL-safe. */
admm_status admm_destroy(admm_handle *h);

/* Diagnostics: launches a grid barrier (the one the solve kernels use)
 * that waits for one more arrival than the grid has, with a wait bound of
 * spin_ns (0 < spin_ns <= 5e9) over `grid` CTAs (1..64).  The wait must run
 * out and record ADMM_ETIMEOUT, which is returned in *status_out; the
 * device stays usable.  No counterpart in the paper: it tests the failure
 * path of the bounded device waits without faulting the GPU. */
admm_status admm_selftest_barrier_timeout(long long spin_ns, int grid, int *status_out);

/* Diagnostics of the bounds-checked build (libadmm_debug.so, compiled with
 * -DADMM_DEBUG_BOUNDS; see ADMM_EBOUNDS): checks an element index that lies
 * past a 16-element device buffer with the same check the element update
 * uses; the check must record it (without any access outside the buffer).
 * *status_out receives ADMM_EBOUNDS and *index_out the recorded index (20).
 * A release build returns ADMM_EUNSUPPORTED.  No counterpart in the paper:
 * it tests the failure path of the checked build without a fault. */
admm_status admm_selftest_bounds(int *status_out, long long *index_out);

/* Quartic benchmark of Sec. III-C: Algorithm 1 (Sec. III-B) plus the clamp
 * of step (a) on `count` independent quartics.  x[t] minimises
 *   A[t] x^4 + B[t] x^3 + C[t] x^2 + D[t] x   over [lo[t], hi[t]]
 * (xmin_mode as in admm_params: the constrained minimiser, or the literal
 * Pi(argmin)).  Arrays are [count], host memory (on_device = 0: copied to
 * and from the device inside the call, the paper's timing with copies) or
 * device memory (on_device = 1, checked: other pointers give ADMM_EINVAL);
 * the caller owns them.  admm_quartic_min
 * uses the solver's FP64 minimiser; admm_quartic_min_f32 the mixed
 * solver's FP32 one (device arrays 8-byte aligned).  Runs on `stream` and
 * returns after it has finished.  Each element needs A >= 0, C > 0 when
 * A = 0, lo <= hi and finite coefficients; any other element gets x = NaN
 * and the call returns ADMM_EINVAL (the others are still solved).
 * ADMM_EINVAL also for NULL arrays, count < 0 or a bad xmin_mode;
 * ADMM_ENOMEM / ADMM_ECUDA on device errors. */
admm_status admm_quartic_min(const double *A, const double *B, const double *C, const double *D, const double *lo,
                             const double *hi, int64_t count, double *x, int32_t xmin_mode, int32_t on_device,
                             void *stream);
admm_status admm_quartic_min_f32(const float *A, const float *B, const float *C, const float *D, const float *lo,
                                 const float *hi, int64_t count, float *x, int32_t xmin_mode, int32_t on_device,
                                 void *stream);

/* Solve without any allocation, for callers that cannot allocate device
 * memory: code in host callbacks or real-time control loops where an
 * allocation may block or fail, controllers with a memory budget fixed at
 * start-up, and plugins whose host application owns every allocation.  The
 * paper has no counterpart; this is a deployment variant of admm_solve.
 *
 * The caller passes everything: `prob` and `state` hold device pointers in
 * the dense layout above (on_device = 1 for both; rows are n values apart,
 * unpadded, so loads may coalesce less well than in admm_solve, whose
 * handle pads rows to 32 doubles).  `state` is in/out: the solve starts
 * from it (state->cold = 1 starts from zero: x is set to clamp(0) and every
 * other array to 0, ignoring their contents) and leaves the final state in
 * it, including rho and cold.  The problem is validated before anything of
 * the caller's is written: ADMM_EINVAL (invalid data as in admm_create)
 * leaves `state` as it was.  `out` may be NULL.
 * The solver's scratch lives in a fixed 4 MiB device array inside the
 * library.  A device holds it from the first call made on it (with CUDA's
 * lazy module loading, that call also loads the library's kernels, which
 * does allocate device memory) until the process exits.  Make the first
 * call on each device a warm-up at start-up, outside any real-time loop or
 * host callback and before any stream capture: it also looks up the
 * array's address.  Later calls allocate nothing.  Calls share the array
 * and it keeps the last call's contents; each call clears what must start
 * at zero, and calls that overlap on the GPU race on it, so the caller must
 * serialise them.  Instances whose scratch would exceed the array are
 * rejected with ADMM_EUNSUPPORTED (at most ADMM_MAX_PAIRS pairs on a
 * 152-SM GPU need under 200 KiB, so today the limit is not reached).  Only
 * ADMM_FP64 is available.  Returns as admm_solve, after the stream has
 * finished.  No cudaMalloc, cudaFree or other allocating call is made. */
admm_status admm_solve_noalloc(const admm_problem *prob, const admm_params *params, admm_state *state,
                               admm_result *out, void *stream);

/* ---- Batched solves --------------------------------------------------
 * Many independent instances of eq. (2), of uneven n, m and q, solved in one
 * persistent launch (replayed from a CUDA graph) in ADMM_MIXED precision.
 * The paper solves one instance at a time; batching is an addition.  Each
 * instance runs the iteration (a)-(i) of App. A on its own team of threads
 * (a whole CTA for instances above small_max_elements = m*q*n, one warp
 * below it) and stops on its own stop test; its arithmetic depends only on
 * its own shape and team kind, so it gives the same bits alone and in any
 * mix with the same configuration. */
typedef struct admm_batch admm_batch;
typedef struct admm_batch_config {
    int32_t warps_per_cta;        /* 4, 8 or 16 */
    int32_t ctas_per_sm;          /* 0 = as many as fit */
    int64_t small_max_elements;   /* instances with m*q*n <= this go to one-warp teams */
    int32_t cluster_size;         /* 1 (off), 2, 4 or 8: CTAs of a thread-block cluster team */
    int32_t reserved;             /* must be 0 */
    int64_t cluster_min_elements; /* instances with m*q*n > this go to cluster teams */
} admm_batch_config;

/* Validates every problem as admm_create does (m <= ADMM_MAX_M, m*q <=
 * ADMM_BATCH_MAX_PAIRS), packs them into device memory owned by the batch
 * (FP32 arrays; the problems may be host or device memory) and sets every
 * instance to the zero start.  params->precision must be ADMM_MIXED;
 * the settings apply to every instance.  Default configuration: 8 warps
 * per CTA, small_max_elements 0 (every instance on a whole-CTA team, the
 * fastest on mixed workloads of 50..400k elements), no clusters.
 * ADMM_EUNSUPPORTED if the packed arrays would exceed 2^32 - 1 elements
 * each (sum over the instances of m*q*ld; the kernel indexes them with
 * 32-bit offsets): split such a batch into several. */
admm_status admm_batch_create(const admm_problem *probs, int32_t count, const admm_params *params,
                              admm_batch **out);
/* Replaces the launch configuration (used from the next admm_batch_solve;
 * instance state is kept).  ADMM_EINVAL for warps_per_cta not 4, 8 or 16,
 * cluster_size not 1, 2, 4 or 8, a negative setting or reserved != 0;
 * ADMM_EUNSUPPORTED if clusters of that size cannot be co-resident. */
admm_status admm_batch_set_config(admm_batch *b, const admm_batch_config *cfg);
/* The configuration in use; ctas_per_sm reports the resident CTAs per SM
 * actually launched. */
admm_status admm_batch_get_config(admm_batch *b, admm_batch_config *cfg);
/* Times each candidate configuration (warps per CTA x team thresholds x
 * cluster size) on this batch, keeps the fastest, and resets every instance
 * to the zero start.  trial_iters > 0: each candidate runs that many
 * iterations (throughput; 4, 8, 16 warps x warp-team thresholds 0, 8192,
 * 32768 x clusters off, of 4 or 8 CTAs); trial_iters = 0: each candidate
 * runs the whole solve, so the time includes the tail of the slowest
 * instances (8 or 16 warps, no warp teams; clusters off, of 2 CTAs for
 * instances above 1e5, 1.5e5 or 2.5e5 elements, or of 4 above 2.5e5).  *chosen (may be NULL)
 * receives the choice.  ADMM_EINVAL for trial_iters < 0. */
admm_status admm_batch_autotune(admm_batch *b, int32_t trial_iters, admm_batch_config *chosen);
/* Enqueues the solve of every unfinished instance from its current state
 * on `stream` (asynchronous; replays a CUDA graph captured on first use). */
admm_status admm_batch_solve(admm_batch *b, void *stream);
/* Waits for `stream` and fills results[0..count-1] (NULL allowed; x and x1
 * buffers inside each result are filled when non-NULL).  Returns the first
 * non-OK instance status, or ADMM_OK. */
admm_status admm_batch_wait(admm_batch *b, void *stream, admm_result *results);
/* Per-instance record as in admm_get_info (valid after admm_batch_wait). */
admm_status admm_batch_get_info(admm_batch *b, int32_t idx, double *info, int32_t count);
/* Copies instance idx's state into `out` as FP64 arrays (layouts as in
 * admm_state; host or device buffers by out->on_device; NULL arrays are
 * skipped).  Synchronous.  ADMM_EINVAL for a bad idx. */
admm_status admm_batch_get_state(admm_batch *b, int32_t idx, admm_state *out);
/* Loads a state (e.g. a warm start) into instance idx and marks it unfinished. */
admm_status admm_batch_set_state(admm_batch *b, int32_t idx, const admm_state *in);
/* Every instance back to the zero start; records cleared. */
admm_status admm_batch_reset(admm_batch *b);
/* Frees everything the batch owns; NULL is accepted. */
admm_status admm_batch_destroy(admm_batch *b);

/* ---- Serving: continuous batching of re-solves --------------------------
 * A request loop for model-predictive control: each request is an instance
 * of eq. (2) (host arrays, copied at submit), optionally tied to a session
 * (one controller).  A worker thread runs ticks of `tick_iters` iterations
 * of the batched kernel over every instance on the GPU; between ticks it
 * retires finished instances and admits queued requests in arrival order
 * while the device store has room (memory-based admission; idle sessions
 * are evicted least-recently-used first) and a slot is free.  A session
 * keeps its instance resident after a solve, and its next request is
 * warm-started from that state moved one step forward on the device (the
 * receding horizon of Sec. II and Alg. 2); requests of a session run one at
 * a time in order.  The paper runs one solve per sampling instant; the
 * server is an addition.  ADMM_MIXED precision only. */
typedef struct admm_server admm_server;
typedef struct admm_server_config {
    int64_t store_elements;      /* device store capacity, in elements m*q*ld (ld = n rounded up to 4) */
    int32_t max_active;          /* instances on the GPU at once */
    int32_t tick_iters;          /* iterations per tick of the costliest active instance; the others
                                    run as many as fit in the same time */
    int32_t max_m, max_q;        /* largest m and q a request may have (m*q <= ADMM_BATCH_MAX_PAIRS) */
    admm_batch_config batch;     /* launch configuration of a tick */
} admm_server_config;

/* store 2^27 elements, 4096 active, 10 iterations per tick, max_m 4,
 * max_q 20, 8 warps per CTA, small_max_elements 0, no clusters. */
void admm_server_default_config(admm_server_config *cfg);
/* Allocates the device store and tables and starts the worker thread on
 * the current device.  ADMM_EUNSUPPORTED unless params->precision is
 * ADMM_MIXED; ADMM_EINVAL for rho <= 0 or a configuration out of range
 * (max_active, tick_iters, max_m, max_q < 1; m*q > ADMM_BATCH_MAX_PAIRS;
 * store_elements < 1024; batch settings as in admm_batch_set_config);
 * ADMM_EUNSUPPORTED for store_elements > 2^32 - 1 (32-bit array offsets
 * in the kernel); ADMM_ENOMEM / ADMM_ECUDA if an allocation or CUDA call
 * fails, with nothing left allocated. */
admm_status admm_server_create(const admm_params *params, const admm_server_config *cfg, admm_server **out);
/* Validates and queues a request; session >= 0 ties it to that session
 * (warm start from the session's resident state when the shapes match),
 * -1 for a one-off solve.  *ticket identifies it for admm_server_poll. */
admm_status admm_server_submit(admm_server *s, const admm_problem *prob, int64_t session, int64_t *ticket);
/* The newest sampling step of a receding horizon: its data at the new
 * last step k = n-1 (f, g [m][q], bounds [m], demand [q]; host memory).  A
 * session whose problem has scenario-shared maps (coef_shared = 1) takes
 * the new step's maps from scenario j = 0. */
typedef struct admm_step {
    int32_t m, q;
    const double *f2, *f1, *f0, *g2, *g1, *g0; /* [m][q] */
    const double *x_lo, *x_hi;                 /* [m] */
    const double *y;                           /* [q] */
} admm_step;
/* Re-solve of a session after one sampling instant: on the device, the
 * session's resident instance (data and state) moves one step forward,
 * `step` becomes its last step, and the solve warm-starts from the moved
 * state.  Only the new step crosses the bus.  The request fails with
 * ADMM_EINVAL (reported by admm_server_poll) if the session holds no
 * resident instance of that m, q (submit a full problem first).  The step
 * is checked elementwise (finite, f2, g2 >= 0, lo <= hi), not for sure
 * infeasibility. */
admm_status admm_server_submit_step(admm_server *s, int64_t session, const admm_step *step, int64_t *ticket);
/* Waits up to wait_ms for a request.  ADMM_EPENDING if not finished; else
 * fills `out` (status inside; x and x1 host buffers filled when non-NULL)
 * and times[0..2] = seconds from submit to admission, seconds from submit
 * to completion, 1 if warm-started; the ticket is then forgotten. */
admm_status admm_server_poll(admm_server *s, int64_t ticket, int32_t wait_ms, admm_result *out, double *times);
/* Takes up to `max` finished requests in ticket order: their tickets,
 * seconds from submit to completion, iterations and status; *count gets
 * how many.  Drained tickets are forgotten (their x is not kept). */
admm_status admm_server_drain(admm_server *s, int32_t max, int64_t *tickets, double *latency_s, int32_t *iters,
                              int32_t *status, int32_t *count);
/* stats[0..9]: ticks, admitted, finished, active, queued, free fraction of
 * the store, sessions, seconds the GPU spent running ticks, seconds it spent
 * moving step requests' instances one step forward, and the sum over ticks
 * of the instances each tick ran. */
admm_status admm_server_stats(admm_server *s, double *stats, int32_t count);
/* Cancels a request.  A queued request leaves the queue at once; a running
 * one leaves at the next tick boundary (its session keeps the state reached
 * so far for the next warm start).  Either way it finishes with status
 * ADMM_ECANCELLED and no x.  A finished request is left as it is.
 * ADMM_EINVAL for an unknown ticket. */
admm_status admm_server_cancel(admm_server *s, int64_t ticket);
/* Stops the worker (in-flight requests are dropped) and frees everything;
 * NULL is accepted. */
admm_status admm_server_destroy(admm_server *s);

/* Message of the last failing call on this thread ("" if none). */
const char *admm_last_error(void);
/* Short English description of a status code ("ok", "invalid argument",
 * ...); a static string. */
const char *admm_status_string(admm_status s);

#ifdef __cplusplus
}
#endif
#endif /* ADMM_H */
