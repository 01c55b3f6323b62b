/*
 * ot_assoc.h -- C ABI of the GB300 entropic-OT device-association library.
 *
 * Method: Paschos, Liakopoulos, Debbah, Wen, "Computational Optimal Transport
 * for 5G Massive C-RAN Device Association" (arXiv 1805.01559).
 *   Sec. II-A   downlink rate R_ij = W log2(1 + SINR_ji), all other RRHs interfere
 *   Sec. II-B   RRH load rho_j = sum_i lambda_i pi_ij / (mu R_ij)
 *   Sec. III-B  regularized OT, Eq. (5); Algorithm 1 (Sinkhorn)
 *   Sec. IV     OT instance: C_ij = 1/(mu R_ij), p = lambda, q = RRH target; Lemma 1
 *   Sec. V      Algorithm 2 (adaptive Sinkhorn association)
 *
 * Conventions (every entry point):
 *   * i indexes devices (rows, I of them), j indexes RRHs (columns, J of them).
 *     Matrices are row-major I x J with a leading dimension `ld` (elements between
 *     the starts of consecutive rows; ld = 0 means ld = J).
 *   * Pointers marked [device] are CUDA device pointers owned by the caller; the
 *     library never frees or retains them past the call.  Pointers marked [host]
 *     are ordinary host memory.  Scratch memory is owned by the context.
 *   * `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is stream-ordered.  Entry points that return host scalars synchronise
 *     the stream before returning; the others only enqueue.
 *   * Errors are returned as ot_status codes; nothing aborts, traps or throws.
 *     On error the message is available from ot_assoc_last_error(ctx).
 *   * Potentials: pi_ij = exp((f_i + g_j - C_ij) / eps) (Sec. III-B, KKT form
 *     pi = xi e^{-alpha} e^{-beta}: f_i = -eps alpha_i, g_j = -eps beta_j, i.e.
 *     a_i = exp(f_i/eps), b_j = exp(g_j/eps) of Algorithm 1).
 *   * The marginals are each normalised by their own sum before iterating; they
 *     must balance (Eqs. 3-4 force sum p = sum q) to 1e-5 relative.  Residuals and
 *     `tol` refer to the unit-mass plan: err = sum_i |sum_j pi_ij - p_i| / sum p.
 *   * Stopping rule ("while accuracy" of Algorithm 1, with the "total absolute
 *     residual" of Sec. III-C): after each full iteration k (a-update then
 *     b-update) the row residual of pi^(k) is compared with `tol`; the loop ends at
 *     the first k with residual <= tol, or at k = max_iter (status
 *     OT_NOT_CONVERGED, results still valid).  The FP32 solvers form that residual
 *     from FP32 cell values and stop at residual <= tol (1 - 2^-5): the FP32 figure
 *     sits within about 1e-8 of the exact residual of the returned potentials, so the
 *     returned plan's exact FP64 residual stays <= tol.
 */
#ifndef OT_ASSOC_H
#define OT_ASSOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OT_OK = 0,
    OT_NOT_CONVERGED = 1,  /* max_iter reached; f, g and the summary are valid */
    OT_EINVAL = -1,        /* bad size, pointer, parameter or input value */
    OT_ENOMEM = -2,        /* scratch would exceed the context's HBM budget, or cudaMalloc failed */
    OT_ECUDA = -3,         /* a CUDA runtime call failed (message has the CUDA error) */
    OT_ETIMEOUT = -4,      /* a bounded device-side wait gave up; the context stays usable */
    OT_EBUSY = -5,         /* serving: no free slot / budget right now */
    OT_EUNSUPPORTED = -6   /* shape outside the compiled kernel range (e.g. J > 8192) */
} ot_status;

typedef struct ot_assoc_ctx ot_assoc_ctx;

/* Library version (major*10000 + minor*100 + patch). */
int ot_assoc_version(void);

/* Human-readable name of a status code (static string). */
const char* ot_assoc_status_string(int status);

/*
 * Create a context on CUDA device `device`.  The context owns all scratch
 * memory; it never holds more than `hbm_budget_bytes` of it (0 = no limit other
 * than the device).  Returns OT_EINVAL for a bad device, OT_ECUDA on a CUDA error.
 * A context is not thread-safe: use one per host thread.  Its scratch is shared by
 * all calls, so calls on different streams must not overlap in time.
 */
ot_status ot_assoc_create(ot_assoc_ctx** ctx, int device, size_t hbm_budget_bytes);

/* Release the context and its scratch (first waiting for asynchronous solves still in
 * flight).  NULL is ignored. */
void ot_assoc_destroy(ot_assoc_ctx* ctx);

/* Last error message of this context ("" if none).  Valid until the next call. */
const char* ot_assoc_last_error(const ot_assoc_ctx* ctx);

/* Bytes of device scratch the context holds right now. */
size_t ot_assoc_scratch_bytes(const ot_assoc_ctx* ctx);

/*
 * Set the iteration bound of every device-side spin wait (grid barriers and
 * batch work queues).  A wait that exceeds it stops the kernel with
 * OT_ETIMEOUT instead of hanging.  Default 1 << 24 polls (seconds).  Values < 1
 * restore the default.
 */
void ot_assoc_set_spin_limit(ot_assoc_ctx* ctx, int64_t polls);

/*
 * Downlink rates, Sec. II-A:
 *   SINR_ij = P_j G_ij / (sum_{k != j} P_k G_ik + N0),   R_ij = W_hz * log2(1 + SINR_ij).
 * G   [device] float, I x J (ld_g, 0 = J): G[i*ld + j] = path gain RRH j -> device i, >= 0.
 * P   [device] float, J: transmit powers, >= 0.
 * R_out [device] float, I x J (ld_r, 0 = J).
 * The interference sum is formed per row in FP64 (total minus own term); the
 * rate uses log1p.  Enqueue only.  OT_EINVAL for I, J <= 0, N0 < 0, W_hz <= 0.
 */
ot_status ot_assoc_build_rates(ot_assoc_ctx* ctx, const float* G, int64_t ld_g, const float* P,
                               int64_t I, int64_t J, double N0, double W_hz, float* R_out,
                               int64_t ld_r, void* stream);

/*
 * Cost per unit traffic, Sec. IV choice (ii):  C_ij = 1 / (mu R_ij).
 * R     [device] float, I x J (ld_r, 0 = J), every entry finite and > 0.
 * C_out [device] float, I x J (ld_c, 0 = J).
 * If eps_out != NULL, also *eps_out [host] = eps_rel * median(C), the median
 * over all I*J entries of the FP32 C (mean of the two middle values when I*J is
 * even); this synchronises the stream.  OT_EINVAL for a non-positive or
 * non-finite R entry (checked on the device), mu <= 0, or eps_rel <= 0 with
 * eps_out given.
 */
ot_status ot_assoc_build_cost(ot_assoc_ctx* ctx, const float* R, int64_t ld_r, int64_t I,
                              int64_t J, double mu, float* C_out, int64_t ld_c, double eps_rel,
                              double* eps_out, void* stream);

/*
 * Rates and cost in one pass over the gains (Sec. II-A then Sec. IV choice (ii)): the same
 * values as ot_assoc_build_rates followed by ot_assoc_build_cost, without writing and
 * re-reading R.  R_out [device] (ld_r) may be NULL; C_out [device] float I x J (ld_c);
 * eps_out / eps_rel as ot_assoc_build_cost (the median synchronises the stream; invalid
 * rates are reported then as OT_EINVAL).  G 16-byte aligned rows are read in place.
 */
ot_status ot_assoc_build_cost_from_gains(ot_assoc_ctx* ctx, const float* G, int64_t ld_g, const float* P,
                                         int64_t I, int64_t J, double N0, double W_hz, double mu,
                                         float* R_out, int64_t ld_r, float* C_out, int64_t ld_c,
                                         double eps_rel, double* eps_out, void* stream);

/*
 * Exact median of n floats (no NaN): the middle order statistic, or the mean of
 * the two middle ones for even n.  x [device]; *median_out [host].  Synchronises.
 */
ot_status ot_assoc_median_f32(ot_assoc_ctx* ctx, const float* x, int64_t n, double* median_out,
                              void* stream);

/*
 * maxSINR (strongest-signal) association, Sec. II-C and Lemma 1: device i picks
 * j*(i) = argmax_j R_ij (lowest j on ties).
 * R        [device] float I x J (ld_r, 0 = J);  traffic [device] float, I.
 * assoc_out  [device] int32, I (may be NULL).
 * Lambda_out [device] double, J: Lambda_j = sum_{i: j*(i)=j} traffic_i (may be NULL).
 * *total_load_out [host] (may be NULL; synchronises): sum_i traffic_i / (mu R_{i j*(i)}).
 */
ot_status ot_assoc_maxsinr(ot_assoc_ctx* ctx, const float* R, int64_t ld_r, const float* traffic,
                           int64_t I, int64_t J, double mu, int32_t* assoc_out,
                           double* Lambda_out, double* total_load_out, void* stream);

/* Outputs of a solve.  Device pointers are caller-owned; NULL = do not produce. */
typedef struct {
    float* pi;             /* [device] I x J plan (mass units of the caller's p), ld = pi_ld */
    int64_t pi_ld;         /* 0 = J */
    double* f;             /* [device] I: potentials f_i (required) */
    double* g;             /* [device] J: potentials g_j (required; read first when warm_start) */
    double* rrh_load;      /* [device] J: rho_j = sum_i C_ij pi_ij (Sec. II-B with x = pi) */
    double transport_cost; /* [host-filled] sum_ij C_ij pi_ij (objective of Eq. 2) */
    double marg_err_row;   /* [host-filled] sum_i |sum_j pi_ij - p_i| / sum p, FP64 reduction */
    double marg_err_col;   /* [host-filled] sum_j |sum_i pi_ij - q_j| / sum p, FP64 reduction */
    int32_t iters;         /* [host-filled] completed Sinkhorn iterations k */
    int32_t status;        /* [host-filled] same as the return value */
    int32_t absorptions;   /* [host-filled] kernel rebuilds (stored-kernel forms; 0 otherwise) */
    int32_t reserved;
} ot_assoc_result;

/*
 * Algorithm 1 on the OT instance of Sec. IV: builds C = 1/(mu R) into context
 * scratch, then solves Eq. (5) in the log domain with FP32 per-cell arithmetic.
 * R             [device] float I x J (ld_r, 0 = J), finite and > 0.
 * traffic       [device] float I: p = lambda (> 0).
 * rrh_marginal  [device] float J: q (> 0), sum q = sum p.
 * eps > 0 (absolute), tol >= 0, max_iter >= 1.  warm_start != 0 starts from
 * b = exp(out->g / eps) instead of b = 1 (Algorithm 1's initialisation).
 * Synchronises the stream (the summary scalars are host-filled).  Returns
 * OT_OK, OT_NOT_CONVERGED, or an error (then `out` is unspecified).
 */
ot_status ot_assoc_solve(ot_assoc_ctx* ctx, const float* R, int64_t ld_r, const float* traffic,
                         const float* rrh_marginal, int64_t I, int64_t J, double mu, double eps,
                         double tol, int32_t max_iter, int32_t warm_start, ot_assoc_result* out,
                         void* stream);

/*
 * Same as ot_assoc_solve for a caller-built cost matrix (Eq. 5 with any finite C;
 * +inf entries mean "no link", but every row and column needs a finite entry).
 * C [device] float I x J with ld_c (0 = J).  A C whose ld_c is a multiple of 4
 * and whose base is 16-byte aligned is read in place, in 16-byte chunks (so the
 * allocation must extend to the end of the last row's final 16-byte chunk);
 * otherwise it is first copied into aligned scratch.
 */
ot_status ot_assoc_solve_cost(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* p,
                              const float* q, int64_t I, int64_t J, double eps, double tol,
                              int32_t max_iter, int32_t warm_start, ot_assoc_result* out,
                              void* stream);

/*
 * Algorithm 1 with the Euclidean cost of Sec. IV (cost choice (i)), C_ij = ||x_i - x_j||,
 * formed inside every sweep from the coordinates instead of read from a matrix: no I x J
 * array exists, each cell costs a square root and an exponential.  C_ij is evaluated in
 * FP32 as sqrt((x_i - x_j)^2 + (y_i - y_j)^2) with every operation correctly rounded and
 * none fused, so a solve on a matrix built with that formula gives the same result.
 *   dev_xy [device] float I x 2 (x, y per device), rrh_xy [device] float J x 2, 8-byte aligned.
 * Other arguments and results as ot_assoc_solve_cost (rrh_load and the transport cost are
 * those of the Euclidean cost).  Synchronises `stream`.
 */
ot_status ot_assoc_solve_euclid(ot_assoc_ctx* ctx, const float* dev_xy, const float* rrh_xy, const float* p,
                                const float* q, int64_t I, int64_t J, double eps, double tol,
                                int32_t max_iter, int32_t warm_start, ot_assoc_result* out, void* stream);

/*
 * Up to three solves of Algorithm 1 on ONE cost matrix (the same C, p and q, an eps sweep:
 * eps[k], tol[k] for k < n) in one persistent launch.  Each solve follows the single-solve
 * algorithm and stopping rule exactly; the plan-scale sweeps of the solves still iterating
 * share each read of C, so the launch reads C max(iters) + 2 n times instead of
 * sum(iters) + 2 n.  outs [host] n results (device pointers as for ot_assoc_solve_cost; host
 * fields filled).  The team width is chosen for three solves' registers, so results agree
 * with ot_assoc_solve_cost to rounding, not bit for bit.  Limits: 1 <= n <= 3, J <= 4096;
 * one status for the launch (a solve that breaks down fails all).  Synchronises `stream`.
 * Returns OT_OK when every solve converged, OT_NOT_CONVERGED when some stopped at max_iter.
 */
ot_status ot_assoc_solve_cost_multi(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* p,
                                    const float* q, int64_t I, int64_t J, int32_t n, const double* eps,
                                    const double* tol, int32_t max_iter, ot_assoc_result* outs,
                                    void* stream);

/*
 * ot_assoc_solve_cost without waiting: the solve is enqueued on `stream` and *ticket [host]
 * identifies it.  `out` supplies the device pointers (f, g, pi, rrh_load), which must stay
 * valid until the solve completes; ot_assoc_wait fills the host fields.  Up to 16 solves may
 * be in flight per context (OT_EBUSY beyond); they share the context's scratch, so they must
 * be enqueued on ONE stream (they then run one after another).  Argument errors are returned
 * at once; device-side outcomes (invalid input, numerical breakdown, timeout, not converged)
 * by ot_assoc_wait.
 */
ot_status ot_assoc_solve_cost_async(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* p,
                                    const float* q, int64_t I, int64_t J, double eps, double tol,
                                    int32_t max_iter, int32_t warm_start, const ot_assoc_result* out,
                                    uint64_t* ticket, void* stream);

/* Block until the asynchronous solve `ticket` has completed and fill out's host fields
 * (transport_cost, residuals, iters, status) as ot_assoc_solve_cost would; returns its
 * status.  Each ticket can be waited for once (OT_EINVAL for an unknown ticket). */
ot_status ot_assoc_wait(ot_assoc_ctx* ctx, uint64_t ticket, ot_assoc_result* out);

/*
 * ot_assoc_solve_cost without any memory allocation (the paper has no counterpart: this
 * is a service of the library, not a step of the method).
 *
 * For callers that cannot allocate device memory when they solve: for example a radio
 * scheduler that re-associates devices every few milliseconds and must not stall on
 * cudaMalloc/cudaFree (which may synchronise the device and take unbounded time), or a
 * process confined to a fixed memory pool.  It takes no context: all scratch lives in one
 * file-scope device array of 8 MiB that is part of the library image, so every GPU that
 * loads the library holds those 8 MiB until the process exits.  Nothing is allocated,
 * freed, or taken from PyTorch's allocator; no event or pinned buffer is created.
 *
 * Limits: I <= 131072 devices, J <= 1024 RRHs (OT_EUNSUPPORTED beyond), C read in place,
 * so ld_c must be a multiple of 4 and C 16-byte aligned (OT_EINVAL otherwise).  Same
 * arguments, outputs, stopping rule and status codes as ot_assoc_solve_cost; error
 * messages are not recorded (there is no context), only the status code.
 *
 * Every call looks up the array's device address in the current device's context
 * (cudaGetSymbolAddress, which allocates nothing), so the entry point keeps working after
 * the context is destroyed and re-created.  The first call on a device may load the
 * library's device code into that context: make it before any stream capture.
 * Every call on a device shares the one array and overwrites what the previous call left
 * there (the state words are cleared at the start of each call): calls whose GPU work
 * overlaps -- on different streams or from different threads -- race and give wrong
 * results, or return OT_ETIMEOUT after the fixed limit of 2^24 polls of a grid barrier
 * (one call's clearing of the state words can reset another call's barrier counters).
 * Synchronises the stream before returning.
 */
ot_status ot_assoc_solve_cost_noalloc(const float* C, int64_t ld_c, const float* p, const float* q,
                                      int64_t I, int64_t J, double eps, double tol, int32_t max_iter,
                                      int32_t warm_start, ot_assoc_result* out, void* stream);

/*
 * FP64 variant of ot_assoc_solve_cost (all per-cell arithmetic in double).
 * C [device] double I x J (ld_c, 0 = J); p [device] double I; q [device] double J.
 * out->pi, if given, is still float.
 */
ot_status ot_assoc_solve_f64(ot_assoc_ctx* ctx, const double* C, int64_t ld_c, const double* p,
                             const double* q, int64_t I, int64_t J, double eps, double tol,
                             int32_t max_iter, int32_t warm_start, ot_assoc_result* out,
                             void* stream);

/*
 * Device timings of the last solve on this context (CUDA events recorded on the
 * solve's stream around each phase; only while timing is enabled).
 */
typedef struct {
    double init_ms;      /* state reset before the persistent kernel */
    double loop_ms;      /* the persistent kernel: setup, iteration 1, every later iteration,
                            the finalize sweep (it reads C iters + 2 times) */
    double finalize_ms;  /* FP64 column totals and the summary */
    int32_t sweeps;      /* completed iterations (the kernel reads C sweeps + 2 times) */
    int32_t valid;       /* 1 when the fields above belong to the last solve */
} ot_assoc_timings;

/* Turn phase timing on (1) or off (0).  Off by default; costs a few events per solve. */
void ot_assoc_enable_timing(ot_assoc_ctx* ctx, int on);

/* Timings of the last solve (valid = 0 if timing was off or the solve failed). */
ot_status ot_assoc_last_timings(const ot_assoc_ctx* ctx, ot_assoc_timings* out);

/* Number of CUDA kernels this context has launched so far (all entry points). */
uint64_t ot_assoc_launch_count(const ot_assoc_ctx* ctx);

/* Storage of the Gibbs kernel in the stored-kernel (scaling-domain) form. */
typedef enum {
    OT_KERNEL_F32 = 0,
    OT_KERNEL_BF16 = 1,
    OT_KERNEL_F16 = 2
} ot_kernel_format;

/*
 * Stored-kernel form of Algorithm 1 (the a/b scaling iteration as printed) with
 * absorption: K~_ij = exp((fh_i + gh_j - C_ij)/eps) is kept in `format`
 * (each row scaled so its largest entry is 1), the scalings a, b are FP32, and
 * whenever a scaling leaves [2^-absorb_log2, 2^absorb_log2] relative to its
 * value at the last rebuild it is folded into (fh, gh) and K~ is rebuilt from C
 * (absorb_log2 <= 0 selects the format's default).  Accumulation is FP32; the
 * final summary uses FP64 reductions.  The first iteration runs in the log
 * domain from C so that no column can underflow.
 * C [device] float I x J (ld_c, 0 = J), kept for rebuilds; other arguments as
 * ot_assoc_solve_cost.
 */
ot_status ot_assoc_solve_lowp(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* p,
                              const float* q, int64_t I, int64_t J, double eps, double tol,
                              int32_t max_iter, int32_t warm_start, int32_t format,
                              double absorb_log2, ot_assoc_result* out, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched ragged solves: many independent instances of Algorithm 1 (each its own I x J
 * cost, marginals and eps) in ONE persistent launch.  The CTAs of the launch form groups;
 * each group takes instances from a queue (largest first), solves one exactly as
 * ot_assoc_solve_cost does (same arithmetic, same stopping rule) and finalizes it in the
 * same launch.  The group size and the stage size (rows of C per bulk copy) come from
 * the context's tuning table per size bucket (ot_assoc_autotune), else from defaults.
 * Limits: J <= 1024 per instance (OT_EUNSUPPORTED above); C read in place, so it must be
 * 16-byte aligned with ld % 4 == 0 (OT_EINVAL otherwise).
 * ------------------------------------------------------------------------------------- */
typedef struct {
    const float* C;     /* [device] I x J cost, ld (0 = J), 16-byte aligned rows */
    int64_t ld;
    int64_t I;
    int32_t J;
    int32_t warm_start; /* != 0: start from b = exp(g / eps) with the g given below */
    const float* p;     /* [device] I, > 0 */
    const float* q;     /* [device] J, > 0, sum q = sum p (1e-5 relative) */
    double eps;         /* > 0, absolute */
    double tol;         /* >= 0, row residual of the unit-mass plan */
    int32_t max_iter;   /* >= 1 */
    int32_t reserved;
    double* f;          /* [device] I: potentials f_i (required) */
    double* g;          /* [device] J: potentials g_j (required; read first when warm_start) */
    double* rrh_load;   /* [device] J: rho_j = sum_i C_ij pi_ij, or NULL */
    float* pi;          /* [device] I x J plan, or NULL */
    int64_t pi_ld;      /* 0 = J */
} ot_assoc_instance;

typedef struct {
    double transport_cost; /* sum_ij C_ij pi_ij (caller's mass units), FP64 reduction */
    double marg_err_row;   /* sum_i |sum_j pi_ij - p_i| / sum p */
    double marg_err_col;   /* sum_j |sum_i pi_ij - q_j| / sum p */
    double err_loop;       /* residual estimate that stopped the loop */
    int32_t iters;         /* completed iterations */
    int32_t status;        /* OT_OK, OT_NOT_CONVERGED, OT_EINVAL (bad marginals or a
                              numerical breakdown), OT_ETIMEOUT (the launch gave up) */
    int32_t converged;     /* 1 when the loop stopped at residual <= tol */
    int32_t reserved;
} ot_assoc_instance_result;

/* A planned batch: schedule, device tables and (unless OT_BATCH_NO_GRAPH) a captured CUDA
 * graph holding descriptor upload, control reset, the persistent launch and the result
 * download.  Owned by the caller; destroy with ot_assoc_batch_destroy before the context. */
typedef struct ot_assoc_batch ot_assoc_batch;

enum { OT_BATCH_NO_GRAPH = 1 /* enqueue the launch directly instead of replaying a graph */ };

/* One-shot: plan, run on `stream`, wait, fill res[0..n) [host].  Returns OT_OK when the
 * launch completed (per-instance outcomes are in res[k].status), else an error. */
ot_status ot_assoc_solve_batched(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int32_t n,
                                 ot_assoc_instance_result* res, void* stream);

/* Plan a batch of n instances [host array, copied] and capture its graph. */
ot_status ot_assoc_batch_create(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int32_t n,
                                int32_t flags, ot_assoc_batch** out);

/* Replace instance k's pointers and parameters (I, J and ld must stay the same); takes
 * effect at the next launch.  Must not be called while a launch of this batch is running. */
ot_status ot_assoc_batch_set(ot_assoc_batch* b, int32_t k, const ot_assoc_instance* inst);

/* Enqueue one run of the batch on `stream` (graph replay); returns at once. */
ot_status ot_assoc_batch_launch(ot_assoc_batch* b, void* stream);

/* Synchronise `stream` and fill res[0..n) [host] (res may be NULL). */
ot_status ot_assoc_batch_wait(ot_assoc_batch* b, void* stream, ot_assoc_instance_result* res);

/* Free the batch's graph, descriptors and scratch.  Call it with no launch of the batch
 * running (after ot_assoc_batch_wait).  NULL is a no-op.  Destroy batches before their
 * context. */
void ot_assoc_batch_destroy(ot_assoc_batch* b);

/* Autotune the tuning table on a batch: bucket by bucket, time the whole batch (iters
 * iterations, outputs to scratch, the callers' buffers untouched) with the bucket's
 * instances on the candidate (group size, stage size) pairs, keep the fastest. */
ot_status ot_assoc_autotune(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int32_t n,
                            int32_t iters, void* stream);

/* Tuning table: per instance size bucket b in [0, 15) (cells class * 3 + J class), the
 * schedule (CTAs per instance group, a divisor of the SM count; 0 = untuned: a model picks
 * it from the instance's estimated sweep time) and the tile (stage size in bytes, rows of
 * C per bulk copy; 0 = 24 KB); rate = cells * iterations / s of the batch it was tuned on.
 * The choice depends on the instance alone, so an instance's result is the same bit for
 * bit in any batch. */
ot_status ot_assoc_tuning_get(const ot_assoc_ctx* ctx, int32_t bucket, int32_t* gsize,
                              int32_t* stage_bytes, double* rate);
/* Set bucket's entry: gsize 0 or a divisor of the SM count, stage_bytes >= 0 (0: 24 KB);
 * OT_EINVAL otherwise (or for a bucket outside [0, 15)).  Applies to batches planned
 * afterwards. */
ot_status ot_assoc_tuning_set(ot_assoc_ctx* ctx, int32_t bucket, int32_t gsize, int32_t stage_bytes);
/* Size bucket of an I x J instance. */
int32_t ot_assoc_bucket(int64_t I, int32_t J);

/* ---------------------------------------------------------------------------------------
 * Policy evaluation (Sec. II-B, Sec. IV).
 * ------------------------------------------------------------------------------------- */
/* Euclidean cost, Sec. IV cost choice (i): C_ij = ||x_i - x_j|| in the coordinates' unit.
 * dev_xy [device] float I x 2 (x, y per device), rrh_xy [device] float J x 2, both 8-byte
 * aligned; C_out [device] float I x J, ld_c (0 = J).  Formed in FP64, rounded once to FP32.
 * Only enqueues. */
ot_status ot_assoc_euclid_cost(ot_assoc_ctx* ctx, const float* dev_xy, const float* rrh_xy, int64_t I,
                               int64_t J, float* C_out, int64_t ld_c, void* stream);

/* Average job completion time of an association, Sec. II-B (processor sharing at each RRH):
 *   rho_j = sum_i C_ij x_ij,  T = (1/I) sum_i sum_j pi_ij C_ij / (1 - rho_j),
 * with C [device] float I x J (ld_c, 0 = J) the LOAD cost 1/(mu R_ij), x the plan in mass
 * units and pi_ij = x_ij / lambda_i the association fractions.  The plan is either
 *   assoc   [device] int32 I: hard association (x_ij = lambda_i when j = assoc_i), or, when
 *           assoc is NULL, the entropic plan x_ij = exp((f_i + g_j - Cp_ij) / eps) of
 *           potentials f [device] double I, g [device] double J on the plan cost Cp =
 *           C_plan [device] float I x J (ld_plan, 0 = J), or on C itself when C_plan is NULL.
 * traffic [device] float I, lambda_i > 0 (OT_EINVAL otherwise).  rho_out [device] double J
 * or NULL.  T_out [host]: +inf when an RRH that carries traffic has rho_j >= 1.  Column sums
 * are FP64 in a fixed order (deterministic).  Synchronises `stream`. */
ot_status ot_assoc_completion_time(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* traffic,
                                   int64_t I, int64_t J, const int32_t* assoc, const float* C_plan,
                                   int64_t ld_plan, const double* f, const double* g, double eps,
                                   double* rho_out, double* T_out, void* stream);

/* Mean over the I rows of min_j C_ij (each device's cheapest link), FP64 sums in a fixed
 * order.  C [device] float I x J (ld_c, 0 = J); *out [host].  Synchronises `stream`.  Used as
 * the scale of eps in the policy comparison (a regularisation relative to the cost of the
 * links a plan actually uses). */
ot_status ot_assoc_mean_row_min(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, int64_t I, int64_t J,
                                double* out, void* stream);

/* ---------------------------------------------------------------------------------------
 * eps-scaling (annealing) for Algorithm 1, in ONE persistent launch.  Stages solve Eq. (5)
 * at eps_s = eps0 * factor^s while that is above eps, then at eps itself; each stage starts
 * from the previous stage's g (the first from b = 1, or from the caller's g when warm_start).
 * Intermediate stages stop at residual <= tol_stage, the last at tol; every stage is capped
 * at max_iter iterations.  The result is the solution at `eps` exactly as ot_assoc_solve_cost
 * defines it (same arithmetic and stopping rule); the stages only choose where its iteration
 * starts.  Arguments as ot_assoc_solve_cost, plus:
 *   eps0 >= eps, 0 < factor < 1 (at most 64 stages);
 *   stage_iters [host] int32 per stage (<= 64 entries) or NULL; *nstages_out [host] or NULL.
 * out->iters is the total over the stages; the summary is the last stage's.  Limits: J <= 1024,
 * C 16-byte aligned with ld_c % 4 == 0.  Synchronises `stream`.
 * ------------------------------------------------------------------------------------- */
ot_status ot_assoc_solve_eps_scaling(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* p,
                                     const float* q, int64_t I, int64_t J, double eps, double eps0,
                                     double factor, double tol_stage, double tol, int32_t max_iter,
                                     int32_t warm_start, ot_assoc_result* out, int32_t* stage_iters,
                                     int32_t* nstages_out, void* stream);

/* Measurement: the FP32 exp2 throughput of ctx's device (the SFU, one ex2.approx a cell and
 * sweep in every Algorithm 1 solver here), from 8 independent exp2 chains a thread over
 * 8 blocks of 256 threads an SM, timed with events (best of 3 after a warm-up launch).
 * *ex2_per_s [host].  Synchronises `stream`; a few ms. */
ot_status ot_assoc_measure_ex2_rate(ot_assoc_ctx* ctx, double* ex2_per_s, void* stream);

/* ---------------------------------------------------------------------------------------
 * Row-sharded Algorithm 1 (Sec. III-C, Eqs. (3)-(5)): the rows of C split into contiguous
 * shards (one per rank / GPU).  The row update (Eq. (3)) only needs a shard's own rows; the
 * column update (Eq. (4)) needs the column sums of every shard, so one iteration is
 *   ot_assoc_shard_sweep(ITER)   on every shard,
 *   a SUM over the shards of col_out (J doubles) and row_out (1 double)  [the caller's
 *   collective, e.g. an all-reduce],
 *   ot_assoc_shard_update(ITER)  on every rank (same inputs, same G).
 * The cell, the stopping rule and the outputs are those of ot_assoc_solve_cost; a driver
 * that strings the calls together is paper_1805_01559_gb300.sharded.  Common arguments:
 *   C        [device] float I x J, this shard's rows; 16-byte aligned, ld_c % 4 == 0 (0 = J)
 *   p        [device] float I, this shard's row marginals (> 0)
 *   inv_mass = 1 / (sum of p over ALL shards) (host), so p^_i = p_i * inv_mass
 *   eps      > 0 (absolute); k = log2(e) / eps
 *   G        [device] double J: column potentials in log2 units (g_j = eps ln2 G_j)
 *   F_in, F_out [device] float 2 I: row potentials F'_i as (hi, lo) FP32 pairs, row-relative
 *            log2 units: t_ij = 2^(F'_i + G_j - k C_ij) = pi_ij / p_i
 * Modes of the sweep (outputs summed over the shards unless said otherwise):
 *   OT_SHARD_FIRST  iteration 1 from G: F_out = F'^1 = -log2 sum_j 2^(G_j - k C_ij);
 *                   col_out[j] = 2^64 sum_i p^_i 2^(F'^1_i + G_j - k C_ij)
 *   OT_SHARD_ITER   F_in = F'^(k-1): F_out = F'^k (Eq. (3)); col_out[j] = s_j =
 *                   sum_i p^_i 2^(F'^k_i + G_j - k C_ij); row_out = sum_i p^_i |r_i - 1|,
 *                   r_i = sum_j t_ij: the row residual of the plan (F'^(k-1), G)
 *   OT_SHARD_COLMAX col_out[j] = max_i (F_in_i + G_j - k C_ij + log2 p^_i)  (reduce with MAX)
 *   OT_SHARD_COLSUM col_out[j] = sum_i 2^(F_in_i + G_j - k C_ij + log2 p^_i - M_j), M = colmax
 *                   (the reduced COLMAX output): COLMAX then COLSUM take iteration 1's
 *                   column sums exactly when FIRST's scaled sums underflow
 *   OT_SHARD_FINAL  plan (F_in, G): col_out[0..J) = sum_i p^_i t_ij, col_out[J..2J) =
 *                   sum_i p^_i C_ij t_ij; row_out = sum_i p^_i |r_i - 1| (FP32 pair row sums);
 *                   f_out [device] double I (this shard) = eps ln2 (F'_i + log2 p_i), or NULL
 * col_out [device] double J (2 J for FINAL); row_out [device] double 1 (ITER, FINAL).
 * state [device] double 4 or NULL: the loop state of ot_assoc_shard_update; while state[0]
 * is not 0 the sweep does nothing (so a caller can enqueue iterations ahead of the stop).
 * Per-block FP64 partials added in block order: deterministic for a given shard and device.
 * Uses the context's scratch: issue a context's shard calls on one stream.  Only enqueues.
 * OT_EUNSUPPORTED for J > 8192; OT_EINVAL for a misaligned C or a missing buffer.
 * ------------------------------------------------------------------------------------- */
enum {
    OT_SHARD_FIRST = 0,
    OT_SHARD_ITER = 1,
    OT_SHARD_COLMAX = 2,
    OT_SHARD_COLSUM = 3,
    OT_SHARD_FINAL = 4
};

/* out [device] double 3: sum of this shard's p, sum of q, and 1.0 when an entry of p or q is
 * not positive and finite (else 0.0).  Fixed summation order.  Only enqueues. */
ot_status ot_assoc_shard_mass(ot_assoc_ctx* ctx, const float* p, int64_t I, const float* q, int64_t J,
                              double* out, void* stream);

ot_status ot_assoc_shard_sweep(ot_assoc_ctx* ctx, int mode, const float* C, int64_t ld_c, const float* p,
                               int64_t I, int64_t J, double inv_mass, double eps, const double* G,
                               const float* F_in, float* F_out, const double* colmax, double* col_out,
                               double* row_out, double* f_out, const double* state, void* stream);

/* Column update (Eq. (4)) from the summed col of every shard, q [device] float J,
 * inv_qmass = 1 / sum q:
 *   FIRST   G_out = G_in + log2 q^ - (log2 col - 64); a column whose scaled sum is below 2^-60
 *           (or not finite) sets bit 1 of *flag and leaves its G_out entry unset: take
 *           iteration 1 again with COLMAX / COLSUM (G_in is unchanged when G_out differs)
 *   COLSUM  G_out = G_in + log2 q^ - (M + log2 col), M = colmax as the sweep rounded it
 *   ITER    G_out = G_in + log2 q^ - log2 col
 * A sum that is not positive and finite sets bit 2 of *flag (numeric failure).  flag
 * [device] int32, only ever OR-ed: the caller zeroes it.  G_out may equal G_in.
 * Loop state (ITER with state [device] double 4, zeroed by the caller before the loop; else
 * NULL and err, iter, tol_stop, max_iter unused): the update first takes the loop test of
 * Algorithm 1 on the summed row residual *err [device] (of the plan (F'^(iter-1), G_in)):
 * when err <= tol_stop or iter - 1 >= max_iter (or err is not finite) it leaves G as it is and
 * sets state = {reason, iter - 1, (iter - 1) & 1, err}, reason 1 = converged, 2 = max_iter,
 * 3 = numeric failure (also set when a column sum fails); (iter - 1) & 1 is the F buffer of the
 * returned plan when F'^k is written to buffer k & 1.  Every update and sweep that sees
 * state[0] != 0 does nothing.  Only enqueues. */
ot_status ot_assoc_shard_update(ot_assoc_ctx* ctx, int mode, const float* q, int64_t J, double inv_qmass,
                                const double* col, const double* colmax, const double* G_in, double* G_out,
                                int32_t* flag, const double* err, int32_t iter, double tol_stop,
                                int32_t max_iter, double* state, void* stream);

/* Totals of the FINAL sweep from the summed col2 (2 J) and row_err (1): summary [device]
 * double 3 = transport cost (mass * sum_j col2[J + j]), row residual, column residual
 * sum_j |col2[j] - q_j inv_qmass|; rho_out [device] double J (mass * col2[J + j]) or NULL;
 * g_out [device] double J = eps ln2 G, or NULL.  mass = sum of p over all shards.  Only
 * enqueues. */
ot_status ot_assoc_shard_finish(ot_assoc_ctx* ctx, const double* col2, const double* row_err, const float* q,
                                int64_t J, double mass, double inv_qmass, double eps, const double* G,
                                double* g_out, double* rho_out, double* summary, void* stream);

/* ---------------------------------------------------------------------------------------
 * Adaptive Sinkhorn association (Algorithm 2, Sec. V) in ONE persistent launch.
 * The RRH targets start from the equal split q_j = sum_i lambda_i / J (Algorithm 2,
 * initialisation).  Each outer step s:
 *   1. solves Algorithm 1 with (C, p = lambda, q^(s), eps), exactly as
 *      ot_assoc_solve_cost does (same arithmetic and stopping rule); steps after the first
 *      start from the previous step's g unless cold_start is set;
 *   2. finalizes the plan in FP64 and forms the RRH loads rho_j = sum_i C_ij pi_ij
 *      (Sec. II-B with x = pi the mass plan);
 *   3. picks j* = argmax_j rho_j (lowest index on ties), "step 5" of Algorithm 2;
 *   4. unless it is the last step, sets q_j* -= d and q_j += d / (J - 1) for j != j*, with
 *      d = delta, or d = q_j* / 2 when delta >= q_j* (a target never reaches zero).
 * The paper gives no stopping rule for the outer loop, so exactly `outer` steps run; the
 * outputs are the last step's plan and the q it used.  The targets are updated in FP64.
 * Arguments:
 *   C        [device] float I x J cost, ld_c (0 = J), 16-byte aligned rows, ld_c % 4 == 0
 *   traffic  [device] float I, lambda_i > 0
 *   prm      [host]   parameters below
 *   f, g     [device] double I and J: potentials of the last step's plan (required; g is
 *            also the warm-start buffer between steps, so its input value is ignored)
 *   q_out    [device] double J: targets used by the last solve (required; the FP64 state)
 *   rrh_load [device] double J: rho_j of the last plan, or NULL
 *   pi, pi_ld [device] float I x J plan of the last step (mass units), or NULL
 *   steps    [host]   outer entries, filled per step (below)
 * Limits: 2 <= J <= 1024 (OT_EUNSUPPORTED above), I >= 1.  Synchronises `stream`.
 * Returns OT_OK when every step converged, OT_NOT_CONVERGED when some step stopped at
 * max_iter (results valid), or the first failing step's error (later steps then carry
 * that status and did not run).
 * ------------------------------------------------------------------------------------- */
typedef struct {
    double eps;         /* > 0, absolute (every step) */
    double tol;         /* >= 0, row residual of the unit-mass plan */
    double delta;       /* >= 0, traffic moved off the most loaded RRH per step (units of lambda) */
    int32_t max_iter;   /* >= 1, Sinkhorn iterations per step */
    int32_t outer;      /* >= 1, outer steps */
    int32_t cold_start; /* != 0: every step starts from g = 0 */
    int32_t reserved;
} ot_assoc_adaptive_params;

typedef struct {
    double max_load;       /* rho_j* of this step's plan */
    double transport_cost; /* sum_ij C_ij pi_ij of this step's plan */
    double marg_err_row;   /* FP64 residuals of this step's plan (unit mass) */
    double marg_err_col;
    double err_loop;       /* residual estimate that stopped the step's loop */
    int32_t jstar;         /* most loaded RRH (-1 when the step did not complete) */
    int32_t iters;         /* Sinkhorn iterations of this step */
    int32_t converged;
    int32_t status;        /* OT_OK, OT_NOT_CONVERGED, or an error */
} ot_assoc_adaptive_step;

ot_status ot_assoc_adaptive(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* traffic,
                            int64_t I, int64_t J, const ot_assoc_adaptive_params* prm, double* f,
                            double* g, double* q_out, double* rrh_load, float* pi, int64_t pi_ld,
                            ot_assoc_adaptive_step* steps, void* stream);


/* ---------------------------------------------------------------------------------------
 * Serving (the paper has no counterpart: a service of the library around Algorithm 1).
 * Cells are registered once and keep their cost C, marginals p, q and potentials f, g
 * resident in HBM.  A request is one new time instance of a cell: new gains (caller-given,
 * or the cell's devices moved by dt on the device, for simulation), from which the rates
 * (Sec. II-A) and C = 1/(mu R) are rebuilt in place, then a solve warm-started from the
 * cell's previous g.  One persistent launch serves all cells: its CTAs form groups, each
 * group takes the next published request (the host appends while the launch runs), so
 * requests that arrive while others are on the GPU start as soon as a group is free.
 * Requests of one cell run in submission order; results depend only on the cell's data,
 * so they are the same alone and in any mix.  Admission: a cell is accepted only if its
 * resident footprint fits the server's HBM budget (OT_EBUSY otherwise).  J <= 1024.
 * ------------------------------------------------------------------------------------- */
typedef struct ot_assoc_server ot_assoc_server;

typedef struct {
    int32_t group_ctas;  /* CTAs per group (divides the SM count); 0 = a quarter of the SMs */
    int32_t max_J;       /* largest J of any cell (group scratch); 0 = 1024 */
    double idle_us;      /* a group with no work waits this long before the launch may end; 0 = 200 */
    size_t hbm_budget;   /* bytes of resident cell state; 0 = no limit */
} ot_assoc_server_config;

typedef struct {
    int64_t I;
    int32_t J;
    int32_t warm_start;  /* != 0: each request starts from the previous request's g */
    double eps, tol;     /* eps <= 0: eps = eps_rel * median(C) of the cell's first instance
                            (drifting cells); tol < 0 = 1e-6 */
    int32_t max_iter;    /* <= 0 = 2000 */
    int32_t reserved;
    double eps_rel;
    double mu, N0, W_hz; /* rates and cost (Sec. II-A, Sec. IV) */
    const float* P;      /* [host] J transmit powers */
    const float* p;      /* [host] I traffic (> 0) */
    const float* q;      /* [host] J RRH marginal (> 0, sum q = sum p) */
    /* drifting cell (all NULL: every request brings its gains) */
    const double* dev_xy;    /* [host] I x 2 device positions (m) */
    const double* dev_v;     /* [host] I x 2 velocities (m/s) */
    const float* rrh_xy;     /* [host] J x 2 RRH positions (m) */
    const float* shadow_db;  /* [host] I x J shadowing (dB), fixed per link */
    double side_m;           /* devices reflect at the walls of [0, side]^2 */
} ot_assoc_cell_desc;

typedef struct {
    uint64_t ticket;
    int32_t cell;
    int32_t status;        /* OT_OK, OT_NOT_CONVERGED, OT_EINVAL, OT_ETIMEOUT */
    int32_t iters;
    int32_t reserved;
    double transport_cost, marg_err_row, marg_err_col;
    double t_submit_us, t_start_us, t_done_us;  /* host steady clock: submitted, published, seen done */
} ot_assoc_server_result;

typedef struct {
    size_t resident_bytes;
    int32_t cells, groups, group_ctas, waiting, inflight, reserved;
    uint64_t launches;
} ot_assoc_server_stats_t;

/*
 * One time instance of a drifting cell, built the way the server rebuilds it inside its
 * kernel, for callers that solve instances one by one (ot_assoc_solve_cost) instead of
 * serving them: every device moves dt seconds along its velocity and reflects at the walls
 * of [0, side_m]^2 (dev_xy and dev_v are updated in place), its gains follow the path-loss
 * model PL = 30 dB + 35 log10(max(d, 10 m)) with the link's fixed shadowing (FP32, evaluated
 * as 2^(a - 1.75 log2 d^2): a simulation input), then the rates with every other RRH
 * interfering (Sec. II-A) and C = 1 / (mu R) (Sec. IV choice (ii)).
 * dev_xy, dev_v [device] double I x 2 (m, m/s); rrh_xy [device] float J x 2 (m);
 * shadow_db [device] float I x J (dB, row-major, ld = J); P [device] float J (W);
 * C_out [device] float I x J (ld_c, 0 = J).
 * Without eps_out the call only enqueues, and a rate that comes out non-positive or not
 * finite leaves C_ij = +inf (a link the plan cannot use).  With eps_out [host] it also sets
 * *eps_out = eps_rel * median(C), synchronises the stream, and returns OT_EINVAL when any
 * rate was invalid.  OT_EINVAL for null pointers, I or J <= 0, dt < 0, side_m <= 0,
 * N0 < 0, W_hz <= 0 or mu <= 0.
 */
ot_status ot_assoc_build_cost_mobile(ot_assoc_ctx* ctx, double* dev_xy, double* dev_v, const float* rrh_xy,
                                     const float* shadow_db, const float* P, int64_t I, int64_t J, double dt,
                                     double side_m, double N0, double W_hz, double mu, float* C_out, int64_t ld_c,
                                     double eps_rel, double* eps_out, void* stream);

/* Create a server on ctx's device (cfg NULL: the defaults above); *out [host] gets the
 * handle.  OT_EINVAL when group_ctas does not divide the SM count or out is NULL,
 * OT_EUNSUPPORTED when max_J is above 1024. */
ot_status ot_assoc_server_create(ot_assoc_ctx* ctx, const ot_assoc_server_config* cfg, ot_assoc_server** out);
/* Waits for work in flight, frees everything.  Destroy before the context. */
void ot_assoc_server_destroy(ot_assoc_server* s);
/* Register a cell (its arrays are copied); OT_EBUSY when it does not fit the budget. */
ot_status ot_assoc_server_add_cell(ot_assoc_server* s, const ot_assoc_cell_desc* d, int32_t* cell_id);
/* Submit a time instance: gains G [device] I x J (16-byte aligned rows, ld_g % 4 == 0; 0 =
 * J), or G = NULL and dt seconds of motion for a drifting cell.  G must stay valid until
 * the request's result is polled.  Returns at once (the scheduler makes progress). */
ot_status ot_assoc_server_submit(ot_assoc_server* s, int32_t cell, const float* G, int64_t ld_g, double dt,
                                 uint64_t* ticket);
/* Make progress and take up to max finished results [host array]; *n gets how many. */
ot_status ot_assoc_server_poll(ot_assoc_server* s, ot_assoc_server_result* out, int32_t max, int32_t* n);
/* Make progress until nothing is pending (results stay available to poll). */
ot_status ot_assoc_server_drain(ot_assoc_server* s, double timeout_s);
/* Device pointers of a cell's resident state (valid while the server lives; read only
 * between requests of that cell). */
ot_status ot_assoc_server_cell_state(const ot_assoc_server* s, int32_t cell, const float** C, double** f,
                                     double** g, double** rrh_load);
/* Counters of the server [host]: resident bytes, cells, groups, requests waiting and in
 * flight, persistent launches so far. */
ot_status ot_assoc_server_stats(const ot_assoc_server* s, ot_assoc_server_stats_t* out);
/* The eps a cell solves with [host]. */
ot_status ot_assoc_server_cell_eps(const ot_assoc_server* s, int32_t cell, double* eps);

#ifdef __cplusplus
}
#endif

#endif /* OT_ASSOC_H */
