// Host-side internals of the library (context, scratch arena, launch helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ot_assoc.h"

// Internal status for a numerical breakdown reported by the device.
#define OT_ENUMERIC_INTERNAL (-7)

namespace ota {

enum ScratchSlot {
    SLOT_COST = 0,     // padded FP32 cost (solve from R, or realigned caller C)
    SLOT_F,            // 2 x I doubles: row potentials (double-buffered)
    SLOT_G,            // Jp doubles: column potentials
    SLOT_COLPART,      // [nCTA][Jp] float2 partials
    SLOT_ERRPART,      // [nCTA] doubles (x4)
    SLOT_FINPART,      // [nCTA][Jp] double2 finalize partials
    SLOT_STATE,        // small device structs
    SLOT_SELECT,       // median select workspace
    SLOT_MISC,         // maxSINR partials etc.
    SLOT_KT,           // stored kernel (low precision form)
    SLOT_SCAL,         // scaling vectors u, v, drift references (low precision form)
    SLOT_ALIGN,        // 16-byte-aligned copies of unaligned caller inputs (G, R)
    SLOT_TUNE,         // autotuner outputs (potentials of the timed runs)
    SLOT_SHARD,        // row-sharded sweeps: per-block column partials
    SLOT_ROWTOT,       // rates: per-row totals N0 + sum_k P_k G_ik (FP32 pairs)
    SLOT_COUNT
};

// Batched solver tuning: group size (schedule) and stage size (tile) per instance size
// bucket (cells class x J class).
static constexpr int TUNE_BUCKETS = 15;
struct TuneEntry {
    int gsize = 0;   // CTAs per instance group (0 = not tuned: use the default)
    int stage = 0;   // bytes of C per bulk copy (target)
    double rate = 0; // measured cells * iterations / s of the chosen pair
};

struct ScratchBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace ota

struct ot_assoc_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;
    size_t held = 0;
    long long spin_limit = 1LL << 24;
    std::string err;
    ota::ScratchBuf slots[ota::SLOT_COUNT];
    void* host_pinned = nullptr;   // small pinned staging area for result readback
    size_t host_pinned_bytes = 0;
    unsigned long long launches = 0;  // kernels launched by this context
    bool timing = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    ot_assoc_timings last_timings = {};
    ota::TuneEntry tune[ota::TUNE_BUCKETS];
    // asynchronous solves: pinned summary slots, their completion and kernel events, tickets
    static constexpr int kAsyncSlots = 16;
    void* async_sum = nullptr;                       // pinned SolveSummary[kAsyncSlots]
    cudaEvent_t async_ev[kAsyncSlots][3] = {};       // done, kernel start, kernel end
    unsigned long long async_ticket[kAsyncSlots] = {};  // 0 = free
    unsigned long long next_ticket = 1;
};

namespace ota {

ot_status set_error(ot_assoc_ctx* ctx, ot_status st, const char* fmt, ...);
ot_status cuda_error(ot_assoc_ctx* ctx, cudaError_t e, const char* what);
// Return a device buffer of at least `bytes` for `slot`, growing it within the budget.
void* scratch(ot_assoc_ctx* ctx, int slot, size_t bytes, ot_status* st);
void* host_staging(ot_assoc_ctx* ctx, size_t bytes, ot_status* st);

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Phase events of a solve (no-ops unless timing is enabled).
void timing_mark(ot_assoc_ctx* ctx, int k, cudaStream_t s);
// After the solve's stream has synchronised: turn the marks into last_timings.
void timing_collect(ot_assoc_ctx* ctx, int sweeps);

// ---- launchers implemented in the .cu files -------------------------------------------------
struct SolveSummary {   // device-written, copied back once per solve
    double err_row;     // FP64 row residual of the returned plan (unit mass)
    double err_col;     // FP64 column residual (unit mass)
    double cost;        // transport cost in the caller's mass units
    double err_loop;    // residual estimate that stopped the loop (FP32 cells)
    int iters;
    int converged;
    int status;         // device status word (DEV_*)
    int absorptions;
};

struct SolveArgs {
    const float* C;   // FP32 cost, 16-byte aligned rows (ld % 4 == 0)
    int64_t ld;
    const float* p;
    const float* q;
    int64_t I;
    int J;
    double eps;
    double tol;
    int max_iter;
    int warm_start;
    ot_assoc_result* out;
    cudaStream_t stream;
    const unsigned long long* input_bad = nullptr;  // nonzero count => invalid input (checked on device)
    const float2* dev_xy = nullptr;  // Euclidean cost on the fly: device and RRH coordinates (C unused)
    const float2* rrh_xy = nullptr;
};

// FP32 log-domain solve (Algorithm 1).  Fills `sum_host` (synchronises).
ot_status launch_solve_f32(ot_assoc_ctx* ctx, const SolveArgs& a, SolveSummary* sum_host);
// Up to three solves on one cost matrix (same p, q; eps[k], tol[k]) in one launch.
ot_status launch_solve_multi(ot_assoc_ctx* ctx, const SolveArgs& a, int n, const double* eps, const double* tol,
                             ot_assoc_result* const* outs, SolveSummary* sum_host);
// The same solve enqueued only: the summary lands in `dest` (pinned host memory) when the
// stream gets there; kev0/kev1 (optional) are recorded around the persistent kernel.
ot_status enqueue_solve_f32(ot_assoc_ctx* ctx, const SolveArgs& a, SolveSummary* dest, cudaEvent_t kev0,
                            cudaEvent_t kev1);

struct SolveArgs64 {
    const double* C;
    int64_t ld;
    const double* p;
    const double* q;
    int64_t I;
    int J;
    double eps;
    double tol;
    int max_iter;
    int warm_start;
    ot_assoc_result* out;
    cudaStream_t stream;
};
ot_status launch_solve_f64(ot_assoc_ctx* ctx, const SolveArgs64& a, SolveSummary* sum_host);

ot_status launch_solve_lowp(ot_assoc_ctx* ctx, const SolveArgs& a, int format, double absorb_log2,
                            SolveSummary* sum_host);
// Pieces of the FP32 solver the stored-kernel form builds on (k_sinkhorn.cu).
ot_status f32_first_iteration(ot_assoc_ctx* ctx, const SolveArgs& a, float2* F_out, double* G_out, int* status);
ot_status f32_finalize_on(ot_assoc_ctx* ctx, const SolveArgs& a, const float2* F_in, const double* G_in, int iters,
                          double err, int converged, SolveSummary* sum_host);

// Rates into R (may be null when C is given); with C non-null also C = (1/mu)/R in the same
// pass, counting rates that are not finite and > 0 into *bad_dev.
ot_status launch_rates(ot_assoc_ctx* ctx, const float* G, int64_t ld_g, const float* P, int64_t I,
                       int J, double N0, double W, float* R, int64_t ld_r, cudaStream_t s, double mu = 1.0,
                       float* C = nullptr, int64_t ld_c = 0, unsigned long long* bad_dev = nullptr);
// C = 1/(mu R); pads columns [J, ld_c) with +inf when pad_inf; counts invalid R into *bad_dev.
ot_status launch_cost(ot_assoc_ctx* ctx, const float* R, int64_t ld_r, int64_t I, int J, double mu,
                      float* C, int64_t ld_c, bool pad_inf, unsigned long long* bad_dev,
                      cudaStream_t s);
// Median of the first n entries of a strided matrix view (rows x cols, ld) of floats; writes
// the result (double) to *out_dev.  Requires no NaN.
ot_status launch_median(ot_assoc_ctx* ctx, const float* x, int64_t rows, int64_t cols, int64_t ld,
                        double* out_dev, cudaStream_t s);
// Batched ragged solve (k_batch.cu).
int batch_bucket(int64_t I, int J);
ot_status batch_create(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int n, int flags, ot_assoc_batch** out,
                       int forced_gsize = 0, int forced_stage = 0);
ot_status batch_set(ot_assoc_batch* b, int k, const ot_assoc_instance* a);
ot_status batch_launch(ot_assoc_batch* b, cudaStream_t s);
ot_status batch_wait(ot_assoc_batch* b, cudaStream_t s, ot_assoc_instance_result* res);
void batch_destroy(ot_assoc_batch* b);
ot_status batch_autotune(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int n, int iters, cudaStream_t s);

// Make `dev` current for the lifetime of the guard (restores the previous device).
struct DeviceGuardLite {
    int prev = -1;
    explicit DeviceGuardLite(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuardLite() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Allow `fn` the largest dynamic shared memory a block may opt in to on the current device
// (the opt-in limit minus the kernel's static shared memory); fails when `need` exceeds it.
// The value set is the same for every call, so one launch plan never lowers the limit
// another plan (or a captured graph) relies on.
cudaError_t allow_max_dynamic_smem(const void* fn, size_t need);

ot_status launch_maxsinr(ot_assoc_ctx* ctx, const float* R, int64_t ld_r, const float* lam,
                         int64_t I, int J, double mu, int32_t* assoc, double* Lambda,
                         double* total_dev, cudaStream_t s);

}  // namespace ota
