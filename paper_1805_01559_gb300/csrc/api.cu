// C ABI entry points: context, scratch arena, argument validation, dispatch.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "ot_common.cuh"
#include "ot_internal.h"

namespace ota {

ot_status set_error(ot_assoc_ctx* ctx, ot_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

ot_status cuda_error(ot_assoc_ctx* ctx, cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky-free error so the context stays usable
    return set_error(ctx, e == cudaErrorMemoryAllocation ? OT_ENOMEM : OT_ECUDA, "%s: %s (%s)", what,
                     cudaGetErrorString(e), cudaGetErrorName(e));
}

void* scratch(ot_assoc_ctx* ctx, int slot, size_t bytes, ot_status* st) {
    ScratchBuf& b = ctx->slots[slot];
    bytes = std::max<size_t>(bytes, 256);
    if (b.bytes >= bytes) return b.ptr;
    const size_t others = ctx->held - b.bytes;
    size_t want = bytes + bytes / 8;  // headroom against repeated small growth
    if (ctx->budget && others + want > ctx->budget) want = bytes;
    if (ctx->budget && others + want > ctx->budget) {
        *st = set_error(ctx, OT_ENOMEM, "scratch slot %d needs %zu bytes: over the HBM budget (%zu held of %zu)",
                        slot, bytes, ctx->held, ctx->budget);
        return nullptr;
    }
    if (b.ptr) {
        cudaFree(b.ptr);
        ctx->held -= b.bytes;
        b.ptr = nullptr;
        b.bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        *st = cuda_error(ctx, e, "cudaMalloc (scratch)");
        return nullptr;
    }
    b.ptr = p;
    b.bytes = want;
    ctx->held += want;
    return p;
}

void* host_staging(ot_assoc_ctx* ctx, size_t bytes, ot_status* st) {
    if (ctx->host_pinned_bytes >= bytes) return ctx->host_pinned;
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    ctx->host_pinned = nullptr;
    ctx->host_pinned_bytes = 0;
    size_t want = std::max<size_t>(bytes, 4096);
    cudaError_t e = cudaMallocHost(&ctx->host_pinned, want);
    if (e != cudaSuccess) {
        *st = cuda_error(ctx, e, "cudaMallocHost");
        return nullptr;
    }
    ctx->host_pinned_bytes = want;
    return ctx->host_pinned;
}

cudaError_t allow_max_dynamic_smem(const void* fn, size_t need) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    const size_t limit = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (need > limit) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
}

void timing_mark(ot_assoc_ctx* ctx, int k, cudaStream_t s) {
    if (!ctx->timing) return;
    if (!ctx->ev[k] && cudaEventCreate(&ctx->ev[k]) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(ctx->ev[k], s);
}

void timing_collect(ot_assoc_ctx* ctx, int sweeps) {
    ot_assoc_timings t = {};
    if (ctx->timing && ctx->ev[0] && ctx->ev[1] && ctx->ev[2] && ctx->ev[3]) {
        float a = 0, b = 0, c = 0;
        if (cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, ctx->ev[1], ctx->ev[2]) == cudaSuccess &&
            cudaEventElapsedTime(&c, ctx->ev[2], ctx->ev[3]) == cudaSuccess) {
            t.init_ms = a;
            t.loop_ms = b;
            t.finalize_ms = c;
            t.sweeps = sweeps;
            t.valid = 1;
        } else {
            cudaGetLastError();
        }
    }
    ctx->last_timings = t;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Make a 16-byte-aligned copy of a strided FP32 matrix when it is not aligned already.
static ot_status aligned_view(ot_assoc_ctx* ctx, const float* C, int64_t ld, int64_t I, int J,
                              cudaStream_t s, const float** out, int64_t* ld_out, int slot = SLOT_COST) {
    if (ld % 4 == 0 && aligned16(C)) {
        *out = C;
        *ld_out = ld;
        return OT_OK;
    }
    ot_status st = OT_OK;
    const int64_t ldp = round_up(J, 4);
    float* dst = (float*)scratch(ctx, slot, sizeof(float) * (size_t)(I * ldp), &st);
    if (st) return st;
    cudaError_t e = cudaMemcpy2DAsync(dst, ldp * sizeof(float), C, ld * sizeof(float), J * sizeof(float),
                                      I, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "realign copy");
    *out = dst;
    *ld_out = ldp;
    return OT_OK;
}

static ot_status check_solve_args(ot_assoc_ctx* ctx, const void* C, const void* p, const void* q, int64_t I,
                                  int64_t J, int64_t ld, double eps, double tol, int32_t max_iter,
                                  const ot_assoc_result* out) {
    if (!ctx) return OT_EINVAL;
    if (!C || !p || !q || !out) return set_error(ctx, OT_EINVAL, "null input or result pointer");
    if (!out->f || !out->g) return set_error(ctx, OT_EINVAL, "out->f and out->g are required");
    if (I <= 0 || J <= 0) return set_error(ctx, OT_EINVAL, "I=%lld J=%lld must be positive", (long long)I, (long long)J);
    if (J > 8192) return set_error(ctx, OT_EUNSUPPORTED, "J=%lld above 8192", (long long)J);
    if (ld != 0 && ld < J) return set_error(ctx, OT_EINVAL, "ld=%lld < J", (long long)ld);
    if (!(eps > 0.0) || !std::isfinite(eps)) return set_error(ctx, OT_EINVAL, "eps must be finite and > 0");
    if (!(tol >= 0.0)) return set_error(ctx, OT_EINVAL, "tol must be >= 0");
    if (max_iter < 1) return set_error(ctx, OT_EINVAL, "max_iter must be >= 1");
    if (out->pi && out->pi_ld != 0 && out->pi_ld < J) return set_error(ctx, OT_EINVAL, "pi_ld < J");
    return OT_OK;
}

static ot_status finish(ot_assoc_ctx* ctx, const SolveSummary& s, ot_assoc_result* out) {
    out->transport_cost = s.cost;
    out->marg_err_row = s.err_row;
    out->marg_err_col = s.err_col;
    out->iters = s.iters;
    out->absorptions = s.absorptions;
    ot_status st;
    if (s.status == DEV_EINVAL)
        st = set_error(ctx, OT_EINVAL,
                       "invalid input: rates must be finite and > 0, marginals finite and > 0 with "
                       "sum p = sum q (1e-5 relative), warm-start g finite");
    else if (s.status == DEV_ETIMEOUT)
        st = set_error(ctx, OT_ETIMEOUT, "a device-side wait exceeded its spin limit");
    else if (s.status == OT_ENUMERIC_INTERNAL)
        st = set_error(ctx, OT_EINVAL, "numerical breakdown: a row or column of the plan lost all its mass");
    else if (s.status != DEV_OK)
        st = set_error(ctx, OT_ECUDA, "device status %d", s.status);
    else
        st = s.converged ? OT_OK : OT_NOT_CONVERGED;
    out->status = st;
    if (st == OT_OK || st == OT_NOT_CONVERGED) ctx->err.clear();
    return st;
}

using DeviceGuard = DeviceGuardLite;

}  // namespace ota

using namespace ota;

extern "C" {

int ot_assoc_version(void) { return 100; }

const char* ot_assoc_status_string(int status) {
    switch (status) {
        case OT_OK: return "OT_OK";
        case OT_NOT_CONVERGED: return "OT_NOT_CONVERGED";
        case OT_EINVAL: return "OT_EINVAL";
        case OT_ENOMEM: return "OT_ENOMEM";
        case OT_ECUDA: return "OT_ECUDA";
        case OT_ETIMEOUT: return "OT_ETIMEOUT";
        case OT_EBUSY: return "OT_EBUSY";
        case OT_EUNSUPPORTED: return "OT_EUNSUPPORTED";
        default: return "OT_UNKNOWN";
    }
}

ot_status ot_assoc_create(ot_assoc_ctx** out, int device, size_t hbm_budget_bytes) {
    if (!out) return OT_EINVAL;
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return OT_ECUDA;
    }
    if (device < 0 || device >= n) return OT_EINVAL;
    DeviceGuard g(device);
    ot_assoc_ctx* ctx = new ot_assoc_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete ctx;
        cudaGetLastError();
        return OT_ECUDA;
    }
    *out = ctx;
    return OT_OK;
}

void ot_assoc_destroy(ot_assoc_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    // asynchronous solves still in flight use the scratch freed below: let them finish
    for (int i = 0; i < ot_assoc_ctx::kAsyncSlots; ++i)
        if (ctx->async_ticket[i] && ctx->async_ev[i][0]) cudaEventSynchronize(ctx->async_ev[i][0]);
    for (auto& b : ctx->slots)
        if (b.ptr) cudaFree(b.ptr);
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    if (ctx->async_sum) cudaFreeHost(ctx->async_sum);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    for (auto& row : ctx->async_ev)
        for (auto& e : row)
            if (e) cudaEventDestroy(e);
    delete ctx;
}

void ot_assoc_enable_timing(ot_assoc_ctx* ctx, int on) {
    if (ctx) ctx->timing = on != 0;
}

ot_status ot_assoc_last_timings(const ot_assoc_ctx* ctx, ot_assoc_timings* out) {
    if (!ctx || !out) return OT_EINVAL;
    *out = ctx->last_timings;
    return OT_OK;
}

uint64_t ot_assoc_launch_count(const ot_assoc_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* ot_assoc_last_error(const ot_assoc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t ot_assoc_scratch_bytes(const ot_assoc_ctx* ctx) { return ctx ? ctx->held : 0; }

void ot_assoc_set_spin_limit(ot_assoc_ctx* ctx, int64_t polls) {
    if (ctx) ctx->spin_limit = polls >= 1 ? polls : (1LL << 24);
}

ot_status ot_assoc_build_cost_from_gains(ot_assoc_ctx* ctx, const float* G, int64_t ld_g, const float* P,
                                         int64_t I, int64_t J, double N0, double W_hz, double mu, float* R_out,
                                         int64_t ld_r, float* C_out, int64_t ld_c, double eps_rel, double* eps_out,
                                         void* stream) {
    if (!ctx) return OT_EINVAL;
    if (!G || !P || !C_out) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0) return set_error(ctx, OT_EINVAL, "I and J must be positive");
    if (J > 8192) return set_error(ctx, OT_EUNSUPPORTED, "J above 8192");
    if (ld_g == 0) ld_g = J;
    if (ld_r == 0) ld_r = J;
    if (ld_c == 0) ld_c = J;
    if (ld_g < J || ld_r < J || ld_c < J) return set_error(ctx, OT_EINVAL, "leading dimension < J");
    if (!(N0 >= 0.0) || !(W_hz > 0.0)) return set_error(ctx, OT_EINVAL, "need N0 >= 0 and W_hz > 0");
    if (!(mu > 0.0) || !std::isfinite(mu)) return set_error(ctx, OT_EINVAL, "mu must be finite and > 0");
    if (eps_out && !(eps_rel > 0.0)) return set_error(ctx, OT_EINVAL, "eps_rel must be > 0");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    ot_status st = aligned_view(ctx, G, ld_g, I, (int)J, s, &G, &ld_g, SLOT_ALIGN);
    if (st) return st;
    char* state = (char*)scratch(ctx, SLOT_MISC, 256, &st);
    if (st) return st;
    unsigned long long* bad = (unsigned long long*)state;
    double* med = (double*)(state + 64);
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "memset");
    st = launch_rates(ctx, G, ld_g, P, I, (int)J, N0, W_hz, R_out, ld_r, s, mu, C_out, ld_c, bad);
    if (st) return st;
    if (!eps_out) return OT_OK;
    st = launch_median(ctx, C_out, I, J, ld_c, med, s);
    if (st) return st;
    struct {
        unsigned long long bad;
        double med;
    }* h = (decltype(h))host_staging(ctx, 64, &st);
    if (st) return st;
    e = cudaMemcpyAsync(&h->bad, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h->med, med, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "build_cost_from_gains");
    if (h->bad) return set_error(ctx, OT_EINVAL, "%llu rate entries are not finite and > 0", h->bad);
    *eps_out = eps_rel * h->med;
    return OT_OK;
}

ot_status ot_assoc_build_rates(ot_assoc_ctx* ctx, const float* G, int64_t ld_g, const float* P, int64_t I,
                               int64_t J, double N0, double W_hz, float* R_out, int64_t ld_r, void* stream) {
    if (!ctx) return OT_EINVAL;
    if (!G || !P || !R_out) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0) return set_error(ctx, OT_EINVAL, "I and J must be positive");
    if (J > 8192) return set_error(ctx, OT_EUNSUPPORTED, "J above 8192");
    if (ld_g == 0) ld_g = J;
    if (ld_r == 0) ld_r = J;
    if (ld_g < J || ld_r < J) return set_error(ctx, OT_EINVAL, "leading dimension < J");
    if (!(N0 >= 0.0) || !(W_hz > 0.0)) return set_error(ctx, OT_EINVAL, "need N0 >= 0 and W_hz > 0");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    ot_status st = aligned_view(ctx, G, ld_g, I, (int)J, s, &G, &ld_g, SLOT_ALIGN);
    if (st) return st;
    return launch_rates(ctx, G, ld_g, P, I, (int)J, N0, W_hz, R_out, ld_r, s);
}

ot_status ot_assoc_build_cost(ot_assoc_ctx* ctx, const float* R, int64_t ld_r, int64_t I, int64_t J, double mu,
                              float* C_out, int64_t ld_c, double eps_rel, double* eps_out, void* stream) {
    if (!ctx) return OT_EINVAL;
    if (!R || !C_out) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0) return set_error(ctx, OT_EINVAL, "I and J must be positive");
    if (J > (1 << 30)) return set_error(ctx, OT_EUNSUPPORTED, "J too large");
    if (ld_r == 0) ld_r = J;
    if (ld_c == 0) ld_c = J;
    if (ld_r < J || ld_c < J) return set_error(ctx, OT_EINVAL, "leading dimension < J");
    if (!(mu > 0.0) || !std::isfinite(mu)) return set_error(ctx, OT_EINVAL, "mu must be finite and > 0");
    if (eps_out && !(eps_rel > 0.0)) return set_error(ctx, OT_EINVAL, "eps_rel must be > 0");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    ot_status st = OT_OK;
    char* state = (char*)scratch(ctx, SLOT_MISC, 256, &st);
    if (st) return st;
    unsigned long long* bad = (unsigned long long*)state;
    double* med = (double*)(state + 64);
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "memset");
    st = launch_cost(ctx, R, ld_r, I, (int)J, mu, C_out, ld_c, false, bad, s);
    if (st) return st;
    if (!eps_out) return OT_OK;
    st = launch_median(ctx, C_out, I, J, ld_c, med, s);
    if (st) return st;
    struct {
        unsigned long long bad;
        double med;
    }* h = (decltype(h))host_staging(ctx, 64, &st);
    if (st) return st;
    e = cudaMemcpyAsync(&h->bad, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h->med, med, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "build_cost");
    if (h->bad) return set_error(ctx, OT_EINVAL, "%llu rate entries are not finite and > 0", h->bad);
    *eps_out = eps_rel * h->med;
    return OT_OK;
}

ot_status ot_assoc_median_f32(ot_assoc_ctx* ctx, const float* x, int64_t n, double* median_out, void* stream) {
    if (!ctx) return OT_EINVAL;
    if (!x || !median_out || n <= 0) return set_error(ctx, OT_EINVAL, "bad median arguments");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    ot_status st = OT_OK;
    char* state = (char*)scratch(ctx, SLOT_MISC, 256, &st);
    if (st) return st;
    double* med = (double*)(state + 64);
    st = launch_median(ctx, x, 1, n, n, med, s);
    if (st) return st;
    double* h = (double*)host_staging(ctx, 64, &st);
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(h, med, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "median");
    *median_out = *h;
    return OT_OK;
}

ot_status ot_assoc_maxsinr(ot_assoc_ctx* ctx, const float* R, int64_t ld_r, const float* traffic, int64_t I,
                           int64_t J, double mu, int32_t* assoc_out, double* Lambda_out, double* total_load_out,
                           void* stream) {
    if (!ctx) return OT_EINVAL;
    if (!R || !traffic) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0) return set_error(ctx, OT_EINVAL, "I and J must be positive");
    if (J > 8192) return set_error(ctx, OT_EUNSUPPORTED, "J above 8192");
    if (ld_r == 0) ld_r = J;
    if (ld_r < J) return set_error(ctx, OT_EINVAL, "leading dimension < J");
    if (!(mu > 0.0)) return set_error(ctx, OT_EINVAL, "mu must be > 0");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    ot_status st = OT_OK;
    char* state = (char*)scratch(ctx, SLOT_MISC, 256, &st);
    if (st) return st;
    double* tot = (double*)(state + 128);
    st = aligned_view(ctx, R, ld_r, I, (int)J, s, &R, &ld_r, SLOT_ALIGN);
    if (st) return st;
    st = launch_maxsinr(ctx, R, ld_r, traffic, I, (int)J, mu, assoc_out, Lambda_out, tot, s);
    if (st) return st;
    if (total_load_out) {
        double* h = (double*)host_staging(ctx, 64, &st);
        if (st) return st;
        cudaError_t e = cudaMemcpyAsync(h, tot, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "maxsinr");
        *total_load_out = *h;
    }
    return OT_OK;
}

ot_status ot_assoc_solve_cost(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* p, const float* q,
                              int64_t I, int64_t J, double eps, double tol, int32_t max_iter, int32_t warm_start,
                              ot_assoc_result* out, void* stream) {
    ot_status st = check_solve_args(ctx, C, p, q, I, J, ld_c, eps, tol, max_iter, out);
    if (st) return st;
    if (ld_c == 0) ld_c = J;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    SolveArgs a;
    st = aligned_view(ctx, C, ld_c, I, (int)J, s, &a.C, &a.ld);
    if (st) return st;
    a.p = p;
    a.q = q;
    a.I = I;
    a.J = (int)J;
    a.eps = eps;
    a.tol = tol;
    a.max_iter = max_iter;
    a.warm_start = warm_start;
    a.out = out;
    a.stream = s;
    SolveSummary sum;
    st = launch_solve_f32(ctx, a, &sum);
    if (st) return st;
    return finish(ctx, sum, out);
}

ot_status ot_assoc_solve_euclid(ot_assoc_ctx* ctx, const float* dev_xy, const float* rrh_xy, const float* p,
                                const float* q, int64_t I, int64_t J, double eps, double tol, int32_t max_iter,
                                int32_t warm_start, ot_assoc_result* out, void* stream) {
    if (!ctx) return OT_EINVAL;
    if (!dev_xy || !rrh_xy) return set_error(ctx, OT_EINVAL, "null coordinates");
    if (((uintptr_t)dev_xy & 7u) || ((uintptr_t)rrh_xy & 7u))
        return set_error(ctx, OT_EINVAL, "coordinates must be 8-byte aligned (x, y float pairs)");
    ot_status st = check_solve_args(ctx, dev_xy, p, q, I, J, 0, eps, tol, max_iter, out);
    if (st) return st;
    DeviceGuard g(ctx->device);
    SolveArgs a;
    a.C = nullptr;
    a.ld = round_up(J, 4);
    a.p = p;
    a.q = q;
    a.I = I;
    a.J = (int)J;
    a.eps = eps;
    a.tol = tol;
    a.max_iter = max_iter;
    a.warm_start = warm_start;
    a.out = out;
    a.stream = (cudaStream_t)stream;
    a.dev_xy = (const float2*)dev_xy;
    a.rrh_xy = (const float2*)rrh_xy;
    SolveSummary sum;
    st = launch_solve_f32(ctx, a, &sum);
    if (st) return st;
    return finish(ctx, sum, out);
}

ot_status ot_assoc_solve_cost_multi(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* p,
                                    const float* q, int64_t I, int64_t J, int32_t n, const double* eps,
                                    const double* tol, int32_t max_iter, ot_assoc_result* outs, void* stream) {
    if (!ctx) return OT_EINVAL;
    if (!eps || !tol || !outs) return set_error(ctx, OT_EINVAL, "null eps, tol or result array");
    if (n < 1 || n > 3) return set_error(ctx, OT_EUNSUPPORTED, "n=%d solves: 1 to 3 share one launch", n);
    for (int k = 0; k < n; ++k) {
        ot_status st = check_solve_args(ctx, C, p, q, I, J, ld_c, eps[k], tol[k], max_iter, &outs[k]);
        if (st) return st;
    }
    if (J > 4096) return set_error(ctx, OT_EUNSUPPORTED, "J=%lld above 4096 (multi-solve)", (long long)J);
    if (ld_c == 0) ld_c = J;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    SolveArgs a;
    ot_status st = aligned_view(ctx, C, ld_c, I, (int)J, s, &a.C, &a.ld);
    if (st) return st;
    a.p = p;
    a.q = q;
    a.I = I;
    a.J = (int)J;
    a.eps = eps[0];
    a.tol = tol[0];
    a.max_iter = max_iter;
    a.warm_start = 0;
    a.out = &outs[0];
    a.stream = s;
    ot_assoc_result* ptrs[3] = {&outs[0], n > 1 ? &outs[1] : nullptr, n > 2 ? &outs[2] : nullptr};
    SolveSummary sum[3];
    st = launch_solve_multi(ctx, a, n, eps, tol, ptrs, sum);
    if (st) return st;
    ot_status worst = OT_OK;
    for (int k = 0; k < n; ++k) {
        const ot_status sk = finish(ctx, sum[k], &outs[k]);
        if (sk < 0 && worst >= 0) worst = sk;
        else if (sk == OT_NOT_CONVERGED && worst == OT_OK) worst = OT_NOT_CONVERGED;
    }
    return worst;
}

ot_status ot_assoc_solve_cost_async(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* p,
                                    const float* q, int64_t I, int64_t J, double eps, double tol, int32_t max_iter,
                                    int32_t warm_start, const ot_assoc_result* out, uint64_t* ticket,
                                    void* stream) {
    ot_status st = check_solve_args(ctx, C, p, q, I, J, ld_c, eps, tol, max_iter, out);
    if (st) return st;
    if (!ticket) return set_error(ctx, OT_EINVAL, "null ticket pointer");
    if (ld_c == 0) ld_c = J;
    DeviceGuard g(ctx->device);
    if (!ctx->async_sum) {
        cudaError_t e = cudaMallocHost(&ctx->async_sum, sizeof(SolveSummary) * ot_assoc_ctx::kAsyncSlots);
        if (e != cudaSuccess) {
            ctx->async_sum = nullptr;
            return cuda_error(ctx, e, "cudaMallocHost (async summaries)");
        }
    }
    int k = -1;
    for (int i = 0; i < ot_assoc_ctx::kAsyncSlots; ++i)
        if (ctx->async_ticket[i] == 0) {
            k = i;
            break;
        }
    if (k < 0) return set_error(ctx, OT_EBUSY, "%d asynchronous solves in flight: wait for one first",
                                ot_assoc_ctx::kAsyncSlots);
    for (auto& e : ctx->async_ev[k])
        if (!e && cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, OT_ECUDA, "cudaEventCreate");
        }
    cudaStream_t s = (cudaStream_t)stream;
    SolveArgs a;
    st = aligned_view(ctx, C, ld_c, I, (int)J, s, &a.C, &a.ld);
    if (st) return st;
    a.p = p;
    a.q = q;
    a.I = I;
    a.J = (int)J;
    a.eps = eps;
    a.tol = tol;
    a.max_iter = max_iter;
    a.warm_start = warm_start;
    a.out = const_cast<ot_assoc_result*>(out);
    a.stream = s;
    SolveSummary* dest = (SolveSummary*)ctx->async_sum + k;
    st = enqueue_solve_f32(ctx, a, dest, ctx->timing ? ctx->async_ev[k][1] : nullptr,
                           ctx->timing ? ctx->async_ev[k][2] : nullptr);
    if (st) return st;
    cudaError_t e = cudaEventRecord(ctx->async_ev[k][0], s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "event record");
    ctx->async_ticket[k] = ctx->next_ticket++;
    *ticket = ctx->async_ticket[k];
    return OT_OK;
}

ot_status ot_assoc_wait(ot_assoc_ctx* ctx, uint64_t ticket, ot_assoc_result* out) {
    if (!ctx) return OT_EINVAL;
    if (!out) return set_error(ctx, OT_EINVAL, "null result pointer");
    int k = -1;
    for (int i = 0; i < ot_assoc_ctx::kAsyncSlots; ++i)
        if (ticket != 0 && ctx->async_ticket[i] == ticket) {
            k = i;
            break;
        }
    if (k < 0) return set_error(ctx, OT_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaEventSynchronize(ctx->async_ev[k][0]);
    ctx->async_ticket[k] = 0;
    if (e != cudaSuccess) return cuda_error(ctx, e, "asynchronous solve");
    const SolveSummary sum = ((const SolveSummary*)ctx->async_sum)[k];
    ctx->last_timings = ot_assoc_timings{};
    float ms = 0.f;
    if (ctx->timing && cudaEventElapsedTime(&ms, ctx->async_ev[k][1], ctx->async_ev[k][2]) == cudaSuccess) {
        ctx->last_timings.loop_ms = ms;
        ctx->last_timings.sweeps = sum.iters;
        ctx->last_timings.valid = 1;
    } else {
        cudaGetLastError();
    }
    return finish(ctx, sum, out);
}

ot_status ot_assoc_solve(ot_assoc_ctx* ctx, const float* R, int64_t ld_r, const float* traffic,
                         const float* rrh_marginal, int64_t I, int64_t J, double mu, double eps, double tol,
                         int32_t max_iter, int32_t warm_start, ot_assoc_result* out, void* stream) {
    ot_status st = check_solve_args(ctx, R, traffic, rrh_marginal, I, J, ld_r, eps, tol, max_iter, out);
    if (st) return st;
    if (!(mu > 0.0) || !std::isfinite(mu)) return set_error(ctx, OT_EINVAL, "mu must be finite and > 0");
    if (ld_r == 0) ld_r = J;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ldc = round_up(J, 4);
    float* C = (float*)scratch(ctx, SLOT_COST, sizeof(float) * (size_t)(I * ldc), &st);
    if (st) return st;
    char* state = (char*)scratch(ctx, SLOT_MISC, 256, &st);
    if (st) return st;
    unsigned long long* bad = (unsigned long long*)state;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "memset");
    st = launch_cost(ctx, R, ld_r, I, (int)J, mu, C, ldc, true, bad, s);
    if (st) return st;
    SolveArgs a;
    a.C = C;
    a.ld = ldc;
    a.p = traffic;
    a.q = rrh_marginal;
    a.I = I;
    a.J = (int)J;
    a.eps = eps;
    a.tol = tol;
    a.max_iter = max_iter;
    a.warm_start = warm_start;
    a.out = out;
    a.stream = s;
    a.input_bad = bad;
    SolveSummary sum;
    st = launch_solve_f32(ctx, a, &sum);
    if (st) return st;
    return finish(ctx, sum, out);
}

ot_status ot_assoc_solve_f64(ot_assoc_ctx* ctx, const double* C, int64_t ld_c, const double* p, const double* q,
                             int64_t I, int64_t J, double eps, double tol, int32_t max_iter, int32_t warm_start,
                             ot_assoc_result* out, void* stream) {
    ot_status st = check_solve_args(ctx, C, p, q, I, J, ld_c, eps, tol, max_iter, out);
    if (st) return st;
    if (ld_c == 0) ld_c = J;
    DeviceGuard g(ctx->device);
    SolveArgs64 a;
    a.C = C;
    a.ld = ld_c;
    a.p = p;
    a.q = q;
    a.I = I;
    a.J = (int)J;
    a.eps = eps;
    a.tol = tol;
    a.max_iter = max_iter;
    a.warm_start = warm_start;
    a.out = out;
    a.stream = (cudaStream_t)stream;
    SolveSummary sum;
    st = launch_solve_f64(ctx, a, &sum);
    if (st) return st;
    return finish(ctx, sum, out);
}

ot_status ot_assoc_solve_lowp(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* p, const float* q,
                              int64_t I, int64_t J, double eps, double tol, int32_t max_iter, int32_t warm_start,
                              int32_t format, double absorb_log2, ot_assoc_result* out, void* stream) {
    ot_status st = check_solve_args(ctx, C, p, q, I, J, ld_c, eps, tol, max_iter, out);
    if (st) return st;
    if (format != OT_KERNEL_F32 && format != OT_KERNEL_BF16 && format != OT_KERNEL_F16)
        return set_error(ctx, OT_EINVAL, "unknown kernel format %d", format);
    if (ld_c == 0) ld_c = J;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    SolveArgs a;
    st = aligned_view(ctx, C, ld_c, I, (int)J, s, &a.C, &a.ld);
    if (st) return st;
    a.p = p;
    a.q = q;
    a.I = I;
    a.J = (int)J;
    a.eps = eps;
    a.tol = tol;
    a.max_iter = max_iter;
    a.warm_start = warm_start;
    a.out = out;
    a.stream = s;
    SolveSummary sum;
    st = launch_solve_lowp(ctx, a, format, absorb_log2, &sum);
    if (st) return st;
    return finish(ctx, sum, out);
}

ot_status ot_assoc_batch_create(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int32_t n, int32_t flags,
                                ot_assoc_batch** out) {
    if (!ctx) return OT_EINVAL;
    if (!out) return set_error(ctx, OT_EINVAL, "null output pointer");
    DeviceGuard g(ctx->device);
    return batch_create(ctx, inst, n, flags, out);
}

ot_status ot_assoc_batch_set(ot_assoc_batch* b, int32_t k, const ot_assoc_instance* inst) {
    if (!b) return OT_EINVAL;
    return batch_set(b, k, inst);
}

ot_status ot_assoc_batch_launch(ot_assoc_batch* b, void* stream) {
    if (!b) return OT_EINVAL;
    return batch_launch(b, (cudaStream_t)stream);
}

ot_status ot_assoc_batch_wait(ot_assoc_batch* b, void* stream, ot_assoc_instance_result* res) {
    if (!b) return OT_EINVAL;
    return batch_wait(b, (cudaStream_t)stream, res);
}

void ot_assoc_batch_destroy(ot_assoc_batch* b) { batch_destroy(b); }

ot_status ot_assoc_solve_batched(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int32_t n,
                                 ot_assoc_instance_result* res, void* stream) {
    if (!ctx) return OT_EINVAL;
    if (!res) return set_error(ctx, OT_EINVAL, "null result array");
    DeviceGuard g(ctx->device);
    ot_assoc_batch* b = nullptr;
    ot_status st = batch_create(ctx, inst, n, OT_BATCH_NO_GRAPH, &b);
    if (st) return st;
    st = batch_launch(b, (cudaStream_t)stream);
    if (!st) st = batch_wait(b, (cudaStream_t)stream, res);
    batch_destroy(b);
    return st;
}

ot_status ot_assoc_autotune(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int32_t n, int32_t iters,
                            void* stream) {
    if (!ctx) return OT_EINVAL;
    if (!inst || n <= 0) return set_error(ctx, OT_EINVAL, "empty tuning set");
    DeviceGuard g(ctx->device);
    return batch_autotune(ctx, inst, n, iters, (cudaStream_t)stream);
}

ot_status ot_assoc_tuning_get(const ot_assoc_ctx* ctx, int32_t bucket, int32_t* gsize, int32_t* stage_bytes,
                              double* rate) {
    if (!ctx || bucket < 0 || bucket >= TUNE_BUCKETS) return OT_EINVAL;
    if (gsize) *gsize = ctx->tune[bucket].gsize;
    if (stage_bytes) *stage_bytes = ctx->tune[bucket].stage;
    if (rate) *rate = ctx->tune[bucket].rate;
    return OT_OK;
}

ot_status ot_assoc_tuning_set(ot_assoc_ctx* ctx, int32_t bucket, int32_t gsize, int32_t stage_bytes) {
    if (!ctx) return OT_EINVAL;
    if (bucket < 0 || bucket >= TUNE_BUCKETS) return set_error(ctx, OT_EINVAL, "bucket out of range");
    if (gsize < 0 || (gsize > 0 && ctx->num_sms % gsize != 0))
        return set_error(ctx, OT_EINVAL, "group size must divide the SM count (%d)", ctx->num_sms);
    if (stage_bytes < 0) return set_error(ctx, OT_EINVAL, "stage size must be >= 0");
    ctx->tune[bucket].gsize = gsize;
    ctx->tune[bucket].stage = stage_bytes;
    ctx->tune[bucket].rate = 0.0;
    return OT_OK;
}

int32_t ot_assoc_bucket(int64_t I, int32_t J) { return batch_bucket(I, J); }

}  // extern "C"
