// Measurement helper: the device's FP32 exp2 (SFU) throughput, the ceiling of the per-cell
// exponential of Algorithm 1 (one ex2 a cell and sweep in every solver here).
#include <cuda_runtime.h>

#include "ot_assoc.h"
#include "ot_common.cuh"
#include "ot_internal.h"

namespace ota {
namespace {

constexpr int PR_CHAINS = 8;

// Eight independent chains a thread, x <- 2^(0.25 - 0.75 x): each step one FMA and one ex2,
// values in (0, 2); the sum keeps the chains live.
__global__ void __launch_bounds__(256) k_ex2_rate(int iters, float* sink) {
    float x[PR_CHAINS];
#pragma unroll
    for (int k = 0; k < PR_CHAINS; ++k) x[k] = 0.01f * (float)((threadIdx.x + k) & 63);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < PR_CHAINS; ++k) x[k] = ex2(fmaf(x[k], -0.75f, 0.25f));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PR_CHAINS; ++k) s += x[k];
    if (s == 12345.0f) sink[threadIdx.x] = s;  // never true: keeps the chains
}

}  // namespace
}  // namespace ota

using namespace ota;

extern "C" {

ot_status ot_assoc_measure_ex2_rate(ot_assoc_ctx* ctx, double* ex2_per_s, void* stream) {
    if (!ctx) return OT_EINVAL;
    DeviceGuardLite guard(ctx->device);
    if (!ex2_per_s) return set_error(ctx, OT_EINVAL, "null pointer");
    ot_status st = OT_OK;
    float* sink = (float*)scratch(ctx, SLOT_MISC, 256 * sizeof(float), &st);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = 8 * ctx->num_sms, iters = 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {  // the first launch warms up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) k_ex2_rate<<<blocks, 256, 0, s>>>(iters, sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ctx->launches += 4;
    if (e != cudaSuccess) return cuda_error(ctx, e, "ex2 rate");
    *ex2_per_s = (double)blocks * 256.0 * iters * PR_CHAINS / (best / 1e3);
    return OT_OK;
}

}  // extern "C"
