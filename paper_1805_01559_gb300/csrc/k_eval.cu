// Cost and evaluation kernels around the association policies of Sec. IV:
//   * the Euclidean cost C_ij = ||x_i - x_j|| (Sec. IV, cost choice (i));
//   * the average job completion time of an association (Sec. II-B): with x the plan in
//     mass units (x_ij = lambda_i pi_ij) and C the load cost 1/(mu R_ij),
//       rho_j = sum_i C_ij x_ij,   T = (1/I) sum_i sum_j pi_ij C_ij / (1 - rho_j)
//             = (1/I) sum_j u_j / (1 - rho_j)   with u_j = sum_i C_ij pi_ij,
//     so one pass over the matrix gives both column sums.  An RRH with rho_j >= 1 that
//     carries traffic makes T infinite (unstable queue).
// The plan is either given by potentials (pi from Eq. (5)'s minimiser on a plan cost that
// may differ from the load cost, e.g. the Euclidean one) or by a hard association.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ot_common.cuh"
#include "ot_internal.h"

namespace ota {

static constexpr int EV_NT = 256;     // threads per block
static constexpr int EV_ROWS = 256;   // rows per block of the completion pass
static constexpr double EV_LOG2E = 1.4426950408889634;

// C_ij = sqrt(dx^2 + dy^2) formed in FP64 with explicit rounding steps (no contraction) and
// rounded once to FP32.
__global__ void __launch_bounds__(EV_NT) k_euclid(const float2* __restrict__ dev, const float2* __restrict__ rrh,
                                                  int64_t I, int J, float* __restrict__ C, int64_t ld) {
    for (int64_t i = blockIdx.x; i < I; i += gridDim.x) {
        const float2 d = dev[i];
        for (int j = threadIdx.x; j < J; j += EV_NT) {
            const float2 r = __ldg(rrh + j);
            const double dx = __dadd_rn((double)d.x, -(double)r.x);
            const double dy = __dadd_rn((double)d.y, -(double)r.y);
            const double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            C[i * ld + j] = __double2float_rn(__dsqrt_rn(s));
        }
    }
}

// Per block of EV_ROWS rows: column partials (rho_j, u_j) in FP64, rows in order.
__global__ void __launch_bounds__(EV_NT) k_completion_part(const float* __restrict__ C, int64_t ld,
                                                           const float* __restrict__ lam, int64_t I, int J,
                                                           const int32_t* __restrict__ assoc,
                                                           const float* __restrict__ Cp, int64_t ldp,
                                                           const double* __restrict__ f,
                                                           const double* __restrict__ g, double inv_eps,
                                                           double2* __restrict__ part, int* __restrict__ bad) {
    const int64_t r0 = (int64_t)blockIdx.x * EV_ROWS;
    const int64_t r1 = min(I, r0 + EV_ROWS);
    int b = 0;
    for (int j0 = 0; j0 < J; j0 += EV_NT) {
        const int j = j0 + threadIdx.x;
        if (j >= J) break;
        const double gj = assoc ? 0.0 : g[j];
        double rho = 0.0, u = 0.0;
        for (int64_t i = r0; i < r1; ++i) {
            const float l = __ldg(lam + i);
            b |= !(l > 0.0f) || !isfinite(l);
            double x;
            if (assoc) {
                x = (__ldg(assoc + i) == j) ? (double)l : 0.0;
            } else {
                const double t = (f[i] + gj - (double)__ldg(Cp + i * ldp + j)) * inv_eps;
                x = (double)exp2f((float)(t * EV_LOG2E));
            }
            const double c = (double)__ldg(C + i * ld + j);
            rho = fma(c, x, rho);
            u = fma(c, x / (double)l, u);
        }
        part[(int64_t)blockIdx.x * J + j] = make_double2(rho, u);
    }
    if (b) atomicOr(bad, 1);
}

// Column totals over the blocks in order, then T over the columns in a fixed tree.
__global__ void __launch_bounds__(EV_NT) k_completion_sum(const double2* __restrict__ part, int nblk, int J,
                                                          int64_t I, double* __restrict__ rho_out,
                                                          double* __restrict__ T_out) {
    __shared__ double s_t[EV_NT];
    __shared__ int s_inf[EV_NT];
    double t = 0.0;
    int inf = 0;
    for (int j = threadIdx.x; j < J; j += EV_NT) {
        double rho = 0.0, u = 0.0;
        for (int k = 0; k < nblk; ++k) {
            const double2 v = part[(int64_t)k * J + j];
            rho += v.x;
            u += v.y;
        }
        if (rho_out) rho_out[j] = rho;
        if (u > 0.0) {
            if (rho >= 1.0) inf = 1;
            else t += u / (1.0 - rho);
        }
    }
    s_t[threadIdx.x] = t;
    s_inf[threadIdx.x] = inf;
    __syncthreads();
    for (int w = EV_NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s_t[threadIdx.x] += s_t[threadIdx.x + w];
            s_inf[threadIdx.x] |= s_inf[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *T_out = s_inf[0] ? INFINITY : s_t[0] / (double)I;
}

// Mean over rows of the row minimum (the cost of each device's cheapest link): per block of
// EV_ROWS rows one FP64 partial, rows in order; then the partials in order.
__global__ void __launch_bounds__(EV_NT) k_rowmin_part(const float* __restrict__ C, int64_t ld, int64_t I, int J,
                                                       double* __restrict__ part) {
    __shared__ float s_m[EV_NT / 32];
    __shared__ double s_sum;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * EV_ROWS;
    const int64_t r1 = min(I, r0 + EV_ROWS);
    if (threadIdx.x == 0) s_sum = 0.0;
    for (int64_t i = r0; i < r1; ++i) {
        float m = INFINITY;
        for (int j = threadIdx.x; j < J; j += EV_NT) m = fminf(m, __ldg(C + i * ld + j));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_m[warp] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            float mm = s_m[0];
            for (int w = 1; w < EV_NT / 32; ++w) mm = fminf(mm, s_m[w]);
            s_sum += (double)mm;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s_sum;
}

__global__ void k_rowmin_sum(const double* __restrict__ part, int nblk, int64_t I, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < nblk; ++k) t += part[k];
        *out = t / (double)I;
    }
}

}  // namespace ota

using namespace ota;

extern "C" {

ot_status ot_assoc_euclid_cost(ot_assoc_ctx* ctx, const float* dev_xy, const float* rrh_xy, int64_t I, int64_t J,
                               float* C_out, int64_t ld_c, void* stream) {
    if (!ctx) return OT_EINVAL;
    DeviceGuardLite guard(ctx->device);
    if (!dev_xy || !rrh_xy || !C_out) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0 || J > (1 << 24)) return set_error(ctx, OT_EINVAL, "bad I or J");
    const int64_t ld = ld_c ? ld_c : J;
    if (ld < J) return set_error(ctx, OT_EINVAL, "ld_c < J");
    if (((uintptr_t)dev_xy & 7u) || ((uintptr_t)rrh_xy & 7u))
        return set_error(ctx, OT_EINVAL, "coordinates must be 8-byte aligned (x, y float pairs)");
    const int grid = (int)std::min<int64_t>(I, 16LL * ctx->num_sms);
    k_euclid<<<grid, EV_NT, 0, (cudaStream_t)stream>>>((const float2*)dev_xy, (const float2*)rrh_xy, I, (int)J,
                                                        C_out, ld);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "euclid cost launch");
    return OT_OK;
}

ot_status ot_assoc_completion_time(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* traffic,
                                   int64_t I, int64_t J, const int32_t* assoc, const float* C_plan,
                                   int64_t ld_plan, const double* f, const double* g, double eps,
                                   double* rho_out, double* T_out, void* stream) {
    if (!ctx) return OT_EINVAL;
    DeviceGuardLite guard(ctx->device);
    if (!C || !traffic || !T_out) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0 || J > (1 << 20)) return set_error(ctx, OT_EINVAL, "bad I or J");
    const int64_t ld = ld_c ? ld_c : J;
    if (ld < J) return set_error(ctx, OT_EINVAL, "ld_c < J");
    const float* Cp = nullptr;
    int64_t ldp = 0;
    double inv_eps = 0.0;
    if (!assoc) {
        if (!f || !g) return set_error(ctx, OT_EINVAL, "potentials f and g (or an association) are required");
        if (!(eps > 0.0) || !std::isfinite(eps)) return set_error(ctx, OT_EINVAL, "eps");
        Cp = C_plan ? C_plan : C;
        ldp = C_plan ? (ld_plan ? ld_plan : J) : ld;
        if (ldp < J) return set_error(ctx, OT_EINVAL, "ld_plan < J");
        inv_eps = 1.0 / eps;
    }
    const int nblk = (int)((I + EV_ROWS - 1) / EV_ROWS);
    ot_status st = OT_OK;
    const size_t off_p = 256, off_t = off_p + (size_t)round_up((int64_t)sizeof(double2) * nblk * J, 256);
    char* ws = (char*)scratch(ctx, SLOT_MISC, off_t + 256, &st);
    if (st) return st;
    int* bad = (int*)ws;
    double2* part = (double2*)(ws + off_p);
    double* Td = (double*)(ws + off_t);
    double* hT = (double*)host_staging(ctx, 2 * sizeof(double), &st);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "completion memset");
    k_completion_part<<<nblk, EV_NT, 0, s>>>(C, ld, traffic, I, (int)J, assoc, Cp, ldp, f, g, inv_eps, part, bad);
    k_completion_sum<<<1, EV_NT, 0, s>>>(part, nblk, (int)J, I, rho_out, Td);
    ctx->launches += 2;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hT, Td, sizeof(double), cudaMemcpyDeviceToHost, s);
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hT + 1, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "completion time");
    std::memcpy(&hbad, hT + 1, sizeof(int));
    if (hbad) return set_error(ctx, OT_EINVAL, "traffic entries must be positive and finite");
    *T_out = hT[0];
    return OT_OK;
}

ot_status ot_assoc_mean_row_min(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, int64_t I, int64_t J,
                                double* out, void* stream) {
    if (!ctx) return OT_EINVAL;
    DeviceGuardLite guard(ctx->device);
    if (!C || !out) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0) return set_error(ctx, OT_EINVAL, "bad I or J");
    const int64_t ld = ld_c ? ld_c : J;
    if (ld < J) return set_error(ctx, OT_EINVAL, "ld_c < J");
    const int nblk = (int)((I + EV_ROWS - 1) / EV_ROWS);
    ot_status st = OT_OK;
    double* part = (double*)scratch(ctx, SLOT_MISC, sizeof(double) * ((size_t)nblk + 1), &st);
    if (st) return st;
    double* h = (double*)host_staging(ctx, sizeof(double), &st);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    k_rowmin_part<<<nblk, EV_NT, 0, s>>>(C, ld, I, (int)J, part);
    k_rowmin_sum<<<1, 32, 0, s>>>(part, nblk, I, part + nblk);
    ctx->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, part + nblk, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "mean row min");
    *out = *h;
    return OT_OK;
}

}  // extern "C"
