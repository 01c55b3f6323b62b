// FP64 Sinkhorn in the log domain (Algorithm 1 of the paper, Sec. III-B), every per-cell
// operation in double precision.  A reference-precision path for small instances (the
// 1000 x 50 configuration): GB300 issues FP64 at a small fraction of its FP32 rate, so the
// FP32 persistent solver is the fast path and this one is for checking it.
//
// One cooperative launch; warps take rows, then columns, grid barriers in between:
//   row update     f_i = eps log p^_i - eps LSE_j((g_j - C_ij) / eps)
//   column update  g_j = eps log q^_j - eps LSE_i((f_i - C_ij) / eps)
// (LSE with the maximum factored out, two passes over the row or column).  As in the FP32
// solver, the row update of iteration s also gives the row residual of the plan of
// iteration s - 1 (sum_j pi_ij = p^_i exp((f_i^(s-1) - f_i^s) / eps)), the loop test
// ("while accuracy") is taken on it, and a stop returns that plan's potentials.  Masses
// are normalised to 1 while iterating; f is shifted by eps log(sum p) at the end so that
// pi = exp((f + g - C) / eps) carries the caller's mass.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "ot_common.cuh"
#include "ot_internal.h"

namespace ota {

static constexpr int F64_NT = 256;
static constexpr int F64_NW = F64_NT / 32;
enum : int { F64_ENUMERIC = -7 };

struct F64State {
    unsigned bar;
    int status;
    int iters;
    int converged;
    double err;
    double sp, sq;
};

struct F64Params {
    const double* C;
    int64_t ld;
    int64_t I;
    int J;
    const double* p;
    const double* q;
    const double* g_warm;
    double eps, tol;
    int max_iter;
    double* fb;     // [2][I] row potentials, unit mass (buffer s & 1 holds f^s)
    double* gb;     // [2][J] column potentials (buffer s & 1 holds g^s)
    double* part;   // [grid][4] per-CTA partial sums
    F64State* st;
    // outputs
    double* f_out;
    double* g_out;
    double* rrh_load;
    float* pi;
    int64_t pi_ld;
    SolveSummary* summ;
    long long spin;
};

// Block sum of one double per thread, in a fixed order; every thread gets the total.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < F64_NW; ++w) t += sh[w];
    return t;
}

__device__ __forceinline__ double warp_maxd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// -eps * LSE over one row (lanes stride the columns): returns eps * log(sum) + eps * max.
__device__ __forceinline__ double row_lse(const double* row, const double* g, int J, double inv_eps, double eps) {
    const int lane = threadIdx.x & 31;
    double m = -INFINITY;
    for (int j = lane; j < J; j += 32) m = fmax(m, (g[j] - row[j]) * inv_eps);
    m = warp_maxd(m);
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int j = lane; j < J; j += 32) s += exp((g[j] - row[j]) * inv_eps - m);
    s = warp_sum(s);
    return eps * (m + log(s));
}

__device__ __forceinline__ double col_lse(const double* C, int64_t ld, int64_t I, int j, const double* f,
                                          double inv_eps, double eps) {
    const int lane = threadIdx.x & 31;
    double m = -INFINITY;
    for (int64_t i = lane; i < I; i += 32) m = fmax(m, (f[i] - C[i * ld + j]) * inv_eps);
    m = warp_maxd(m);
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int64_t i = lane; i < I; i += 32) s += exp((f[i] - C[i * ld + j]) * inv_eps - m);
    s = warp_sum(s);
    return eps * (m + log(s));
}

__global__ void __launch_bounds__(F64_NT) sk_solve64(F64Params P) {
    __shared__ double sh[F64_NW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = gridDim.x, b = blockIdx.x;
    const int gw = b * F64_NW + warp, nw = nb * F64_NW;
    const int64_t I = P.I;
    const int J = P.J;
    const double eps = P.eps, inv_eps = 1.0 / P.eps;
    int* status = &P.st->status;
    unsigned gen = 0;
#define F64_BARRIER()                                                                   \
    do {                                                                                \
        if (!grid_barrier(&P.st->bar, (unsigned)nb * ++gen, status, P.spin)) return;   \
    } while (0)

    // ---- setup: sums of p and q (fixed order), checks, starting g -------------------------
    {
        double sp = 0.0, sq = 0.0;
        int bad = 0;
        for (int64_t i = b * (int64_t)F64_NT + threadIdx.x; i < I; i += (int64_t)nb * F64_NT) {
            const double v = P.p[i];
            bad |= !(v > 0.0) || !isfinite(v);
            sp += v;
        }
        for (int j = b * F64_NT + threadIdx.x; j < J; j += nb * F64_NT) {
            const double v = P.q[j];
            bad |= !(v > 0.0) || !isfinite(v);
            sq += v;
            const double g0 = P.g_warm ? P.g_warm[j] : 0.0;
            bad |= !isfinite(g0);
            P.gb[j] = g0;  // g^0 in buffer 0
        }
        sp = block_sum(sp, sh);
        sq = block_sum(sq, sh);
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(status, DEV_OK, DEV_EINVAL);
        if (threadIdx.x == 0) {
            P.part[4 * b + 0] = sp;
            P.part[4 * b + 1] = sq;
        }
    }
    F64_BARRIER();
    double sp = 0.0, sq = 0.0;
    for (int bb = 0; bb < nb; ++bb) {
        sp += P.part[4 * bb + 0];
        sq += P.part[4 * bb + 1];
    }
    if (!(fabs(sp - sq) <= 1e-5 * sp)) {
        if (b == 0 && threadIdx.x == 0) atomicCAS(status, DEV_OK, DEV_EINVAL);
        return;  // the same decision in every CTA
    }
    const double lsp = log(sp), lsq = log(sq);
    F64_BARRIER();  // every CTA has read the sums before `part` is reused

    // ---- iterations --------------------------------------------------------------------------
    int ret = 0;  // buffer holding the returned potentials
    for (int s = 1;; ++s) {
        const double* gprev = P.gb + ((s - 1) & 1) * J;
        double* fcur = P.fb + (s & 1) * I;
        const double* fprev = P.fb + ((s - 1) & 1) * I;
        double res = 0.0;
        for (int64_t i = gw; i < I; i += nw) {
            const double v = log(P.p[i]) - lsp - row_lse(P.C + i * P.ld, gprev, J, inv_eps, eps) * inv_eps;
            const double fi = eps * v;
            if (lane == 0) {
                if (!isfinite(fi)) atomicCAS(status, DEV_OK, F64_ENUMERIC);
                fcur[i] = fi;
                if (s > 1) res += exp(log(P.p[i]) - lsp) * fabs(expm1((fprev[i] - fi) * inv_eps));
            }
        }
        res = block_sum(res, sh);
        if (threadIdx.x == 0) P.part[4 * b + 2] = res;
        F64_BARRIER();
        if (s > 1) {
            double e = 0.0;
            for (int bb = 0; bb < nb; ++bb) e += P.part[4 * bb + 2];
            const bool stop = (e <= P.tol) || (s - 1 >= P.max_iter) || ld_volatile_i32(status) != DEV_OK;
            if (stop) {
                if (b == 0 && threadIdx.x == 0) {
                    P.st->iters = s - 1;
                    P.st->err = e;
                    P.st->converged = (e <= P.tol);
                }
                ret = (s - 1) & 1;
                break;
            }
        }
        double* gcur = P.gb + (s & 1) * J;
        for (int j = gw; j < J; j += nw) {
            const double v = log(P.q[j]) - lsq - col_lse(P.C, P.ld, I, j, fcur, inv_eps, eps) * inv_eps;
            if (lane == 0) {
                if (!isfinite(v)) atomicCAS(status, DEV_OK, F64_ENUMERIC);
                gcur[j] = eps * v;
            }
        }
        F64_BARRIER();
    }

    // ---- finalize: plan of (f^ret, g^ret), FP64 marginals, loads, cost ------------------------
    const double* fr = P.fb + ret * I;
    const double* gr = P.gb + ret * J;
    {
        double er = 0.0;
        for (int64_t i = gw; i < I; i += nw) {
            const double* row = P.C + i * P.ld;
            double rsum = 0.0;
            for (int j = lane; j < J; j += 32) {
                const double pij = exp((fr[i] + gr[j] - row[j]) * inv_eps);
                rsum += pij;
                if (P.pi) P.pi[i * P.pi_ld + j] = (float)(pij * sp);
            }
            rsum = warp_sum(rsum);
            if (lane == 0) {
                er += fabs(rsum - P.p[i] / sp);
                P.f_out[i] = fr[i] + eps * lsp;
            }
        }
        double ec = 0.0, cost = 0.0;
        for (int j = gw; j < J; j += nw) {
            double csum = 0.0, rho = 0.0;
            for (int64_t i = lane; i < I; i += 32) {
                const double c = P.C[i * P.ld + j];
                const double pij = exp((fr[i] + gr[j] - c) * inv_eps);
                csum += pij;
                rho += pij > 0.0 ? c * pij : 0.0;
            }
            csum = warp_sum(csum);
            rho = warp_sum(rho);
            if (lane == 0) {
                ec += fabs(csum - P.q[j] / sq);
                cost += rho;
                if (P.rrh_load) P.rrh_load[j] = rho * sp;
                P.g_out[j] = gr[j];
            }
        }
        er = block_sum(er, sh);
        ec = block_sum(ec, sh);
        cost = block_sum(cost, sh);
        if (threadIdx.x == 0) {
            P.part[4 * b + 0] = er;
            P.part[4 * b + 1] = ec;
            P.part[4 * b + 3] = cost;
        }
    }
    F64_BARRIER();
    if (b == 0 && threadIdx.x == 0) {
        double er = 0.0, ec = 0.0, co = 0.0;
        for (int bb = 0; bb < nb; ++bb) {
            er += P.part[4 * bb + 0];
            ec += P.part[4 * bb + 1];
            co += P.part[4 * bb + 3];
        }
        P.summ->err_row = er;
        P.summ->err_col = ec;
        P.summ->cost = co * sp;
        P.summ->err_loop = P.st->err;
        P.summ->iters = P.st->iters;
        P.summ->converged = P.st->converged;
        P.summ->status = P.st->status;
        P.summ->absorptions = 0;
    }
#undef F64_BARRIER
}

__global__ void sk_summary64(const F64State* st, SolveSummary* summ) {
    // status of a launch that stopped early (invalid input or a wait that gave up)
    if (threadIdx.x == 0 && st->status != DEV_OK) {
        summ->status = st->status;
        summ->iters = st->iters;
        summ->converged = 0;
    }
}

ot_status launch_solve_f64(ot_assoc_ctx* ctx, const SolveArgs64& a, SolveSummary* sum_host) {
    ot_status st = OT_OK;
    const int64_t I = a.I;
    const int J = a.J;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sk_solve64, F64_NT, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return set_error(ctx, OT_ECUDA, "FP64 solver cannot be resident");
    }
    const int64_t work = std::max<int64_t>(I, J);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((work + F64_NW - 1) / F64_NW, (int64_t)ctx->num_sms));
    double* fb = (double*)scratch(ctx, SLOT_F, sizeof(double) * 2 * (size_t)I, &st);
    if (st) return st;
    double* gb = (double*)scratch(ctx, SLOT_G, sizeof(double) * 2 * (size_t)round_up(J, 4), &st);
    if (st) return st;
    double* part = (double*)scratch(ctx, SLOT_ERRPART, sizeof(double) * 4 * (size_t)grid, &st);
    if (st) return st;
    char* state = (char*)scratch(ctx, SLOT_STATE, 4096, &st);
    if (st) return st;
    F64State* fst = (F64State*)state;
    SolveSummary* summ = (SolveSummary*)(state + 512);
    SolveSummary* hsum = (SolveSummary*)host_staging(ctx, sizeof(SolveSummary), &st);
    if (st) return st;
    cudaStream_t s = a.stream;
    cudaError_t e = cudaMemsetAsync(state, 0, 1024, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "memset");
    F64Params P;
    P.C = a.C;
    P.ld = a.ld;
    P.I = I;
    P.J = J;
    P.p = a.p;
    P.q = a.q;
    P.g_warm = a.warm_start ? a.out->g : nullptr;
    P.eps = a.eps;
    P.tol = a.tol;
    P.max_iter = a.max_iter;
    P.fb = fb;
    P.gb = gb;
    P.part = part;
    P.st = fst;
    P.f_out = a.out->f;
    P.g_out = a.out->g;
    P.rrh_load = a.out->rrh_load;
    P.pi = a.out->pi;
    P.pi_ld = a.out->pi_ld > 0 ? a.out->pi_ld : J;
    P.summ = summ;
    P.spin = ctx->spin_limit;
    void* args[] = {&P};
    e = cudaLaunchCooperativeKernel((const void*)sk_solve64, dim3(grid), dim3(F64_NT), args, 0, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "FP64 solve launch");
    sk_summary64<<<1, 32, 0, s>>>(fst, summ);
    ctx->launches += 2;
    e = cudaMemcpyAsync(hsum, summ, sizeof(SolveSummary), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "FP64 solve");
    *sum_host = *hsum;
    if (sum_host->status == F64_ENUMERIC) sum_host->status = OT_ENUMERIC_INTERNAL;
    return OT_OK;
}

}  // namespace ota
