// Rate and cost construction (Sec. II-A, Sec. IV choice (ii)) and the maxSINR rule (Sec. II-C).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "ot_common.cuh"
#include "ot_internal.h"

namespace ota {

static constexpr int NTC = 256;

// Dispatch a team-per-row kernel template over (TW, VPT) by the row length J.
#define OTA_ROW_DISPATCH(J, KERNEL, ...)                                                      \
    do {                                                                                      \
        const int J4_ = ((J) + 3) / 4;                                                        \
        if (J4_ <= 32) KERNEL<1, 1> __VA_ARGS__;                                              \
        else if (J4_ <= 64) KERNEL<1, 2> __VA_ARGS__;                                         \
        else if (J4_ <= 128) KERNEL<1, 4> __VA_ARGS__;                                        \
        else if (J4_ <= 256) KERNEL<1, 8> __VA_ARGS__;                                        \
        else if (J4_ <= 512) KERNEL<2, 8> __VA_ARGS__;                                        \
        else if (J4_ <= 1024) KERNEL<4, 8> __VA_ARGS__;                                       \
        else KERNEL<8, 8> __VA_ARGS__;                                                        \
    } while (0)

// ------------------------------------------------------------------------------------------
// Rates: SINR_ij = P_j G_ij / (T_i - P_j G_ij), T_i = N0 + sum_k P_k G_ik,
//        R_ij = W log2(1 + SINR_ij).
// The row total is a compensated (Neumaier) FP32 sum per thread, combined across threads
// as error-free FP32 pairs (no FP64: GB300 issues it at a small fraction of the FP32 rate).  Each own term P_j G_ij is kept as an exact hi + lo pair, so
// T_i - own loses nothing when one RRH dominates (T_hi - own_hi is exact by Sterbenz).
// ------------------------------------------------------------------------------------------
// Two passes: k_rowtot forms T_i per row (a team per row, the compensated sum above), then
// k_rate_cells forms every cell's rate (and with C non-null the cost C_ij = (1/mu) / R_ij, one
// IEEE FP32 division, as k_cost, counting rates that are not finite and > 0; R may then be
// null) with one thread per 4-column chunk.  The cells' arithmetic (a division, log1pf and
// a correctly rounded reciprocal: about 65 instructions a cell) needs more warps than a
// team-per-row kernel at 128 registers keeps; the second read of G costs less than that
// (the single pass ran at 249 us on 50,000 x 800).
template <int TW, int VPT>
__global__ void __launch_bounds__(NTC, 4) k_rowtot(const float* __restrict__ G, int64_t ld_g,
                                                const float* __restrict__ P, int64_t I, int J, float2 N0,
                                                float2* __restrict__ T_out) {
    constexpr int TT = 32 * TW, NTEAMS = NTC / TT;
    constexpr int JMAX = 4 * TT * VPT;  // columns a team covers
    __shared__ float2 red[2 * NTEAMS * TW];
    __shared__ __align__(16) float pws[JMAX];  // transmit powers (0 past J): shared, not per-thread registers
    const Team<TW> tm;
    for (int j = threadIdx.x; j < JMAX; j += NTC) pws[j] = j < J ? P[j] : 0.0f;
    __syncthreads();
    int par = 0;
    const int64_t team_g = (int64_t)blockIdx.x * NTEAMS + tm.team;
    const int64_t nteams_g = (int64_t)gridDim.x * NTEAMS;
    for (int64_t i = team_g; i < I; i += nteams_g) {
        float4 x[VPT];
        load_row<TW, VPT>(G + i * ld_g, J, tm.tl, x, 0.0f);
        float s = 0.f, cmp = 0.f;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            float4 pw = *reinterpret_cast<const float4*>(pws + 4 * (tm.tl + TT * v));
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float hi = comp(pw, c) * comp(x[v], c);
                const float lo = fmaf(comp(pw, c), comp(x[v], c), -hi);
                const float t = s + hi;
                cmp += (fabsf(s) >= fabsf(hi)) ? ((s - t) + hi) : ((hi - t) + s);
                cmp += lo;
                s = t;
            }
        }
        // row total as an FP32 pair: warp sum of the (sum, compensation) pairs, then the team
        float2 T = warp_sum_df(make_float2(s, cmp));
        if constexpr (TW > 1) {
            float2* r = red + (par * NTEAMS + tm.team) * TW;
            if (tm.lane == 0) r[tm.wit] = T;
            bar_named(1 + tm.team, TT);
            T = r[0];
            for (int w = 1; w < TW; ++w) T = df_add2(T, r[w]);
            par ^= 1;
        }
        if (tm.tl == 0) T_out[i] = df_add2(T, N0);
    }
}

// One thread per (row, 4-column chunk) of a block's rows [blockIdx.x * rows, + rows).
__global__ void __launch_bounds__(NTC) k_rate_cells(const float* __restrict__ G, int64_t ld_g,
                                                    const float* __restrict__ P, int64_t I, int J, int rows,
                                                    const float2* __restrict__ T, float w_log2e,
                                                    float* __restrict__ R, int64_t ld_r, int vec_out, float inv_mu,
                                                    float* __restrict__ C, int64_t ld_c, int vec_c,
                                                    unsigned long long* bad) {
    unsigned long long nbad = 0;
    const int J4 = (J + 3) >> 2;
    const int64_t r0 = (int64_t)blockIdx.x * rows;
    const int nrow = (int)min((int64_t)rows, I - r0);
    const int n = nrow * J4;
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
        const int rr = f / J4, c4 = f - rr * J4;
        const int64_t i = r0 + rr;
        const int col = 4 * c4;
        // rows are 16-byte aligned, so a chunk that starts below J stays inside the padded row
        float4 x = __ldg(reinterpret_cast<const float4*>(G + i * ld_g + col));
        float4 pw;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const bool in = col + c < J;
            if (!in) comp(x, c) = 0.0f;
            comp(pw, c) = in ? __ldg(P + col + c) : 0.0f;
        }
        const float2 Ti = T[i];
        float4 r;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            // the own term as the same exact pair as in the row total
            const float own = comp(pw, c) * comp(x, c);
            const float own_lo = fmaf(comp(pw, c), comp(x, c), -own);
            const float interf = (Ti.x - own) + (Ti.y - own_lo);
            const float sinr = interf > 0.f ? own / interf : INFINITY;
            comp(r, c) = w_log2e * log1pf(sinr);
        }
        if (R) {
            float* rrow = R + i * ld_r;
            if (col + 4 <= J && vec_out) {
                *reinterpret_cast<float4*>(rrow + col) = r;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (col + c < J) rrow[col + c] = comp(r, c);
            }
        }
        if (C) {
            float4 o;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float rv = comp(r, c);
                nbad += (col + c < J) && !(rv > 0.0f && isfinite(rv));
                comp(o, c) = __fdiv_rn(inv_mu, rv);
            }
            float* crow = C + i * ld_c;
            if (col + 4 <= J && vec_c) {
                *reinterpret_cast<float4*>(crow + col) = o;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (col + c < J) crow[col + c] = comp(o, c);
            }
        }
    }
    if (nbad) atomicAdd(bad, nbad);
}

ot_status launch_rates(ot_assoc_ctx* ctx, const float* G, int64_t ld_g, const float* P, int64_t I, int J,
                       double N0, double W, float* R, int64_t ld_r, cudaStream_t s, double mu, float* C,
                       int64_t ld_c, unsigned long long* bad_dev) {
    if (ld_g % 4 != 0 || ((uintptr_t)G & 15u))
        return set_error(ctx, OT_EINVAL, "G rows must be 16-byte aligned (ld_g %% 4 == 0, aligned base)");
    const int vec_out = R && (ld_r % 4 == 0) && !((uintptr_t)R & 15u);
    const int vec_c = C && (ld_c % 4 == 0) && !((uintptr_t)C & 15u);
    const float inv_mu = C ? (float)(1.0 / mu) : 0.0f;
    const float w_log2e = (float)(W / 0.69314718055994530942);
    const int nteams = NTC / (32 * (J <= 1024 ? 1 : (J <= 2048 ? 2 : (J <= 4096 ? 4 : 8))));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((I + nteams - 1) / nteams, 8LL * ctx->num_sms));
    const float n0_hi = (float)N0;
    const float2 n0 = make_float2(n0_hi, (float)(N0 - (double)n0_hi));
    ot_status st = OT_OK;
    float2* T = (float2*)scratch(ctx, SLOT_ROWTOT, sizeof(float2) * (size_t)I, &st);
    if (st) return st;
    OTA_ROW_DISPATCH(J, k_rowtot, <<<grid, NTC, 0, s>>>(G, ld_g, P, I, J, n0, T));
    const int J4 = (J + 3) / 4;
    const int rows = std::max(1, 8 * NTC / J4);  // about 8 chunks a thread
    const int64_t nblk = (I + rows - 1) / rows;
    k_rate_cells<<<(unsigned)nblk, NTC, 0, s>>>(G, ld_g, P, I, J, rows, T, w_log2e, R, ld_r, vec_out, inv_mu, C, ld_c,
                                                vec_c, bad_dev);
    ctx->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "rates launch");
    return OT_OK;
}

// ------------------------------------------------------------------------------------------
// Cost: C_ij = (1/mu) / R_ij with one IEEE FP32 division; padding columns [J, ld_c) = +inf.
// ------------------------------------------------------------------------------------------
__global__ void k_cost(const float* __restrict__ R, int64_t ld_r, int64_t I, int J, float inv_mu,
                       float* __restrict__ C, int64_t ld_c, int pad_inf, int vec_in, int vec_out,
                       unsigned long long* bad) {
    const int row_ch = (int)((ld_c + 3) / 4);  // chunks per output row (incl. padding)
    const int rpb = max(1, (int)blockDim.x / row_ch);  // rows handled together by one block
    const int sub = threadIdx.x / row_ch;
    const int ch0 = threadIdx.x - sub * row_ch;
    unsigned long long nbad = 0;
    for (int64_t i0 = (int64_t)blockIdx.x * rpb; i0 < I; i0 += (int64_t)gridDim.x * rpb) {
        const int64_t i = i0 + sub;
        if (sub >= rpb || i >= I) continue;
        for (int ch = (rpb > 1 ? ch0 : (int)threadIdx.x); ch < row_ch; ch += (rpb > 1 ? row_ch : (int)blockDim.x)) {
            const int col = ch * 4;
            float r[4];
            if (vec_in && col + 4 <= J) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(R + i * ld_r + col));
                r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) r[c] = (col + c < J) ? __ldg(R + i * ld_r + col + c) : 1.0f;
            }
            float o[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (col + c < J) {
                    const bool ok = r[c] > 0.0f && isfinite(r[c]);
                    nbad += !ok;
                    o[c] = __fdiv_rn(inv_mu, r[c]);
                } else {
                    o[c] = INFINITY;
                }
            }
            float* crow = C + i * ld_c;
            if (vec_out && col + 4 <= ld_c && (pad_inf || col + 4 <= J)) {
                *reinterpret_cast<float4*>(crow + col) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (col + c < J || (pad_inf && col + c < ld_c)) crow[col + c] = o[c];
            }
        }
    }
    if (nbad) atomicAdd(bad, nbad);
}

ot_status launch_cost(ot_assoc_ctx* ctx, const float* R, int64_t ld_r, int64_t I, int J, double mu, float* C,
                      int64_t ld_c, bool pad_inf, unsigned long long* bad_dev, cudaStream_t s) {
    const int vec_in = (ld_r % 4 == 0) && !((uintptr_t)R & 15u);
    const int vec_out = (ld_c % 4 == 0) && !((uintptr_t)C & 15u);
    const float inv_mu = (float)(1.0 / mu);
    const int64_t row_ch = (ld_c + 3) / 4;
    const int64_t rpb = std::max<int64_t>(1, 256 / row_ch);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((I + rpb - 1) / rpb, 16LL * ctx->num_sms));
    k_cost<<<grid, 256, 0, s>>>(R, ld_r, I, J, inv_mu, C, ld_c, pad_inf ? 1 : 0, vec_in, vec_out, bad_dev);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "cost launch");
    return OT_OK;
}

// ------------------------------------------------------------------------------------------
// maxSINR: j*(i) = argmax_j R_ij (lowest j on ties); Lambda_j = sum_{j*(i)=j} lambda_i;
// total load = sum_i lambda_i / (mu R_{i j*(i)}).  Deterministic: Lambda is formed per
// contiguous row block in row order, then the blocks are summed in block order.
// ------------------------------------------------------------------------------------------
static constexpr int MS_ROWS = 1024;  // rows per block of the Lambda pass

template <int TW, int VPT>
__global__ void __launch_bounds__(NTC) k_argmax(const float* __restrict__ R, int64_t ld_r, int64_t I, int J,
                                                int32_t* __restrict__ assoc, float* __restrict__ rbest) {
    constexpr int TT = 32 * TW, NTEAMS = NTC / TT;
    __shared__ float redv[2 * NTEAMS * TW];
    __shared__ float redi[2 * NTEAMS * TW];
    const Team<TW> tm;
    int par = 0, par2 = 0;
    const int64_t team_g = (int64_t)blockIdx.x * NTEAMS + tm.team;
    const int64_t nteams_g = (int64_t)gridDim.x * NTEAMS;
    for (int64_t i = team_g; i < I; i += nteams_g) {
        float4 x[VPT];
        load_row<TW, VPT>(R + i * ld_r, J, tm.tl, x, -INFINITY);
        float best = -INFINITY;
        int bidx = 0x7fffffff;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int col = 4 * (tm.tl + TT * v);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float r = comp(x[v], c);
                if (col + c < J && (r > best || (r == best && col + c < bidx))) {
                    best = r;
                    bidx = col + c;
                }
            }
        }
        const float m = team_reduce<TW, float, true>(best, redv, NTEAMS, tm, par);
        // lowest index among the threads holding the maximum (exact comparison)
        const float cand = (best == m) ? -(float)bidx : -INFINITY;
        const float ci = team_reduce<TW, float, true>(cand, redi, NTEAMS, tm, par2);
        if (tm.tl == 0) {
            assoc[i] = (int32_t)(-ci);
            rbest[i] = m;
        }
    }
}

// Per-block Lambda partials and total-load partials.  Thread t owns columns t, t+NTC, ...
__global__ void __launch_bounds__(NTC) k_lambda_part(const int32_t* __restrict__ assoc,
                                                     const float* __restrict__ rbest,
                                                     const float* __restrict__ lam, int64_t I, int J,
                                                     double inv_mu, double* __restrict__ part,
                                                     double* __restrict__ tpart) {
    __shared__ int32_t sa[MS_ROWS];
    __shared__ float sl[MS_ROWS];
    const int64_t r0 = (int64_t)blockIdx.x * MS_ROWS;
    const int nrow = (int)std::min<int64_t>(MS_ROWS, I - r0);
    double tl = 0.0;
    for (int k = threadIdx.x; k < nrow; k += NTC) {
        sa[k] = assoc[r0 + k];
        sl[k] = lam[r0 + k];
    }
    __syncthreads();
    // total load: fixed order within the block (thread 0 walks the rows)
    if (threadIdx.x == 0) {
        for (int k = 0; k < nrow; ++k) tl += (double)sl[k] * inv_mu / (double)rbest[r0 + k];
        tpart[blockIdx.x] = tl;
    }
    for (int j = threadIdx.x; j < J; j += NTC) {
        double a = 0.0;
        for (int k = 0; k < nrow; ++k)
            if (sa[k] == j) a += (double)sl[k];
        part[(int64_t)blockIdx.x * J + j] = a;
    }
}

__global__ void k_lambda_sum(const double* __restrict__ part, const double* __restrict__ tpart, int nblk,
                             int J, double* __restrict__ Lambda, double* __restrict__ total) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < J && Lambda) {
        double a = 0.0;
        for (int b = 0; b < nblk; ++b) a += part[(int64_t)b * J + j];
        Lambda[j] = a;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && total) {
        double t = 0.0;
        for (int b = 0; b < nblk; ++b) t += tpart[b];
        *total = t;
    }
}

ot_status launch_maxsinr(ot_assoc_ctx* ctx, const float* R, int64_t ld_r, const float* lam, int64_t I, int J,
                         double mu, int32_t* assoc, double* Lambda, double* total_dev, cudaStream_t s) {
    if (ld_r % 4 != 0 || ((uintptr_t)R & 15u))
        return set_error(ctx, OT_EINVAL, "R rows must be 16-byte aligned (ld_r %% 4 == 0, aligned base)");
    ot_status st = OT_OK;
    const int nblk = (int)((I + MS_ROWS - 1) / MS_ROWS);
    // workspace: assoc (if not given), best rate per row, partials
    size_t off_a = 0, off_r = round_up(sizeof(int32_t) * I, 256), off_p = off_r + round_up(sizeof(float) * I, 256);
    size_t off_t = off_p + round_up(sizeof(double) * (size_t)nblk * J, 256);
    size_t total_bytes = off_t + round_up(sizeof(double) * nblk, 256);
    char* ws = (char*)scratch(ctx, SLOT_SELECT, total_bytes, &st);
    if (st) return st;
    int32_t* a = assoc ? assoc : (int32_t*)(ws + off_a);
    float* rb = (float*)(ws + off_r);
    double* part = (double*)(ws + off_p);
    double* tpart = (double*)(ws + off_t);
    const int nteams = NTC / (32 * (J <= 1024 ? 1 : (J <= 2048 ? 2 : (J <= 4096 ? 4 : 8))));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((I + nteams - 1) / nteams, 8LL * ctx->num_sms));
    OTA_ROW_DISPATCH(J, k_argmax, <<<grid, NTC, 0, s>>>(R, ld_r, I, J, a, rb));
    k_lambda_part<<<nblk, NTC, 0, s>>>(a, rb, lam, I, J, 1.0 / mu, part, tpart);
    k_lambda_sum<<<(J + 255) / 256, 256, 0, s>>>(part, tpart, nblk, J, Lambda, total_dev);
    ctx->launches += 3;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "maxsinr launch");
    return OT_OK;
}

}  // namespace ota
