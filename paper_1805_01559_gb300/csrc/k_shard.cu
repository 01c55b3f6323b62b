// Row-sharded Algorithm 1 (Sec. III-C, Eqs. (3)-(5), Algorithm 1): the steps of one
// iteration as separate calls, so that ranks holding different blocks of rows of C can add
// their column sums and row residuals between the sweep and the column update.
//
// A sweep over the shard's rows is one launch of k_shard_sweep (one team of 1, 2, 4 or 8 warps
// per row, each lane 8 float4 chunks of the row: J <= 1024 * team width) and one of
// k_shard_reduce, which adds the blocks' FP64 partials in block order (deterministic for a
// given shard and device).  The cell is the same as in the single-GPU solver:
// t_ij = 2^(F'_i + G_j - k C_ij) in log2 units with F' an FP32 pair and G an FP64 column
// potential held as an FP32 pair.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "ot_assoc.h"
#include "ot_common.cuh"
#include "ot_internal.h"
#include "sk_core.cuh"

namespace ota {
namespace {

constexpr int SH_NW = 8;   // warps a block
constexpr int SH_VPT = 8;  // float4 chunks a lane

struct ShardArgs {
    const float* C;
    int64_t ld;
    const float* p;
    int64_t I;
    int J, Jp;
    float inv_mass;     // 1 / (sum of p over every shard), rounded to FP32 as the solver does
    float k_hi, k_lo;   // log2(e) / eps as an FP32 pair
    double eps_ln2;     // eps ln 2: natural units of the potentials
    const double* G;    // [J] column potentials, log2 units
    const float2* F_in;
    float2* F_out;
    const double* colmax;  // [J] COLSUM: the reduced column maxima
    double* part;          // [nb][NACC][Jp]
    double* epart;         // [nb]
    double* f_out;         // FINAL: natural-unit row potentials, or null
    const double* state;   // loop state (state[0] != 0: the loop has stopped, do nothing), or null
};

template <int MODE>
struct ShardMode {
    static constexpr int NACC = MODE == OT_SHARD_FINAL ? 2 : 1;
    static constexpr bool MAX = MODE == OT_SHARD_COLMAX;
};

// One sweep over the shard's rows.  Dynamic shared memory: G pairs (2 Jp floats), the
// column maxima (Jp floats, COLSUM), then the teams' column accumulators (NTEAMS x NACC x Jp).
template <int TW, int MODE>
__global__ void __launch_bounds__(SH_NW * 32) k_shard_sweep(ShardArgs a) {
    constexpr int NTEAMS = SH_NW / TW, TT = 32 * TW, VPT = SH_VPT;
    constexpr int NACC = ShardMode<MODE>::NACC;
    constexpr bool MAX = ShardMode<MODE>::MAX;
    extern __shared__ __align__(16) float shs[];
    if (a.state && a.state[0] != 0.0) return;  // written only by earlier launches on the stream
    const int J = a.J, Jp = a.Jp;
    float* Gs = shs;              // [2 Jp]: hi, then lo
    float* Ms = shs + 2 * Jp;     // [Jp]
    float* slots = Ms + Jp;       // [NTEAMS][NACC][Jp]
    __shared__ float red[4 * SH_NW];
    __shared__ float errs[NTEAMS];
    for (int j = threadIdx.x; j < Jp; j += blockDim.x) {
        const double g = j < J ? a.G[j] : 0.0;
        const float hi = (float)g;
        Gs[j] = hi;
        Gs[Jp + j] = (float)(g - (double)hi);
        if (MODE == OT_SHARD_COLSUM) Ms[j] = j < J ? (float)a.colmax[j] : 0.f;
    }
    __syncthreads();
    const Team<TW> tm;
    int par = 0;
    float4 acc[NACC][VPT];
#pragma unroll
    for (int u = 0; u < NACC; ++u)
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const float z = MAX ? -INFINITY : 0.f;
            acc[u][v] = make_float4(z, z, z, z);
        }
    float err = 0.f;  // this team's rows: sum of p^_i |r_i - 1|
    const int64_t stride = (int64_t)gridDim.x * NTEAMS;
    float4 xn[VPT];  // the team's next row, loaded while the current one is worked on
    int64_t i = (int64_t)blockIdx.x * NTEAMS + tm.team;
    if (i < a.I) load_row<TW, VPT>(a.C + i * a.ld, J, tm.tl, xn);  // columns >= J read as +inf
    for (; i < a.I; i += stride) {
        float4 x[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) x[v] = xn[v];
        if (i + stride < a.I) load_row<TW, VPT>(a.C + (i + stride) * a.ld, J, tm.tl, xn);
        const float ph = __ldg(a.p + i) * a.inv_mass;     // p^_i
        if constexpr (MODE == OT_SHARD_FIRST) {
            // F'^1_i = -log2 sum_j 2^(G_j - k C_ij), shifted by the row's largest exponent
            float m = -INFINITY;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int col = 4 * (tm.tl + TT * v);
                if (col < Jp) {
                    const float4 gh = *reinterpret_cast<const float4*>(Gs + col);
                    m = fmaxf(m, fmaf(-x[v].x, a.k_hi, gh.x));
                    m = fmaxf(m, fmaf(-x[v].y, a.k_hi, gh.y));
                    m = fmaxf(m, fmaf(-x[v].z, a.k_hi, gh.z));
                    m = fmaxf(m, fmaf(-x[v].w, a.k_hi, gh.w));
                }
            }
            m = team_reduce<TW, float, true>(m, red, NTEAMS, tm, par);
            float sum = 0.f;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int col = 4 * (tm.tl + TT * v);
                float4 gh = make_float4(0.f, 0.f, 0.f, 0.f), gl = gh;
                if (col < Jp) {
                    gh = *reinterpret_cast<const float4*>(Gs + col);
                    gl = *reinterpret_cast<const float4*>(Gs + Jp + col);
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float t = ex2(expo2(-m, comp(gl, c), comp(gh, c), comp(x[v], c), a.k_hi, a.k_lo));
                    comp(x[v], c) = t;
                    sum += t;
                }
            }
            sum = team_reduce<TW, float, false>(sum, red, NTEAMS, tm, par);
            const float ls = log2f(sum);
            if (tm.tl == 0) {
                float hi, lo;
                two_sum(m, ls, hi, lo);
                a.F_out[i] = (sum > 0.f && m > -INFINITY) ? make_float2(-hi, -lo) : make_float2(NAN, NAN);
            }
            // the half-step plan's rows are normalised (t / sum <= 1): column sums of
            // p^_i t_ij / sum_i scaled by 2^64 cannot overflow
            const float w = __fdividef(ph, sum) * 0x1p64f;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                acc[0][v].x = fmaf(x[v].x, w, acc[0][v].x);
                acc[0][v].y = fmaf(x[v].y, w, acc[0][v].y);
                acc[0][v].z = fmaf(x[v].z, w, acc[0][v].z);
                acc[0][v].w = fmaf(x[v].w, w, acc[0][v].w);
            }
        } else {
            const float2 F = a.F_in[i];
            const float lp = (MODE == OT_SHARD_COLMAX || MODE == OT_SHARD_COLSUM) ? log2f(ph) : 0.f;
            float rsum = 0.f;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int col = 4 * (tm.tl + TT * v);
                float4 gh = make_float4(0.f, 0.f, 0.f, 0.f), gl = gh, mj = gh;
                if (col < Jp) {
                    gh = *reinterpret_cast<const float4*>(Gs + col);
                    gl = *reinterpret_cast<const float4*>(Gs + Jp + col);
                    if (MODE == OT_SHARD_COLSUM) mj = *reinterpret_cast<const float4*>(Ms + col);
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float cost = comp(x[v], c);
                    const float e = expo2(F.x, F.y + comp(gl, c), comp(gh, c), cost, a.k_hi, a.k_lo);
                    if constexpr (MODE == OT_SHARD_COLMAX) {
                        comp(acc[0][v], c) = fmaxf(comp(acc[0][v], c), e + lp);
                    } else if constexpr (MODE == OT_SHARD_COLSUM) {
                        comp(acc[0][v], c) += ex2((e + lp) - comp(mj, c));
                    } else {
                        const float t = ex2(e);
                        rsum += t;
                        if constexpr (MODE == OT_SHARD_FINAL) {
                            comp(acc[0][v], c) = fmaf(ph, t, comp(acc[0][v], c));
                            comp(acc[1][v], c) = fmaf(ph, t > 0.f ? cost * t : 0.f, comp(acc[1][v], c));
                        }
                        comp(x[v], c) = t;
                    }
                }
            }
            if constexpr (MODE == OT_SHARD_ITER) {
                const float r = team_reduce<TW, float, false>(rsum, red, NTEAMS, tm, par);
                if (tm.tl == 0) a.F_out[i] = df_sub(F, log2_corr(r));
                err = fmaf(ph, fabsf(r - 1.0f), err);
                const float d = __fdividef(ph, r);  // p^_i / r_i: the row of pi^(k) over t
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    acc[0][v].x = fmaf(x[v].x, d, acc[0][v].x);
                    acc[0][v].y = fmaf(x[v].y, d, acc[0][v].y);
                    acc[0][v].z = fmaf(x[v].z, d, acc[0][v].z);
                    acc[0][v].w = fmaf(x[v].w, d, acc[0][v].w);
                }
            } else if constexpr (MODE == OT_SHARD_FINAL) {
                const float2 r = team_sum_pair<TW>(rsum, red, NTEAMS, tm, par);
                err = fmaf(ph, fabsf((r.x - 1.0f) + r.y), err);
                if (a.f_out && tm.tl == 0)
                    a.f_out[i] = a.eps_ln2 * ((double)F.x + (double)F.y + log2((double)__ldg(a.p + i)));
            }
        }
    }
    // the block's column partials: teams in order, in FP64
#pragma unroll
    for (int u = 0; u < NACC; ++u)
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int col = 4 * (tm.tl + TT * v);
            if (col < Jp) *reinterpret_cast<float4*>(slots + ((size_t)tm.team * NACC + u) * Jp + col) = acc[u][v];
        }
    if (tm.tl == 0) errs[tm.team] = err;
    __syncthreads();
    double* out = a.part + (size_t)blockIdx.x * NACC * Jp;
    for (int u = 0; u < NACC; ++u)
        for (int j = threadIdx.x; j < J; j += blockDim.x) {
            double s = MAX ? -INFINITY : 0.0;
            for (int t = 0; t < NTEAMS; ++t) {
                const double y = (double)slots[((size_t)t * NACC + u) * Jp + j];
                s = MAX ? fmax(s, y) : s + y;
            }
            out[(size_t)u * Jp + j] = s;
        }
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int t = 0; t < NTEAMS; ++t) e += (double)errs[t];
        a.epart[blockIdx.x] = e;
    }
}

// Columns (and the row residual) over the sweep's blocks.  A block of 32 warps takes 32
// columns (one a lane); warp w adds the blocks w, w + 32, ... and the 32 warp sums are added
// in warp order: a fixed order, so the result is deterministic.  Block 0 also adds the row
// residuals (a fixed butterfly per warp, then the warps in order).
constexpr int SR_WARPS = 32;
__global__ void __launch_bounds__(SR_WARPS * 32) k_shard_reduce(const double* __restrict__ part,
                                                                const double* __restrict__ epart, int nb, int nacc,
                                                                int Jp, int J, int is_max, double* col_out,
                                                                double* row_out, const double* state) {
    __shared__ double sh[SR_WARPS][33];
    if (state && state[0] != 0.0) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;  // column over the nacc accumulators
    const bool in = j < nacc * J;
    const int u = in ? j / J : 0, jj = in ? j - u * J : 0;
    double s = is_max ? -INFINITY : 0.0;
    if (in)
        for (int b = w; b < nb; b += SR_WARPS) {
            const double y = part[((size_t)b * nacc + u) * Jp + jj];
            s = is_max ? fmax(s, y) : s + y;
        }
    sh[w][lane] = s;
    double e = 0.0;
    if (row_out && blockIdx.x == 0) {
        for (int b = threadIdx.x; b < nb; b += blockDim.x) e += epart[b];
        e = warp_sum(e);
    }
    __syncthreads();
    if (w == 0 && in) {
        double t = sh[0][lane];
        for (int k = 1; k < SR_WARPS; ++k) t = is_max ? fmax(t, sh[k][lane]) : t + sh[k][lane];
        col_out[(size_t)u * J + jj] = t;
    }
    if (row_out && blockIdx.x == 0) {
        __syncthreads();
        if (lane == 0) sh[w][32] = e;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < SR_WARPS; ++k) t += sh[k][32];
            *row_out = t;
        }
    }
}

// G^k_j = G^(k-1)_j + log2 q^_j - log2 s_j from the sums of every shard.  With a loop state
// (ITER): the loop test on the reduced residual of the plan (F'^(k-1), G^(k-1)) first; on a
// stop every thread leaves G as it is and thread 0 records iterations k - 1, the parity of the
// row-potential buffer that holds F'^(k-1), the residual and the reason in the state.
__global__ void k_shard_update(int mode, const float* __restrict__ q, int J, double inv_qmass,
                               const double* __restrict__ col, const double* __restrict__ colmax,
                               const double* G_in, double* G_out, int* flag, const double* err_in, int iter,
                               double tol_stop, int max_iter, double* state) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (state) {
        if (state[0] != 0.0) return;
        if (mode == OT_SHARD_ITER) {
            const double err = *err_in;  // every thread reads the same value: one decision
            const bool conv = err <= tol_stop;
            if (!isfinite(err) || conv || iter - 1 >= max_iter) {
                if (j == 0) {
                    state[1] = (double)(iter - 1);
                    state[2] = (double)((iter - 1) & 1);
                    state[3] = err;
                    state[0] = !isfinite(err) ? 3.0 : (conv ? 1.0 : 2.0);
                }
                return;
            }
        }
    }
    if (j >= J) return;
    const double lq = log2((double)q[j] * inv_qmass);
    const double c = col[j];
    if (mode == OT_SHARD_FIRST) {
        // scaled by 2^64; a sum below 2^-60 (true sum below 2^-124) lost bits to FP32
        // underflow: the caller takes iteration 1 again with the exact column passes
        if (!(c >= 0x1p-60) || !isfinite(c)) {
            atomicOr(flag, 1);
            return;
        }
        G_out[j] = G_in[j] + lq - (log2(c) - 64.0);
    } else {
        // COLSUM: the sums were shifted by the column maximum as the sweep rounded it
        const double M = mode == OT_SHARD_COLSUM ? (double)(float)colmax[j] : 0.0;
        if (!(c > 0.0) || !isfinite(c) || !isfinite(M)) {
            atomicOr(flag, 2);
            if (state) state[0] = 3.0;  // numeric failure: later launches do nothing
            return;
        }
        G_out[j] = G_in[j] + lq - (M + log2(c));
    }
}

// Totals of the finalize sweep: transport cost, loads rho_j, residuals, g in natural units.
__global__ void k_shard_finish(const double* __restrict__ col2, const double* __restrict__ row_err,
                               const float* __restrict__ q, int J, double mass, double inv_qmass, double eps_ln2,
                               const double* __restrict__ G, double* g_out, double* rho_out, double* summary) {
    __shared__ double sh[2][32];
    double ec = 0.0, co = 0.0;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        const double s = col2[j], r = col2[J + j];
        ec += fabs(s - (double)q[j] * inv_qmass);
        co += r;
        if (rho_out) rho_out[j] = r * mass;
        if (g_out) g_out[j] = eps_ln2 * G[j];
    }
    ec = warp_sum(ec);
    co = warp_sum(co);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = ec;
        sh[1][threadIdx.x >> 5] = co;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0, c = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            e += sh[0][w];
            c += sh[1][w];
        }
        summary[0] = c * mass;
        summary[1] = *row_err;
        summary[2] = e;
    }
}

// Sum of p (the shard's rows) and of q, in a fixed order; out[2] = 1 when an entry is not
// positive and finite.
__global__ void k_shard_mass(const float* __restrict__ p, int64_t I, const float* __restrict__ q, int J,
                             double* out) {
    __shared__ double sh[2][32];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    double sp = 0.0, sq = 0.0;
    int b = 0;
    for (int64_t i = threadIdx.x; i < I; i += blockDim.x) {
        const float x = p[i];
        b |= !(x > 0.f) || !isfinite(x);
        sp += (double)x;
    }
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        const float x = q[j];
        b |= !(x > 0.f) || !isfinite(x);
        sq += (double)x;
    }
    if (b) atomicOr(&bad, 1);
    sp = warp_sum(sp);
    sq = warp_sum(sq);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = sp;
        sh[1][threadIdx.x >> 5] = sq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[0][w];
            c += sh[1][w];
        }
        out[0] = a;
        out[1] = c;
        out[2] = bad ? 1.0 : 0.0;
    }
}

template <int TW>
struct ShardKernels {
    static const void* get(int mode) {
        switch (mode) {
            case OT_SHARD_FIRST: return (const void*)k_shard_sweep<TW, OT_SHARD_FIRST>;
            case OT_SHARD_ITER: return (const void*)k_shard_sweep<TW, OT_SHARD_ITER>;
            case OT_SHARD_COLMAX: return (const void*)k_shard_sweep<TW, OT_SHARD_COLMAX>;
            case OT_SHARD_COLSUM: return (const void*)k_shard_sweep<TW, OT_SHARD_COLSUM>;
            case OT_SHARD_FINAL: return (const void*)k_shard_sweep<TW, OT_SHARD_FINAL>;
            default: return nullptr;
        }
    }
};

}  // namespace
}  // namespace ota

using namespace ota;

extern "C" {

ot_status ot_assoc_shard_mass(ot_assoc_ctx* ctx, const float* p, int64_t I, const float* q, int64_t J, double* out,
                              void* stream) {
    if (!ctx) return OT_EINVAL;
    DeviceGuardLite guard(ctx->device);
    if (!p || !q || !out) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0 || J > INT32_MAX) return set_error(ctx, OT_EINVAL, "bad I or J");
    k_shard_mass<<<1, 512, 0, (cudaStream_t)stream>>>(p, I, q, (int)J, out);
    ctx->launches += 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OT_OK : cuda_error(ctx, e, "shard mass");
}

ot_status ot_assoc_shard_sweep(ot_assoc_ctx* ctx, int mode, const float* C, int64_t ld_c, const float* p, int64_t I,
                               int64_t J, double inv_mass, double eps, const double* G, const float* F_in,
                               float* F_out, const double* colmax, double* col_out, double* row_out,
                               double* f_out, const double* state, void* stream) {
    if (!ctx) return OT_EINVAL;
    DeviceGuardLite guard(ctx->device);
    if (mode < OT_SHARD_FIRST || mode > OT_SHARD_FINAL) return set_error(ctx, OT_EINVAL, "unknown shard mode %d", mode);
    if (!C || !p || !G || !col_out) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0) return set_error(ctx, OT_EINVAL, "bad I or J");
    if (J > 8192) return set_error(ctx, OT_EUNSUPPORTED, "J=%lld above 8192", (long long)J);
    const int64_t ld = ld_c ? ld_c : J;
    if (ld < J) return set_error(ctx, OT_EINVAL, "ld_c < J");
    if ((reinterpret_cast<uintptr_t>(C) & 15) || (ld & 3))
        return set_error(ctx, OT_EINVAL, "C must be 16-byte aligned with ld_c %% 4 == 0");
    if (mode == OT_SHARD_FIRST && !F_out) return set_error(ctx, OT_EINVAL, "F_out is required");
    if (mode != OT_SHARD_FIRST && !F_in) return set_error(ctx, OT_EINVAL, "F_in is required");
    if (mode == OT_SHARD_ITER && (!F_out || !row_out)) return set_error(ctx, OT_EINVAL, "F_out and row_out are required");
    if (mode == OT_SHARD_FINAL && !row_out) return set_error(ctx, OT_EINVAL, "row_out is required");
    if (mode == OT_SHARD_COLSUM && !colmax) return set_error(ctx, OT_EINVAL, "colmax is required");
    if (!(inv_mass > 0.0) || !std::isfinite(inv_mass)) return set_error(ctx, OT_EINVAL, "inv_mass");
    if (!(eps > 0.0) || !std::isfinite(eps)) return set_error(ctx, OT_EINVAL, "eps");
    const int J4 = (int)((J + 3) / 4);
    const int TW = J4 <= 256 ? 1 : (J4 <= 512 ? 2 : (J4 <= 1024 ? 4 : 8));
    const int nteams = SH_NW / TW;
    const void* fn = TW == 1 ? ShardKernels<1>::get(mode)
                     : TW == 2 ? ShardKernels<2>::get(mode)
                     : TW == 4 ? ShardKernels<4>::get(mode)
                               : ShardKernels<8>::get(mode);
    const int Jp = (int)round_up(J, 4);
    const int nacc = mode == OT_SHARD_FINAL ? 2 : 1;
    // two blocks an SM (what fits at these register counts); every block adds its rows'
    // column sums into one row of partials that k_shard_reduce then adds
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((I + nteams - 1) / nteams, 2LL * ctx->num_sms));
    const size_t smem = sizeof(float) * ((size_t)3 * Jp + (size_t)nteams * nacc * Jp);
    ot_status st = OT_OK;
    const size_t off_e = round_up((int64_t)sizeof(double) * nb * nacc * Jp, 256);
    char* ws = (char*)scratch(ctx, SLOT_SHARD, off_e + sizeof(double) * (size_t)nb, &st);
    if (st) return st;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(ctx, e, "shard sweep attribute");
    float k_hi, k_lo;
    split_k(LOG2E / eps, &k_hi, &k_lo);
    ShardArgs A;
    A.C = C;
    A.ld = ld;
    A.p = p;
    A.I = I;
    A.J = (int)J;
    A.Jp = Jp;
    A.inv_mass = (float)inv_mass;
    A.k_hi = k_hi;
    A.k_lo = k_lo;
    A.eps_ln2 = eps * 0.69314718055994530942;
    A.G = G;
    A.F_in = reinterpret_cast<const float2*>(F_in);
    A.F_out = reinterpret_cast<float2*>(F_out);
    A.colmax = colmax;
    A.part = (double*)ws;
    A.epart = (double*)(ws + off_e);
    A.f_out = mode == OT_SHARD_FINAL ? f_out : nullptr;
    A.state = state;
    cudaStream_t s = (cudaStream_t)stream;
    void* args[] = {&A};
    e = cudaLaunchKernel(fn, dim3(nb), dim3(SH_NW * 32), args, smem, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "shard sweep");
    const int n = nacc * (int)J;
    k_shard_reduce<<<(n + 31) / 32, SR_WARPS * 32, 0, s>>>(A.part, A.epart, nb, nacc, Jp, (int)J,
                                                   mode == OT_SHARD_COLMAX ? 1 : 0, col_out,
                                                   (mode == OT_SHARD_ITER || mode == OT_SHARD_FINAL) ? row_out : nullptr,
                                                   state);
    ctx->launches += 2;
    e = cudaGetLastError();
    return e == cudaSuccess ? OT_OK : cuda_error(ctx, e, "shard reduce");
}

ot_status ot_assoc_shard_update(ot_assoc_ctx* ctx, int mode, const float* q, int64_t J, double inv_qmass,
                                const double* col, const double* colmax, const double* G_in, double* G_out,
                                int32_t* flag, const double* err, int32_t iter, double tol_stop, int32_t max_iter,
                                double* state, void* stream) {
    if (!ctx) return OT_EINVAL;
    DeviceGuardLite guard(ctx->device);
    if (mode != OT_SHARD_FIRST && mode != OT_SHARD_ITER && mode != OT_SHARD_COLSUM)
        return set_error(ctx, OT_EINVAL, "shard update mode must be FIRST, ITER or COLSUM");
    if (!q || !col || !G_in || !G_out || !flag) return set_error(ctx, OT_EINVAL, "null pointer");
    if (mode == OT_SHARD_COLSUM && !colmax) return set_error(ctx, OT_EINVAL, "colmax is required");
    if (J <= 0 || J > 8192) return set_error(ctx, OT_EINVAL, "bad J");
    if (!(inv_qmass > 0.0) || !std::isfinite(inv_qmass)) return set_error(ctx, OT_EINVAL, "inv_qmass");
    if (state && mode == OT_SHARD_ITER && (!err || iter < 2 || max_iter < 1 || !(tol_stop >= 0.0)))
        return set_error(ctx, OT_EINVAL, "a loop state needs err, iter >= 2, max_iter >= 1 and tol_stop >= 0");
    k_shard_update<<<(int)((J + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        mode, q, (int)J, inv_qmass, col, colmax, G_in, G_out, flag, err, (int)iter, tol_stop, (int)max_iter, state);
    ctx->launches += 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OT_OK : cuda_error(ctx, e, "shard update");
}

ot_status ot_assoc_shard_finish(ot_assoc_ctx* ctx, const double* col2, const double* row_err, const float* q,
                                int64_t J, double mass, double inv_qmass, double eps, const double* G, double* g_out,
                                double* rho_out, double* summary, void* stream) {
    if (!ctx) return OT_EINVAL;
    DeviceGuardLite guard(ctx->device);
    if (!col2 || !row_err || !q || !G || !summary) return set_error(ctx, OT_EINVAL, "null pointer");
    if (J <= 0 || J > 8192) return set_error(ctx, OT_EINVAL, "bad J");
    if (!(mass > 0.0) || !std::isfinite(mass) || !(inv_qmass > 0.0) || !std::isfinite(inv_qmass))
        return set_error(ctx, OT_EINVAL, "mass");
    if (!(eps > 0.0) || !std::isfinite(eps)) return set_error(ctx, OT_EINVAL, "eps");
    k_shard_finish<<<1, 512, 0, (cudaStream_t)stream>>>(col2, row_err, q, (int)J, mass, inv_qmass,
                                                        eps * 0.69314718055994530942, G, g_out, rho_out, summary);
    ctx->launches += 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OT_OK : cuda_error(ctx, e, "shard finish");
}

}  // extern "C"
