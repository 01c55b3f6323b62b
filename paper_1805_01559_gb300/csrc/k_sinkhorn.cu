// Entropic-OT Sinkhorn solver, FP32 log domain (Algorithm 1 of the paper, Sec. III-B).
//
// Notation (log2 units, so every exponential is one MUFU.EX2):
//   k      = log2(e) / eps, split k = k_hi + k_lo (two FP32 numbers, ~2^-48 relative).
//   G_j    = g_j * k                    column potential (b_j = 2^G_j)
//   F'_i   = f_i * k - log2 p_i         row potential relative to the row mass
//   t_ij   = 2^(F'_i + G_j - k C_ij)    = pi_ij / p_i of the current plan
// Iteration 1 is the exact log-domain step from b = 1 (or a warm-start b): a row
// log-sum-exp with the row maximum factored out, then a column log-sum-exp with an
// online (max, sum) pair per column, so no column can underflow however far the
// starting potentials are.  From then on every plan pi^(k-1) has exact columns
// (sum q_j <= 1) and rows >= p_i * min q, so iteration k can work directly on
// t_ij = pi^(k-1)_ij / p_i: one read of C and ONE exp per cell give
//   a-update:  r_i = sum_j t_ij,  F'_i <- F'_i - log2 r_i       (Alg. 1, a-line)
//   b-update:  s_j = sum_i t_ij p^_i / r_i,  G_j <- G_j + log2 q^_j - log2 s_j
//                                                                (Alg. 1, b-line)
// and r_i also yields the row residual of pi^(k-1) for the stopping test, one sweep
// late: when it passes, the previous iterate (kept in the other F buffer) is
// returned, which is the iterate Algorithm 1's loop test examines.
// Row potentials are kept in FP64 and enter each cell as an FP32 hi/lo pair whose large
// part cancels against C k_hi inside an exact FMA product; column potentials enter as the
// FP32 value G_used and are updated in FP64 from that value, so rounding never accumulates.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "ot_common.cuh"
#include "ot_internal.h"

namespace ota {

static constexpr int NT = 256;    // threads per CTA, sweep kernels
static constexpr int NT_F = 512;  // threads per CTA, finalize kernel (one team per row)
static constexpr double LN2 = 0.69314718055994530942;
static constexpr double LOG2E = 1.44269504088896340736;

enum : int { DEV_ENUMERIC = -7 };

struct DevScalars {
    double sp, sq;          // sums of the caller's p and q
    double inv_sp, inv_sq;
    float inv_sp_f;
    int status;
};

struct LoopState {
    unsigned bar;
    int status;
    int iters;
    int converged;
    double err;
};

template <int TW, int VPT>
__device__ __forceinline__ void load_G(const double* __restrict__ G, int J, int tl, float4 (&g)[VPT]) {
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int col = 4 * (tl + 32 * TW * v);
#pragma unroll
        for (int c = 0; c < 4; ++c) comp(g[v], c) = (col + c < J) ? (float)G[col + c] : 0.0f;
    }
}

// Cell exponent x = F + G - k C in log2 units, with F = F_hi + F_lo (a float pair holding
// the FP64 row potential) and k = k_hi + k_lo.  The exact FMA product cancels the large
// parts F_hi - C k_hi first, so the only roundings happen at the magnitude of |G| and |x|,
// however large k C and F are on the support.  k_lo > 0 always (see split_k), so a +inf
// cost (masked column, forbidden link) gives -inf and never inf - inf.
__device__ __forceinline__ float expo(float F_hi, float F_lo_plus_G, float c, float k_hi, float k_lo) {
    return fmaf(-c, k_hi, F_hi) + fmaf(-c, k_lo, F_lo_plus_G);
}

__device__ __forceinline__ void split_f(double F, float* hi, float* lo) {
    *hi = (float)F;
    *lo = (float)(F - (double)*hi);
}

// k = k_hi + k_lo with k_hi rounded down and 0 < k_lo <= ulp(k_hi): the low part is never
// zero or negative, so -inf * k_lo = -inf and no inf - inf can occur for C = +inf.
static void split_k(double k, float* hi, float* lo) {
    float h = (float)k;
    if ((double)h >= k) h = nextafterf(h, 0.0f);
    float l = (float)(k - (double)h);
    if (!(l > 0.0f)) l = 1.4e-45f;  // smallest subnormal; adds nothing measurable
    *hi = h;
    *lo = l;
}

// ------------------------------------------------------------------------------------------
// prep: sums and validity of the marginals, starting column potentials.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) sk_prep(const float* __restrict__ p, const float* __restrict__ q,
                                                int64_t I, int J, const double* __restrict__ g_warm,
                                                double k, const unsigned long long* __restrict__ input_bad,
                                                DevScalars* sc, double* G) {
    __shared__ double sh_p[32], sh_q[32];
    __shared__ int sh_bad;
    if (threadIdx.x == 0) sh_bad = 0;
    __syncthreads();
    double sp = 0.0, sq = 0.0;
    int bad = 0;
    for (int64_t i = threadIdx.x; i < I; i += blockDim.x) {
        const float v = p[i];
        bad |= !(v > 0.0f) || !isfinite(v);
        sp += (double)v;
    }
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        const float v = q[j];
        bad |= !(v > 0.0f) || !isfinite(v);
        sq += (double)v;
        G[j] = g_warm ? g_warm[j] * k : 0.0;
        if (g_warm && !isfinite(g_warm[j])) bad = 1;
    }
    sp = warp_sum(sp);
    sq = warp_sum(sq);
    if ((threadIdx.x & 31) == 0) {
        sh_p[threadIdx.x >> 5] = sp;
        sh_q[threadIdx.x >> 5] = sq;
    }
    if (bad) atomicOr(&sh_bad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        double tp = 0.0, tq = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            tp += sh_p[w];
            tq += sh_q[w];
        }
        int st = DEV_OK;
        if (sh_bad || !(fabs(tp - tq) <= 1e-5 * tp) || (input_bad && *input_bad)) st = DEV_EINVAL;
        sc->sp = tp;
        sc->sq = tq;
        sc->inv_sp = 1.0 / tp;
        sc->inv_sq = 1.0 / tq;
        sc->inv_sp_f = (float)(1.0 / tp);
        sc->status = st;
    }
}

// ------------------------------------------------------------------------------------------
// Iteration 1, rows: exact row LSE, then per-column online (max, sum) of log2 pi^(1/2).
// ------------------------------------------------------------------------------------------
template <int TW, int VPT>
__global__ void __launch_bounds__(NT) sk_init_rows(const float* __restrict__ C, int64_t ld, int64_t I,
                                                   int J, int Jp, const float* __restrict__ p,
                                                   const DevScalars* __restrict__ sc,
                                                   const double* __restrict__ G0, double* __restrict__ F1,
                                                   float2* __restrict__ part, float k_hi, float k_lo) {
    constexpr int TT = 32 * TW, NTEAMS = NT / TT;
    extern __shared__ float4 dyn_smem[];
    float2* comb = reinterpret_cast<float2*>(dyn_smem);  // [NTEAMS][Jp]
    __shared__ float red[2 * NTEAMS * TW];
    const Team<TW> tm;
    if (sc->status != DEV_OK) return;
    const int nb = gridDim.x, b = blockIdx.x;
    const int64_t r0 = I * b / nb, r1 = I * (b + 1) / nb;
    float4 g[VPT], M[VPT], S[VPT];
    load_G<TW, VPT>(G0, J, tm.tl, g);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        M[v] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
        S[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float inv_sp = sc->inv_sp_f;
    int par = 0;
    for (int64_t i = r0 + tm.team; i < r1; i += NTEAMS) {
        float4 x[VPT];
        load_row<TW, VPT>(C + i * ld, J, tm.tl, x);
        // row maximum of y = G0 - k C (approximate values suffice for the shift)
        float m = -INFINITY;
#pragma unroll
        for (int v = 0; v < VPT; ++v)
#pragma unroll
            for (int c = 0; c < 4; ++c) m = fmaxf(m, fmaf(-comp(x[v], c), k_hi, comp(g[v], c)));
        m = team_reduce<TW, float, true>(m, red, NTEAMS, tm, par);
        // z = y - m formed with the large parts cancelled by the exact product
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < VPT; ++v)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float z = expo(-m, comp(g[v], c), comp(x[v], c), k_hi, k_lo);
                comp(x[v], c) = z;
                s += ex2(z);
            }
        s = team_reduce<TW, float, false>(s, red, NTEAMS, tm, par);
        const float ls = log2f(s);
        if (tm.tl == 0) F1[i] = -((double)m + (double)ls);   // F'^1 = -LSE2_j(y)
        const float cst = log2f(__ldg(p + i) * inv_sp) - ls;
#pragma unroll
        for (int v = 0; v < VPT; ++v)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float u = comp(x[v], c) + cst;  // log2 pi^(1/2)_ij = z - log2 s + log2 p^
                float& Mc = comp(M[v], c);
                float& Sc = comp(S[v], c);
                if (u > Mc) {
                    Sc = fmaf(Sc, ex2(Mc - u), 1.0f);
                    Mc = u;
                } else if (u > -INFINITY) {
                    Sc += ex2(u - Mc);
                }
            }
    }
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int col = 4 * (tm.tl + TT * v);
        if (col < Jp)
#pragma unroll
            for (int c = 0; c < 4; ++c) comb[tm.team * Jp + col + c] = make_float2(comp(M[v], c), comp(S[v], c));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < J; j += NT) {
        float m = comb[j].x, s = comb[j].y;
        for (int t = 1; t < NTEAMS; ++t) {
            const float2 o = comb[t * Jp + j];
            lse2_merge(m, s, o.x, o.y);
        }
        part[(int64_t)b * Jp + j] = make_float2(m, s);
    }
}

// Iteration 1, columns: G^1_j = G^0_j + log2 q^_j - log2(column sum of pi^(1/2)).
__global__ void sk_init_cols(const float2* __restrict__ part, int nb, int Jp, int J,
                             const float* __restrict__ q, DevScalars* sc, double* G) {
    if (sc->status != DEV_OK) return;
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = w; j < J; j += nw) {
        float m = -INFINITY;
        for (int bb = lane; bb < nb; bb += 32) m = fmaxf(m, part[(int64_t)bb * Jp + j].x);
        m = warp_max(m);
        double s = 0.0;
        if (m > -INFINITY)
            for (int bb = lane; bb < nb; bb += 32) {
                const float2 v = part[(int64_t)bb * Jp + j];
                if (v.x > -INFINITY) s += (double)v.y * (double)ex2(v.x - m);
            }
        s = warp_sum(s);
        if (lane == 0) {
            if (!(s > 0.0) || !isfinite(s)) {
                atomicCAS(&sc->status, DEV_OK, DEV_ENUMERIC);
            } else {
                const double Gu = (double)(float)G[j];
                const double qh = (double)q[j] * sc->inv_sq;
                G[j] = Gu + log2(qh) - ((double)m + log2(s));
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Iterations 2.. : persistent cooperative kernel, one read of C and one ex2 per cell.
// ------------------------------------------------------------------------------------------
struct LoopParams {
    const float* C;
    int64_t ld;
    int64_t I;
    int J;
    int Jp;
    const float* p;
    const float* q;
    const DevScalars* sc;
    double* F0;
    double* F1;
    double* G;
    float* colpart;   // [nb][Jp]
    double* errpart;  // [nb]
    LoopState* st;
    float k_hi, k_lo;
    double tol;
    int max_iter;
    long long spin;
};

template <int TW, int VPT>
__global__ void __launch_bounds__(NT, 2) sk_loop(LoopParams P) {
    constexpr int TT = 32 * TW, NTEAMS = NT / TT;
    extern __shared__ float4 dyn_smem[];
    float* comb = reinterpret_cast<float*>(dyn_smem);  // [NTEAMS][Jp]
    __shared__ float red[2 * NTEAMS * TW];
    __shared__ double errs[NTEAMS];
    __shared__ int s_stop;
    const Team<TW> tm;
    if (P.sc->status != DEV_OK) return;
    const int J = P.J, Jp = P.Jp;
    const int nb = gridDim.x, b = blockIdx.x;
    const int warp = threadIdx.x >> 5;
    const int64_t r0 = P.I * b / nb, r1 = P.I * (b + 1) / nb;
    const float inv_sp = P.sc->inv_sp_f;
    float4 g[VPT];
    load_G<TW, VPT>(P.G, J, tm.tl, g);
    unsigned gen = 0;
    for (int s = 2;; ++s) {
        const double* __restrict__ Fold = (s & 1) ? P.F0 : P.F1;  // F^(s-1) lives in buffer (s-1)&1
        double* __restrict__ Fnew = (s & 1) ? P.F1 : P.F0;
        float4 acc[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        double errt = 0.0;
        int par = 0;
        for (int64_t i = r0 + tm.team; i < r1; i += NTEAMS) {
            float4 x[VPT];
            load_row<TW, VPT>(P.C + i * P.ld, J, tm.tl, x);
            const double Fd = Fold[i];
            float Fh, Fl;
            split_f(Fd, &Fh, &Fl);
            float rs = 0.f;
#pragma unroll
            for (int v = 0; v < VPT; ++v)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float t = ex2(expo(Fh, Fl + comp(g[v], c), comp(x[v], c), P.k_hi, P.k_lo));
                    comp(x[v], c) = t;
                    rs += t;
                }
            rs = team_reduce<TW, float, false>(rs, red, NTEAMS, tm, par);
            const float ph = __ldg(P.p + i) * inv_sp;
            if (tm.tl == 0) {
                Fnew[i] = Fd - (double)log2_rel(rs);
                errt += (double)ph * fabs((double)rs - 1.0);
            }
            const float d = ph / rs;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                acc[v].x = fmaf(x[v].x, d, acc[v].x);
                acc[v].y = fmaf(x[v].y, d, acc[v].y);
                acc[v].z = fmaf(x[v].z, d, acc[v].z);
                acc[v].w = fmaf(x[v].w, d, acc[v].w);
            }
        }
        // CTA combine of the column partials, teams in a fixed order.
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int col = 4 * (tm.tl + TT * v);
            if (col < Jp) *reinterpret_cast<float4*>(comb + tm.team * Jp + col) = acc[v];
        }
        if (tm.tl == 0) errs[tm.team] = errt;
        __syncthreads();
        for (int j = threadIdx.x; j < J; j += NT) {
            float sum = comb[j];
            for (int t = 1; t < NTEAMS; ++t) sum += comb[t * Jp + j];
            P.colpart[(int64_t)b * Jp + j] = sum;
        }
        if (threadIdx.x == 0) {
            double e = errs[0];
            for (int t = 1; t < NTEAMS; ++t) e += errs[t];
            P.errpart[b] = e;
        }
        if (!grid_barrier(&P.st->bar, (unsigned)nb * ++gen, &P.st->status, P.spin)) return;
        // Loop test on pi^(s-1): every CTA forms the same total in the same order.
        if (warp == 0) {
            double e = 0.0;
            for (int bb = tm.lane; bb < nb; bb += 32) e += P.errpart[bb];
            e = warp_sum(e);
            if (tm.lane == 0) {
                const int stop = (e <= P.tol) || (s - 1 >= P.max_iter);
                s_stop = stop;
                if (stop && b == 0) {
                    P.st->iters = s - 1;
                    P.st->err = e;
                    P.st->converged = (e <= P.tol);
                }
            }
        }
        __syncthreads();
        if (s_stop) return;
        // b-update, one warp per column.
        {
            const int gw = b * (NT / 32) + warp, nw = nb * (NT / 32);
            for (int j = gw; j < J; j += nw) {
                double sum = 0.0;
                for (int bb = tm.lane; bb < nb; bb += 32) sum += (double)P.colpart[(int64_t)bb * Jp + j];
                sum = warp_sum(sum);
                if (tm.lane == 0) {
                    if (!(sum > 0.0) || !isfinite(sum)) {
                        atomicCAS(&P.st->status, DEV_OK, DEV_ENUMERIC);
                    } else {
                        const double Gu = (double)(float)P.G[j];
                        const double qh = (double)__ldg(P.q + j) * P.sc->inv_sq;
                        P.G[j] = Gu + log2(qh) - log2(sum);
                    }
                }
            }
        }
        if (!grid_barrier(&P.st->bar, (unsigned)nb * ++gen, &P.st->status, P.spin)) return;
        load_G<TW, VPT>(P.G, J, tm.tl, g);
    }
}

// ------------------------------------------------------------------------------------------
// Finalize: plan, potentials in natural units, FP64 reductions of marginals, cost and loads.
// One team of NT_F threads per row; per-thread column accumulators in FP64.
// ------------------------------------------------------------------------------------------
struct FinParams {
    const float* C;
    int64_t ld;
    int64_t I;
    int J;
    int Jp;
    const float* p;
    const DevScalars* sc;
    const double* F0;
    const double* F1;
    const LoopState* st;
    const double* G;
    float k_hi, k_lo;
    double eps_ln2;
    float* pi;
    int64_t pi_ld;
    double* f_out;
    double2* fpart;   // [nb][Jp] (sum p^ t, sum p^ C t)
    double* epart;    // [nb][2] (row residual, cost)
};

template <int VPT>
__global__ void __launch_bounds__(NT_F) sk_finalize(FinParams P) {
    constexpr int TW = NT_F / 32;
    __shared__ double redd[2 * TW];
    const Team<TW> tm;
    if (P.sc->status != DEV_OK || P.st->status != DEV_OK) return;
    const int J = P.J;
    const int nb = gridDim.x, b = blockIdx.x;
    const int64_t r0 = P.I * b / nb, r1 = P.I * (b + 1) / nb;
    const double* __restrict__ F = (P.st->iters & 1) ? P.F1 : P.F0;
    float4 g[VPT];
    load_G<TW, VPT>(P.G, J, tm.tl, g);
    double apI[VPT * 4], arho[VPT * 4];
#pragma unroll
    for (int k = 0; k < VPT * 4; ++k) apI[k] = arho[k] = 0.0;
    double errt = 0.0, costt = 0.0;
    int par = 0;
    for (int64_t i = r0; i < r1; ++i) {
        float4 x[VPT];
        load_row<TW, VPT>(P.C + i * P.ld, J, tm.tl, x);
        const double Fd = F[i];
        float Fh, Fl;
        split_f(Fd, &Fh, &Fl);
        const float pi_ = __ldg(P.p + i);
        const double ph = (double)pi_ * P.sc->inv_sp;
        float rs = 0.f, cs = 0.f;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int col = 4 * (tm.tl + NT_F * v);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float cost = comp(x[v], c);
                const float t = ex2(expo(Fh, Fl + comp(g[v], c), cost, P.k_hi, P.k_lo));
                const float ct = t > 0.f ? cost * t : 0.f;
                rs += t;
                cs += ct;
                apI[v * 4 + c] = fma(ph, (double)t, apI[v * 4 + c]);
                arho[v * 4 + c] = fma(ph, (double)ct, arho[v * 4 + c]);
                if (P.pi && col + c < J) P.pi[i * P.pi_ld + col + c] = pi_ * t;
            }
        }
        const double rsd = team_reduce<TW, double, false>((double)rs, redd, 1, tm, par);
        const double csd = team_reduce<TW, double, false>((double)cs, redd, 1, tm, par);
        if (tm.tl == 0) {
            errt += ph * fabs(rsd - 1.0);
            costt += ph * csd;
            P.f_out[i] = P.eps_ln2 * (Fd + log2((double)pi_));
        }
    }
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int col = 4 * (tm.tl + NT_F * v);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (col + c < J) P.fpart[(int64_t)b * P.Jp + col + c] = make_double2(apI[v * 4 + c], arho[v * 4 + c]);
    }
    if (threadIdx.x == 0) {
        P.epart[2 * b] = errt;
        P.epart[2 * b + 1] = costt;
    }
}

__global__ void sk_finalize_cols(const double2* __restrict__ fpart, int nb, int Jp, int J,
                                 const float* __restrict__ q, const DevScalars* sc,
                                 const LoopState* st, const double* __restrict__ G, double eps_ln2,
                                 double* g_out, double* rrh_load, double* colerr) {
    if (sc->status != DEV_OK || st->status != DEV_OK) return;
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = w; j < J; j += nw) {
        double s = 0.0, r = 0.0;
        for (int bb = lane; bb < nb; bb += 32) {
            const double2 v = fpart[(int64_t)bb * Jp + j];
            s += v.x;
            r += v.y;
        }
        s = warp_sum(s);
        r = warp_sum(r);
        if (lane == 0) {
            colerr[j] = fabs(s - (double)q[j] * sc->inv_sq);
            if (rrh_load) rrh_load[j] = r * sc->sp;
            g_out[j] = eps_ln2 * G[j];
        }
    }
}

__global__ void sk_summary(const double* __restrict__ epart, int nb, const double* __restrict__ colerr,
                           int J, const DevScalars* sc, const LoopState* st, SolveSummary* out) {
    __shared__ double sh[3][32];
    double er = 0.0, co = 0.0, ec = 0.0;
    const bool ok = sc->status == DEV_OK && st->status == DEV_OK;
    if (ok) {
        for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) {
            er += epart[2 * bb];
            co += epart[2 * bb + 1];
        }
        for (int j = threadIdx.x; j < J; j += blockDim.x) ec += colerr[j];
    }
    er = warp_sum(er);
    co = warp_sum(co);
    ec = warp_sum(ec);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = er;
        sh[1][threadIdx.x >> 5] = co;
        sh[2][threadIdx.x >> 5] = ec;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0, e = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[0][w];
            c += sh[1][w];
            e += sh[2][w];
        }
        out->err_row = a;
        out->err_col = e;
        out->cost = c * sc->sp;
        out->err_loop = st->err;
        out->iters = st->iters;
        out->converged = st->converged;
        out->status = sc->status != DEV_OK ? sc->status : st->status;
        out->absorptions = 0;
    }
}

// ------------------------------------------------------------------------------------------
// Host launcher.
// ------------------------------------------------------------------------------------------
namespace {

struct Kernels {
    const void* init_rows;
    const void* loop;
    int tw, vpt;
};

template <int TW, int VPT>
Kernels kernels_for() {
    return Kernels{(const void*)sk_init_rows<TW, VPT>, (const void*)sk_loop<TW, VPT>, TW, VPT};
}

bool pick_kernels(int J, Kernels* k) {
    const int J4 = (J + 3) / 4;
    if (J4 <= 32) *k = kernels_for<1, 1>();
    else if (J4 <= 64) *k = kernels_for<1, 2>();
    else if (J4 <= 128) *k = kernels_for<1, 4>();
    else if (J4 <= 256) *k = kernels_for<1, 8>();
    else if (J4 <= 512) *k = kernels_for<2, 8>();
    else if (J4 <= 1024) *k = kernels_for<4, 8>();
    else if (J4 <= 2048) *k = kernels_for<8, 8>();
    else return false;
    return true;
}

const void* pick_finalize(int J) {
    const int J4 = (J + 3) / 4;
    if (J4 <= NT_F) return (const void*)sk_finalize<1>;
    if (J4 <= 2 * NT_F) return (const void*)sk_finalize<2>;
    if (J4 <= 4 * NT_F) return (const void*)sk_finalize<4>;
    return nullptr;
}

}  // namespace

ot_status launch_solve_f32(ot_assoc_ctx* ctx, const SolveArgs& a, SolveSummary* sum_host) {
    ot_status st = OT_OK;
    const int J = a.J;
    const int64_t I = a.I;
    const int Jp = (int)round_up(J, 4);
    Kernels kk;
    const void* kfin = pick_finalize(J);
    if (!pick_kernels(J, &kk) || !kfin) return set_error(ctx, OT_EUNSUPPORTED, "J=%d above 8192", J);
    const int nteams = NT / (32 * kk.tw);
    cudaError_t e;

    // Grid sizes.
    const size_t smem_loop = (size_t)nteams * Jp * sizeof(float);
    const size_t smem_init = (size_t)nteams * Jp * sizeof(float2);
    for (const void* fn : {kk.loop, kk.init_rows}) {
        const size_t sm = fn == kk.loop ? smem_loop : smem_init;
        if (sm > 48 * 1024) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return cuda_error(ctx, e, "cudaFuncSetAttribute");
        }
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kk.loop, NT, smem_loop);
    if (e != cudaSuccess) return cuda_error(ctx, e, "occupancy");
    if (occ < 1) return set_error(ctx, OT_EUNSUPPORTED, "solver kernel does not fit on an SM");
    const int64_t rows_per_team_min = 8;
    int64_t want = (I + (int64_t)nteams * rows_per_team_min - 1) / ((int64_t)nteams * rows_per_team_min);
    const int nb_loop = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)occ * ctx->num_sms));
    int occ_i = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_i, kk.init_rows, NT, smem_init);
    if (e != cudaSuccess) return cuda_error(ctx, e, "occupancy");
    const int nb_init = (int)std::max<int64_t>(
        1, std::min<int64_t>((I + nteams - 1) / nteams, (int64_t)std::max(occ_i, 1) * ctx->num_sms));
    const int nb_fin = (int)std::max<int64_t>(1, std::min<int64_t>(I, (int64_t)4 * ctx->num_sms));
    const int nb_part = std::max(std::max(nb_loop, nb_init), nb_fin);

    // Scratch.
    double* F = (double*)scratch(ctx, SLOT_F, sizeof(double) * 2 * (size_t)I, &st);
    if (st) return st;
    double* G = (double*)scratch(ctx, SLOT_G, sizeof(double) * (size_t)Jp, &st);
    if (st) return st;
    void* colpart = scratch(ctx, SLOT_COLPART, sizeof(double2) * (size_t)nb_part * Jp, &st);
    if (st) return st;
    double* errpart = (double*)scratch(ctx, SLOT_ERRPART, sizeof(double) * 2 * (size_t)nb_part, &st);
    if (st) return st;
    char* state = (char*)scratch(ctx, SLOT_STATE, 4096 + sizeof(double) * (size_t)Jp, &st);
    if (st) return st;
    DevScalars* sc = (DevScalars*)state;
    LoopState* ls = (LoopState*)(state + 256);
    SolveSummary* summ = (SolveSummary*)(state + 512);
    double* colerr = (double*)(state + 4096);
    SolveSummary* hsum = (SolveSummary*)host_staging(ctx, sizeof(SolveSummary), &st);
    if (st) return st;

    const double k = LOG2E / a.eps;
    float k_hi, k_lo;
    split_k(k, &k_hi, &k_lo);
    cudaStream_t s = a.stream;

    ctx->last_timings.valid = 0;
    timing_mark(ctx, 0, s);
    e = cudaMemsetAsync(state, 0, 1024, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "memset");
    sk_prep<<<1, 1024, 0, s>>>(a.p, a.q, I, J, a.warm_start ? a.out->g : nullptr, k, a.input_bad, sc, G);
    {
        double* F1 = F + I;
        void* args[] = {(void*)&a.C, (void*)&a.ld, (void*)&I,       (void*)&J,
                        (void*)&Jp,  (void*)&a.p,  (void*)&sc,      (void*)&G,
                        (void*)&F1,  &colpart,     (void*)&k_hi,    (void*)&k_lo};
        e = cudaLaunchKernel(kk.init_rows, dim3(nb_init), dim3(NT), args, smem_init, s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "init_rows launch");
    }
    sk_init_cols<<<(J + 7) / 8, 256, 0, s>>>((const float2*)colpart, nb_init, Jp, J, a.q, sc, G);

    LoopParams P;
    P.C = a.C;
    P.ld = a.ld;
    P.I = I;
    P.J = J;
    P.Jp = Jp;
    P.p = a.p;
    P.q = a.q;
    P.sc = sc;
    P.F0 = F;
    P.F1 = F + I;
    P.G = G;
    P.colpart = (float*)colpart;
    P.errpart = errpart;
    P.st = ls;
    P.k_hi = k_hi;
    P.k_lo = k_lo;
    P.tol = a.tol;
    P.max_iter = a.max_iter;
    P.spin = ctx->spin_limit;
    timing_mark(ctx, 1, s);
    {
        void* args[] = {&P};
        e = cudaLaunchCooperativeKernel(kk.loop, dim3(nb_loop), dim3(NT), args, smem_loop, s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "cooperative solver launch");
    }
    timing_mark(ctx, 2, s);

    FinParams Q;
    Q.C = a.C;
    Q.ld = a.ld;
    Q.I = I;
    Q.J = J;
    Q.Jp = Jp;
    Q.p = a.p;
    Q.sc = sc;
    Q.F0 = F;
    Q.F1 = F + I;
    Q.st = ls;
    Q.G = G;
    Q.k_hi = k_hi;
    Q.k_lo = k_lo;
    Q.eps_ln2 = a.eps * LN2;
    Q.pi = a.out->pi;
    Q.pi_ld = a.out->pi_ld > 0 ? a.out->pi_ld : J;
    Q.f_out = a.out->f;
    Q.fpart = (double2*)colpart;
    Q.epart = errpart;
    {
        void* args[] = {&Q};
        e = cudaLaunchKernel(kfin, dim3(nb_fin), dim3(NT_F), args, 0, s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "finalize launch");
    }
    sk_finalize_cols<<<(J + 15) / 16, 512, 0, s>>>((const double2*)colpart, nb_fin, Jp, J, a.q, sc, ls, G,
                                                   a.eps * LN2, a.out->g, a.out->rrh_load, colerr);
    sk_summary<<<1, 256, 0, s>>>(errpart, nb_fin, colerr, J, sc, ls, summ);
    timing_mark(ctx, 3, s);
    ctx->launches += 8;
    e = cudaMemcpyAsync(hsum, summ, sizeof(SolveSummary), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "summary copy");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "solve");
    *sum_host = *hsum;
    timing_collect(ctx, hsum->iters);
    return OT_OK;
}

}  // namespace ota

// ------------------------------------------------------------------------------------------
// Solve without any allocation: the same kernels as launch_solve_f32, with every scratch
// buffer carved out of one file-scope device array instead of context memory.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree at solve time -- a radio
// scheduler that re-associates devices every few milliseconds and cannot afford the device
// synchronisation or unbounded latency those calls can bring, or a host process that runs
// under a fixed memory pool and has no room to grow one.  The array is part of the loaded
// library image: every GPU that loads the library holds NOALLOC_BYTES of it until exit.
// ------------------------------------------------------------------------------------------
namespace ota {

static constexpr size_t NOALLOC_BYTES = size_t(8) << 20;  // 8 MiB
static constexpr int64_t NOALLOC_MAX_I = 131072;
static constexpr int NOALLOC_MAX_J = 1024;
static constexpr int NOALLOC_MAX_CTAS = 320;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Byte offsets inside g_noalloc_scratch (all multiples of 256).
static constexpr size_t NA_STATE = 0;                                    // DevScalars/LoopState/summary
static constexpr size_t NA_COLERR = 4096;                                // Jp doubles
static constexpr size_t NA_G = NA_COLERR + 8 * NOALLOC_MAX_J;            // Jp doubles
static constexpr size_t NA_ERRPART = NA_G + 8 * NOALLOC_MAX_J;           // 2 * CTAs doubles
static constexpr size_t NA_COLPART = NA_ERRPART + 16 * NOALLOC_MAX_CTAS; // CTAs * Jp double2
static constexpr size_t NA_F = NA_COLPART + 16 * (size_t)NOALLOC_MAX_CTAS * NOALLOC_MAX_J;
static constexpr size_t NA_END = NA_F + 16 * (size_t)NOALLOC_MAX_I;      // 2 * I doubles
static_assert(NA_END <= NOALLOC_BYTES, "no-allocation scratch layout does not fit");
static_assert(NA_COLPART % 256 == 0 && NA_F % 256 == 0, "alignment");

// Device address of g_noalloc_scratch per device, looked up once with that device current.
static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_ptr[128];

static ot_status noalloc_base(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 128) return OT_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return OT_ECUDA;
        }
        g_noalloc_ptr[dev] = (unsigned char*)p;
    }
    *out = g_noalloc_ptr[dev];
    return OT_OK;
}

static ot_status noalloc_solve(const SolveArgs& a, SolveSummary* sum_host) {
    const int J = a.J;
    const int64_t I = a.I;
    const int Jp = (int)round_up(J, 4);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return OT_ECUDA;
    }
    unsigned char* base = nullptr;
    ot_status st = noalloc_base(dev, &base);
    if (st) return st;
    Kernels kk;
    const void* kfin = pick_finalize(J);
    if (!pick_kernels(J, &kk) || !kfin) return OT_EUNSUPPORTED;
    const int nteams = NT / (32 * kk.tw);
    const size_t smem_loop = (size_t)nteams * Jp * sizeof(float);
    const size_t smem_init = (size_t)nteams * Jp * sizeof(float2);
    cudaError_t e;
    for (const void* fn : {kk.loop, kk.init_rows}) {
        const size_t sm = fn == kk.loop ? smem_loop : smem_init;
        if (sm > 48 * 1024 &&
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
            cudaGetLastError();
            return OT_ECUDA;
        }
    }
    int occ = 0, occ_i = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kk.loop, NT, smem_loop) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_i, kk.init_rows, NT, smem_init) != cudaSuccess) {
        cudaGetLastError();
        return OT_ECUDA;
    }
    if (occ < 1) return OT_EUNSUPPORTED;
    const int64_t cap = NOALLOC_MAX_CTAS;
    const int64_t want = (I + (int64_t)nteams * 8 - 1) / ((int64_t)nteams * 8);
    const int nb_loop = (int)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)occ * nsm, cap}));
    const int nb_init = (int)std::max<int64_t>(
        1, std::min<int64_t>({(I + nteams - 1) / nteams, (int64_t)std::max(occ_i, 1) * nsm, cap}));
    const int nb_fin = (int)std::max<int64_t>(1, std::min<int64_t>({I, (int64_t)4 * nsm, cap}));

    char* state = (char*)(base + NA_STATE);
    DevScalars* sc = (DevScalars*)state;
    LoopState* ls = (LoopState*)(state + 256);
    SolveSummary* summ = (SolveSummary*)(state + 512);
    double* colerr = (double*)(base + NA_COLERR);
    double* G = (double*)(base + NA_G);
    double* errpart = (double*)(base + NA_ERRPART);
    void* colpart = (void*)(base + NA_COLPART);
    double* F = (double*)(base + NA_F);

    const double k = LOG2E / a.eps;
    float k_hi, k_lo;
    split_k(k, &k_hi, &k_lo);
    cudaStream_t s = a.stream;
    // The state words must start at zero on every call (the array keeps the last call's data).
    e = cudaMemsetAsync(state, 0, 1024, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return OT_ECUDA;
    }
    sk_prep<<<1, 1024, 0, s>>>(a.p, a.q, I, J, a.warm_start ? a.out->g : nullptr, k, nullptr, sc, G);
    {
        double* F1 = F + I;
        void* args[] = {(void*)&a.C, (void*)&a.ld, (void*)&I,    (void*)&J,  (void*)&Jp,   (void*)&a.p,
                        (void*)&sc,  (void*)&G,    (void*)&F1,   &colpart,   (void*)&k_hi, (void*)&k_lo};
        e = cudaLaunchKernel(kk.init_rows, dim3(nb_init), dim3(NT), args, smem_init, s);
    }
    if (e == cudaSuccess) {
        sk_init_cols<<<(J + 7) / 8, 256, 0, s>>>((const float2*)colpart, nb_init, Jp, J, a.q, sc, G);
        LoopParams P;
        P.C = a.C;
        P.ld = a.ld;
        P.I = I;
        P.J = J;
        P.Jp = Jp;
        P.p = a.p;
        P.q = a.q;
        P.sc = sc;
        P.F0 = F;
        P.F1 = F + I;
        P.G = G;
        P.colpart = (float*)colpart;
        P.errpart = errpart;
        P.st = ls;
        P.k_hi = k_hi;
        P.k_lo = k_lo;
        P.tol = a.tol;
        P.max_iter = a.max_iter;
        P.spin = 1LL << 24;
        void* args[] = {&P};
        e = cudaLaunchCooperativeKernel(kk.loop, dim3(nb_loop), dim3(NT), args, smem_loop, s);
    }
    if (e == cudaSuccess) {
        FinParams Q;
        Q.C = a.C;
        Q.ld = a.ld;
        Q.I = I;
        Q.J = J;
        Q.Jp = Jp;
        Q.p = a.p;
        Q.sc = sc;
        Q.F0 = F;
        Q.F1 = F + I;
        Q.st = ls;
        Q.G = G;
        Q.k_hi = k_hi;
        Q.k_lo = k_lo;
        Q.eps_ln2 = a.eps * LN2;
        Q.pi = a.out->pi;
        Q.pi_ld = a.out->pi_ld > 0 ? a.out->pi_ld : J;
        Q.f_out = a.out->f;
        Q.fpart = (double2*)colpart;
        Q.epart = errpart;
        void* args[] = {&Q};
        e = cudaLaunchKernel(kfin, dim3(nb_fin), dim3(NT_F), args, 0, s);
    }
    if (e == cudaSuccess) {
        sk_finalize_cols<<<(J + 15) / 16, 512, 0, s>>>((const double2*)colpart, nb_fin, Jp, J, a.q, sc, ls, G,
                                                       a.eps * LN2, a.out->g, a.out->rrh_load, colerr);
        sk_summary<<<1, 256, 0, s>>>(errpart, nb_fin, colerr, J, sc, ls, summ);
        e = cudaMemcpyAsync(sum_host, summ, sizeof(SolveSummary), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return OT_ECUDA;
    }
    return OT_OK;
}

}  // namespace ota

extern "C" ot_status ot_assoc_solve_cost_noalloc(const float* C, int64_t ld_c, const float* p, const float* q,
                                                 int64_t I, int64_t J, double eps, double tol, int32_t max_iter,
                                                 int32_t warm_start, ot_assoc_result* out, void* stream) {
    using namespace ota;
    if (!C || !p || !q || !out || !out->f || !out->g) return OT_EINVAL;
    if (I <= 0 || J <= 0) return OT_EINVAL;
    if (I > NOALLOC_MAX_I || J > NOALLOC_MAX_J) return OT_EUNSUPPORTED;
    if (ld_c == 0) ld_c = J;
    if (ld_c < J || ld_c % 4 != 0 || ((uintptr_t)C & 15u)) return OT_EINVAL;
    if (!(eps > 0.0) || !std::isfinite(eps) || !(tol >= 0.0) || max_iter < 1) return OT_EINVAL;
    if (out->pi && out->pi_ld != 0 && out->pi_ld < J) return OT_EINVAL;
    SolveArgs a;
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
    ot_status st = noalloc_solve(a, &sum);
    if (st) return st;
    out->transport_cost = sum.cost;
    out->marg_err_row = sum.err_row;
    out->marg_err_col = sum.err_col;
    out->iters = sum.iters;
    out->absorptions = 0;
    if (sum.status == DEV_EINVAL || sum.status == DEV_ENUMERIC) st = OT_EINVAL;
    else if (sum.status == DEV_ETIMEOUT) st = OT_ETIMEOUT;
    else if (sum.status != DEV_OK) st = OT_ECUDA;
    else st = sum.converged ? OT_OK : OT_NOT_CONVERGED;
    out->status = st;
    return st;
}
