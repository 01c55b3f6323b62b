// Stored-kernel (scaling-domain) form of Algorithm 1 with absorption.
//
// The Gibbs kernel is stored relative to reference potentials (F^'_i, G^_j) taken from the
// log-domain solver:  K~_ij = 2^(F^'_i + G^_j - k C_ij)  (the plan pi_ij / p_i at those
// potentials, so every row sums to about 1), in FP32, BF16 or FP16.  The iteration is the
// a/b scaling of Algorithm 1 on K~ with row scalings alpha and column scalings beta
// (t_ij = alpha_i K~_ij beta_j = pi_ij / p_i), fused into one read of K~ per iteration:
//   s_i = sum_j K~_ij beta_j,   alpha_i <- 1 / s_i,
//   c_j = sum_i K~_ij p^_i / s_i,   beta_j <- q^_j / c_j,
// with FP32 accumulation, the row residual of the previous plan (p^_i |alpha_i s_i - 1|) as
// the loop test, and the same row partitions and fixed reduction orders as the log-domain
// solver.  Absorption: when a scaling leaves [2^-tau, 2^tau], the launch ends with the
// current potentials F' = F^' + log2 alpha, G = G^ + log2 beta, the kernel is rebuilt from C
// at those potentials (alpha = beta = 1 again) and the iteration goes on.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "ot_common.cuh"
#include "sk_core.cuh"
#include "ot_internal.h"

namespace ota {

struct LpState {
    unsigned bar;
    int status;
    int iters;        // iterations completed when the launch ended
    int converged;
    double err;
    int exit_reason;  // 0: loop test or max_iter; 1: absorption requested
    int absorb[2];    // absorption requests, by iteration parity
    int pad;
};

struct LpParams {
    const void* K;      // [I][ldk] stored kernel
    int64_t ldk;
    int64_t I;
    int J, Jp, V;
    const float* p;
    const float* q;
    const float2* Fref;  // [I] F^' (pairs)
    const double* Gref;  // [Jp] G^ (log2 units)
    float* beta;         // [2][Jp]
    float* colpart;      // [V][Jp]
    double* errpart;     // [V] (float2 pairs)
    float2* Fm;          // [I] out: F' of the plan the launch ends on
    double* Gm;          // [Jp] out: G of that plan
    LpState* st;
    double tol;
    int max_iter;
    int it0;             // iterations completed before this launch
    float tau;           // absorption threshold (log2)
    long long spin;
};

// 16-byte chunk of a stored row, widened to FP32.
template <typename T>
struct Chunk;
template <>
struct Chunk<float> {
    static constexpr int N = 4;
    __device__ __forceinline__ static void load(const float* src, float (&v)[4]) {
        const float4 x = *reinterpret_cast<const float4*>(src);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    }
    __device__ __forceinline__ static void store(float* dst, const float (&v)[4]) {
        *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Chunk<__nv_bfloat16> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16* src, float (&v)[8]) {
        const uint4 x = *reinterpret_cast<const uint4*>(src);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // a bf16 is the top half of an FP32: widening is a shift
            v[2 * k] = __uint_as_float(w[k] << 16);
            v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static void store(__nv_bfloat16* dst, const float (&v)[8]) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
            w[k] = *reinterpret_cast<const uint32_t*>(&h);
        }
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
};
template <>
struct Chunk<__half> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const __half* src, float (&v)[8]) {
        const uint4 x = *reinterpret_cast<const uint4*>(src);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        }
    }
    __device__ __forceinline__ static void store(__half* dst, const float (&v)[8]) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __half2 h = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
            w[k] = *reinterpret_cast<const uint32_t*>(&h);
        }
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
};

// Four stored values (columns 4q .. 4q+3): 16 bytes for FP32, 8 for the 16-bit formats,
// rounded pair by pair as the 16-byte chunk stores round them.
template <typename T>
__device__ __forceinline__ void store_quad(T* dst, const float (&v)[4]);
template <>
__device__ __forceinline__ void store_quad<float>(float* dst, const float (&v)[4]) {
    *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store_quad<__nv_bfloat16>(__nv_bfloat16* dst, const float (&v)[4]) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
    *reinterpret_cast<uint2*>(dst) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}
template <>
__device__ __forceinline__ void store_quad<__half>(__half* dst, const float (&v)[4]) {
    const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
    *reinterpret_cast<uint2*>(dst) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}

// Build K~ from C at potentials (F', G): one warp per row; lane l takes the column quads
// l, l + 32, ... (consecutive lanes on consecutive 16-byte pieces of the row, BUILD_U quads a
// lane in flight); columns J..ldk-1 are written as 0.  C is read in float4 pieces when its
// rows are 16-byte aligned, else element by element.  Also records the references
// F^' = F', G^ = G.  Dynamic shared memory: G as FP32 pairs (2 Jp floats).
constexpr int BUILD_U = 4;
template <typename T>
__global__ void __launch_bounds__(256) lp_build(const float* __restrict__ C, int64_t ldc, T* __restrict__ K,
                                                int64_t ldk, int64_t I, int J, int Jp, const float2* __restrict__ F,
                                                const double* __restrict__ G, float2* Fref, double* Gref,
                                                float k_hi, float k_lo) {
    extern __shared__ float Gs_build[];  // G as FP32 pairs: high parts, then low parts
    for (int j = threadIdx.x; j < Jp; j += blockDim.x) {
        const double x = j < J ? G[j] : 0.0;
        const float hi = (float)x;
        Gs_build[j] = hi;
        Gs_build[Jp + j] = (float)(x - (double)hi);
    }
    if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < Jp; j += blockDim.x) Gref[j] = G[j];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nq = (int)(ldk >> 2);  // ldk is a multiple of 4 (of 8 for the 16-bit formats)
    const bool vec = ((reinterpret_cast<uintptr_t>(C) | (uintptr_t)(ldc * (int64_t)sizeof(float))) & 15) == 0;
    for (int64_t i = w0; i < I; i += nw) {
        const float2 Fi = F[i];
        if (lane == 0) Fref[i] = Fi;
        const float* row = C + i * ldc;
        T* out = K + i * ldk;
        for (int q0 = lane; q0 < nq; q0 += 32 * BUILD_U) {
            float4 c[BUILD_U];
#pragma unroll
            for (int u = 0; u < BUILD_U; ++u) {  // every load of the round first
                const int col = 4 * (q0 + 32 * u);
                if (vec && col + 3 < J) {
                    c[u] = __ldg(reinterpret_cast<const float4*>(row + col));
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) comp(c[u], e) = col + e < J ? __ldg(row + col + e) : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < BUILD_U; ++u) {
                const int q = q0 + 32 * u;
                if (q >= nq) break;
                const int col = 4 * q;
                float v[4] = {0.f, 0.f, 0.f, 0.f};
                if (col < J) {  // col + 3 < Jp
                    const float4 gh = *reinterpret_cast<const float4*>(Gs_build + col);
                    const float4 gl = *reinterpret_cast<const float4*>(Gs_build + Jp + col);
                    const float ghv[4] = {gh.x, gh.y, gh.z, gh.w}, glv[4] = {gl.x, gl.y, gl.z, gl.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (col + e < J) v[e] = ex2(expo2(Fi.x, Fi.y + glv[e], ghv[e], comp(c[u], e), k_hi, k_lo));
                }
                store_quad<T>(out + col, v);
            }
        }
    }
}

// Consumer warps of the stored-kernel loop.  Returns false when the launch must end early
// (failed instance or a wait that gave up).
// RR: a row's values are read twice from the staged stage (once for the row sum, once for the
// column partials) instead of being kept in registers, so a lane can hold twice the columns'
// accumulators and rows of 4096 columns keep narrow teams (more rows in flight per CTA).
// NCW: consumer warps of the block (teams of TW warps).
template <typename T, int TW, int VPT, bool RR, int NCW>
__device__ __forceinline__ bool lp_consumers(const LpParams& P, const StreamCfg& S, GroupCtx& g, SkShared* sh,
                                             unsigned char* dyn, int64_t r0, int64_t r1) {
    constexpr int N = Chunk<T>::N;
    static_assert(NCW <= 24 && NCW / TW <= 16 && 2 * (NCW / TW) * TW <= 64, "SkShared sizes");
    constexpr int TT = 32 * TW, NTEAMS = NCW / TW, NC = NCW * 32;
    uint64_t* full = reinterpret_cast<uint64_t*>(dyn);
    uint64_t* empty = full + MAX_STAGES;
    float* comb = reinterpret_cast<float*>(dyn + SMEM_HDR);   // [Jp] merge row
    float* Bs = reinterpret_cast<float*>(dyn + S.off_G);      // [Jp] beta
    float* As = reinterpret_cast<float*>(dyn + S.off_F);      // [2][rmax] alpha
    float* Ps = reinterpret_cast<float*>(dyn + S.off_P);      // [rmax] p^
    const T* ring = reinterpret_cast<const T*>(dyn + S.off_ring);
    volatile int& s_stop = sh->s_stop;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int nb = g.nb, b = g.b;
    const int V = P.V, rs_ = S.rows_per_stage, J = P.J, Jp = P.Jp;
    int v0, v1;
    cta_parts(V, b, nb, &v0, &v1);
    const int nrow = (int)max((int64_t)0, r1 - r0);
    int* status = g.status;
    for (int v = v0 + tid; v < v1; v += NC) sh->pend[v - v0] = (int)((part_row(P.I, rs_, V, v + 1) - r0 + rs_ - 1) / rs_);
    const int* pend = sh->pend - v0;
#define LP_BARRIER()                                                                                     \
    do {                                                                                                 \
        if (!grid_barrier_named(g.bar, (unsigned)nb * ++g.gen, g.abort, P.spin, CONS_BAR, NC, &sh->s_ok)) { \
            if (tid == 0) s_stop = 1;                                                                    \
            return false;                                                                                \
        }                                                                                                \
    } while (0)

    // ---- setup: sums of p per partition, of q in every CTA, checks; alpha = beta = 1 --------
    {
        int bad = 0;
        for (int v = v0; v < v1; ++v) {
            const int a = (int)(part_row(P.I, rs_, V, v) - r0), e = (int)(part_row(P.I, rs_, V, v + 1) - r0);
            double sp = 0.0;
            for (int r = a + tid; r < e; r += NC) {
                const float x = __ldg(P.p + r0 + r);
                bad |= !(x > 0.0f) || !isfinite(x);
                sp += (double)x;
                Ps[r] = x;
            }
            sp = warp_sum(sp);
            if (lane == 0) sh->sh_sum[warp][0] = sp;
            bar_named(CONS_BAR, NC);
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < NCW; ++w) t += sh->sh_sum[w][0];
                P.errpart[v] = t;
            }
            bar_named(CONS_BAR, NC);
        }
        if (bad) atomicOr(&sh->s_bad, 1);
        bar_named(CONS_BAR, NC);
        if (tid == 0 && sh->s_bad) atomicCAS(status, DEV_OK, DEV_EINVAL);
    }
    LP_BARRIER();
    if (ld_volatile_i32(status) != DEV_OK) {
        if (tid == 0) s_stop = 1;
        return false;
    }
    double sp = 0.0, sq = 0.0;
    {
        double a = 0.0, c = 0.0;
        for (int bb = tid; bb < V; bb += NC) a += P.errpart[bb];
        for (int j = tid; j < J; j += NC) c += (double)__ldg(P.q + j);
        a = warp_sum(a);
        c = warp_sum(c);
        bar_named(CONS_BAR, NC);
        if (lane == 0) {
            sh->sh_sum[warp][0] = a;
            sh->sh_sum[warp][1] = c;
        }
        bar_named(CONS_BAR, NC);
        for (int w = 0; w < NCW; ++w) {
            sp += sh->sh_sum[w][0];
            sq += sh->sh_sum[w][1];
        }
    }
    const float inv_sp_f = (float)(1.0 / sp);
    const double inv_sq = 1.0 / sq;
    for (int r = tid; r < nrow; r += NC) {
        Ps[r] *= inv_sp_f;
        As[((P.it0) & 1) * S.rmax + r] = 1.0f;  // alpha of the plan the launch starts from
    }
    for (int j = tid; j < Jp; j += NC) Bs[j] = j < J ? 1.0f : 0.0f;
    bar_named(CONS_BAR, NC);
    LP_BARRIER();  // the sums in errpart are read everywhere before the loop reuses errpart

    const Team<TW> tm;
    uint32_t cseq = 0;
    int par = 0;
    float2* errp = reinterpret_cast<float2*>(P.errpart);
    const float tau = P.tau;
    for (int s = P.it0 + 1;; ++s) {
        const float* Aold = As + ((s - 1) & 1) * S.rmax;
        float* Anew = As + (s & 1) * S.rmax;
        float acc[VPT][N];
#pragma unroll
        for (int v = 0; v < VPT; ++v)
#pragma unroll
            for (int e = 0; e < N; ++e) acc[v][e] = 0.f;
        float errt = 0.f;
        int absorb = 0, numeric = 0;
        int kb = 0;
        for (int vp = v0; vp < v1; ++vp) {
            const int vend = pend[vp];
            for (; kb < vend; ++kb) {
                const int st = (int)(cseq % (uint32_t)S.stages);
                const uint32_t ph = (cseq / (uint32_t)S.stages) & 1u;
                const bool ok = mbar_try_wait(&full[st], ph) || mbar_wait_bounded(&full[st], ph, P.spin, g.abort);
                const int lr0 = kb * rs_;
                const int rows = min(rs_, nrow - lr0);
                const T* stage = ring + (size_t)st * S.stage_floats;
                for (int jr = 0; ok && jr < S.rpt; ++jr) {
                    const int rr = tm.team + NTEAMS * jr;
                    if (rr >= rows) break;
                    const int lr = lr0 + rr;
                    const T* row = stage + (size_t)rr * P.ldk;
                    float x[RR ? 1 : VPT][N];
                    float ssum = 0.f;
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        const int col = N * (tm.tl + TT * v);
                        float xv[N];
                        if (col < J) {
                            Chunk<T>::load(row + col, xv);
#pragma unroll
                            for (int e = 0; e < N; e += 4) {  // beta four at a time (16-byte loads)
                                const float4 bq = *reinterpret_cast<const float4*>(Bs + col + e);
                                ssum = fmaf(xv[e], bq.x, ssum);
                                ssum = fmaf(xv[e + 1], bq.y, ssum);
                                ssum = fmaf(xv[e + 2], bq.z, ssum);
                                ssum = fmaf(xv[e + 3], bq.w, ssum);
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < N; ++e) xv[e] = 0.f;
                        }
                        if constexpr (!RR)
#pragma unroll
                            for (int e = 0; e < N; ++e) x[v][e] = xv[e];
                    }
                    ssum = team_reduce<TW, float, false>(ssum, sh->red, NTEAMS, tm, par);
                    const float ph = Ps[lr];
                    errt = fmaf(ph, fabsf(fmaf(Aold[lr], ssum, -1.0f)), errt);
                    const float an = 1.0f / ssum;
                    numeric |= !(ssum > 0.f) || !isfinite(an);
                    absorb |= fabsf(__log2f(an)) > tau;
                    if (tm.tl == 0) Anew[lr] = an;
                    const float w = ph * an;
                    if constexpr (RR) {
#pragma unroll
                        for (int v = 0; v < VPT; ++v) {
                            const int col = N * (tm.tl + TT * v);
                            if (col < J) {
                                float xv[N];
                                Chunk<T>::load(row + col, xv);
#pragma unroll
                                for (int e = 0; e < N; ++e) acc[v][e] = fmaf(xv[e], w, acc[v][e]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < VPT; ++v)
#pragma unroll
                            for (int e = 0; e < N; ++e) acc[v][e] = fmaf(x[v][e], w, acc[v][e]);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[st]);
                ++cseq;
            }
            // end of partition vp: column partials and row residual.  The teams add their
            // partials into one merge row one team after the other (team order), so the
            // shared memory of a second row goes to the ring instead.
            if (tm.tl == 0) sh->errf[tm.team] = errt;
            for (int t = 0; t < NTEAMS; ++t) {
                if (tm.team == t) {
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        const int col = N * (tm.tl + TT * v);
                        if (col < Jp)
#pragma unroll
                            for (int e = 0; e < N; e += 4) {
                                float4* d = reinterpret_cast<float4*>(comb + col + e);
                                float4 o = t == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : *d;
                                o.x += acc[v][e];
                                o.y += acc[v][e + 1];
                                o.z += acc[v][e + 2];
                                o.w += acc[v][e + 3];
                                *d = o;
                            }
                    }
                }
                bar_named(CONS_BAR, NC);
            }
            float* cp = P.colpart + (int64_t)vp * Jp;
            for (int j = tid; j < J; j += NC) cp[j] = comb[j];
            if (tid == 0) {
                float2 e = make_float2(sh->errf[0], 0.f);
                for (int t = 1; t < NTEAMS; ++t) e = df_add(e, sh->errf[t]);
                errp[vp] = e;
            }
#pragma unroll
            for (int v = 0; v < VPT; ++v)
#pragma unroll
                for (int e = 0; e < N; ++e) acc[v][e] = 0.f;
            errt = 0.f;
            bar_named(CONS_BAR, NC);  // comb and errf are free again
        }
        if (__any_sync(0xffffffffu, numeric) && lane == 0) atomicCAS(status, DEV_OK, DEV_ENUMERIC);
        if (__any_sync(0xffffffffu, absorb) && lane == 0) atomicOr(&P.st->absorb[s & 1], 1);
        LP_BARRIER();
        if (b == 0 && tid == 0) P.st->absorb[(s + 1) & 1] = 0;  // every CTA has read it (iteration s - 1)
        // loop test on the plan of iteration s - 1 (warp 0) while the other warps form beta^s
        if (warp == 0) {
            float2 e = make_float2(0.f, 0.f);
            for (int bb = lane; bb < V; bb += 32) e = df_add2(e, errp[bb]);
            e = warp_sum_df(e);
            if (lane == 0) {
                const double ed = (double)e.x + (double)e.y;
                const int stop = (ed <= stop_tol(P.tol)) || (s - 1 >= P.max_iter) || ld_volatile_i32(status) != DEV_OK;
                sh->s_dec = stop;
                if (stop && b == 0) {
                    P.st->iters = s - 1;
                    P.st->err = ed;
                    P.st->converged = (ed <= stop_tol(P.tol));
                    P.st->exit_reason = 0;
                }
            }
        }
        const float* Bold = P.beta + ((s - 1) & 1) * Jp;
        float* Bnew = P.beta + (s & 1) * Jp;
        {
            const int gw = b * (NCW - 1) + (warp - 1), nw = nb * (NCW - 1);
            int ab = 0;
            for (int j = gw; warp > 0 && j < J; j += nw) {
                float2 sum = make_float2(0.f, 0.f);
                for (int bb = lane; bb < V; bb += 32) sum = df_add(sum, P.colpart[(int64_t)bb * Jp + j]);
                sum = warp_sum_df(sum);
                if (lane == 0) {
                    const float c = sum.x + sum.y;
                    if (!(c > 0.f) || !isfinite(c)) {
                        atomicCAS(status, DEV_OK, DEV_ENUMERIC);
                    } else {
                        const float bn = (float)((double)__ldg(P.q + j) * inv_sq) / c;
                        Bnew[j] = bn;
                        ab |= fabsf(__log2f(bn)) > tau;
                    }
                }
            }
            if (ab) atomicOr(&P.st->absorb[s & 1], 1);
        }
        bar_named(CONS_BAR, NC);
        if (sh->s_dec) {  // return the plan of iteration s - 1
            for (int r = tid; r < nrow; r += NC)
                P.Fm[r0 + r] = df_sub(P.Fref[r0 + r], -__log2f(Aold[r]));
            const int gw = b * NC + tid, nw = nb * NC;
            const bool first = (s - 1 == P.it0);  // beta of the start plan is 1
            for (int j = gw; j < J; j += nw) P.Gm[j] = P.Gref[j] + (first ? 0.0 : (double)__log2f(Bold[j]));
            if (tid == 0) s_stop = 1;
            return true;
        }
        LP_BARRIER();
        if (ld_volatile_i32(status) != DEV_OK) {
            if (tid == 0) s_stop = 1;
            return false;
        }
        if (ld_volatile_i32(&P.st->absorb[s & 1])) {  // end the launch on the plan of iteration s
            for (int r = tid; r < nrow; r += NC) P.Fm[r0 + r] = df_sub(P.Fref[r0 + r], -__log2f(Anew[r]));
            const int gw = b * NC + tid, nw = nb * NC;
            for (int j = gw; j < J; j += nw) P.Gm[j] = P.Gref[j] + (double)__log2f(Bnew[j]);
            if (b == 0 && tid == 0) {
                P.st->iters = s;
                P.st->exit_reason = 1;
                P.st->converged = 0;
            }
            if (tid == 0) s_stop = 1;
            return true;
        }
        for (int j = tid; j < Jp; j += NC) Bs[j] = j < J ? Bnew[j] : 0.f;
        bar_named(CONS_BAR, NC);
    }
#undef LP_BARRIER
}

template <typename T, int TW, int VPT, bool RR, int NCW>
__global__ void __launch_bounds__(32 * (NCW + 1), 1) lp_loop(LpParams P, StreamCfg S) {
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ SkShared sh;
    uint64_t* full = reinterpret_cast<uint64_t*>(dyn);
    uint64_t* empty = full + MAX_STAGES;
    T* ring = reinterpret_cast<T*>(dyn + S.off_ring);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t r0, r1;
    cta_rows(P.I, S.rows_per_stage, P.V, blockIdx.x, gridDim.x, &r0, &r1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        sh.s_stop = 0;
        sh.s_bad = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == NCW) {
        if (lane == 0)
            stream_rows_producer<T>(reinterpret_cast<const T*>(P.K), P.ldk, r0, r1, S, ring, full, empty, &sh.s_stop,
                                    &P.st->status, P.spin);
        return;
    }
    GroupCtx g{(int)gridDim.x, (int)blockIdx.x, &P.st->bar, 0u, &P.st->status, &P.st->status};
    lp_consumers<T, TW, VPT, RR, NCW>(P, S, g, &sh, dyn, r0, r1);
}

// ------------------------------------------------------------------------------------------
// Host side.
// ------------------------------------------------------------------------------------------
struct LpKernel {
    const void* fn;
    int tw, ncw;
};

template <typename T, int TW, int VPT, bool RR = false, int NCW = Cons<TW>::NCW>
LpKernel lp_kernel() {
    return LpKernel{(const void*)lp_loop<T, TW, VPT, RR, NCW>, TW, NCW};
}

// One-warp teams while a lane holds at most 32 values (8 chunks of 4 or 4 of 8); 16-bit
// kernels then read each row twice from shared memory to hold 64 accumulators a lane (8
// chunks of 8); wider teams beyond.  Two-warp teams run 14 consumer warps (15 with the
// producer: still at most 4 warps, 128 registers, a sub-partition): the loop is bound by its
// consumers' latency, and 14 warps instead of 12 took 25 iterations at 400,000 x 4,096
// (BF16) from 20.2 to 17.8 ms.
template <typename T>
bool lp_pick(int J, LpKernel* k) {
    constexpr int N = Chunk<T>::N;
    const int Jc = (J + N - 1) / N;
    if constexpr (N == 4) {
        if (Jc <= 32) *k = lp_kernel<T, 1, 1>();
        else if (Jc <= 64) *k = lp_kernel<T, 1, 2>();
        else if (Jc <= 128) *k = lp_kernel<T, 1, 4>();
        else if (Jc <= 256) *k = lp_kernel<T, 1, 8>();
        else if (Jc <= 512) *k = lp_kernel<T, 2, 8, false, 14>();
        else if (Jc <= 1024) *k = lp_kernel<T, 4, 8>();
        else if (Jc <= 2048) *k = lp_kernel<T, 8, 8>();
        else return false;
    } else {
        if (Jc <= 32) *k = lp_kernel<T, 1, 1>();
        else if (Jc <= 64) *k = lp_kernel<T, 1, 2>();
        else if (Jc <= 128) *k = lp_kernel<T, 1, 4>();
        else if (Jc <= 256) *k = lp_kernel<T, 1, 8, true>();
        else if (Jc <= 512) *k = lp_kernel<T, 2, 8, true, 14>();
        else if (Jc <= 1024) *k = lp_kernel<T, 4, 8, true>();
        else return false;
    }
    return true;
}

template <typename T>
ot_status lowp_solve_t(ot_assoc_ctx* ctx, const SolveArgs& a, double absorb_log2, SolveSummary* sum_host) {
    constexpr int N = Chunk<T>::N;
    ot_status st = OT_OK;
    const int64_t I = a.I;
    const int J = a.J, Jp = (int)round_up(J, 8);  // 8: whole 16-byte chunks of 16-bit rows
    const int64_t ldk = round_up(J, N);
    cudaStream_t s = a.stream;
    LpKernel kk;
    if (!lp_pick<T>(J, &kk)) return set_error(ctx, OT_EUNSUPPORTED, "J=%d above 8192", J);
    // launch geometry of the loop: one CTA per row partition
    const int nteams = kk.ncw / kk.tw;
    StreamCfg S;
    size_t smem = 0;
    int V = 1;
    // one float a row per scaling buffer, and one merge row for the teams' column partials
    // (merged team after team): the room goes to the ring of stages
    if (!plan_stage(nteams, I, Jp, ldk, 1, 24576, (size_t)1 << 40, &S, &smem, &V, (int)sizeof(T), 1, 4, 1))
        return set_error(ctx, OT_EUNSUPPORTED, "stored-kernel geometry");
    const int grid = std::max(1, std::min(V, ctx->num_sms));
    if (!plan_stage(nteams, I, Jp, ldk, grid, 24576, 232448 - 4096, &S, &smem, &V, (int)sizeof(T), 1, 4, 1))
        return set_error(ctx, OT_EUNSUPPORTED, "stored kernel does not fit the shared memory (I=%lld J=%d)",
                         (long long)I, J);
    if (allow_max_dynamic_smem(kk.fn, smem) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, OT_ECUDA, "stored-kernel loop: shared memory");
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kk.fn, 32 * (kk.ncw + 1), smem) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        return set_error(ctx, OT_EUNSUPPORTED, "stored-kernel loop cannot be resident");
    }
    // buffers: K~ in its own slot; potentials, scalings and partials in another
    T* K = (T*)scratch(ctx, SLOT_KT, sizeof(T) * (size_t)(I * ldk), &st);
    if (st) return st;
    const size_t o_Fm = 0, o_Fref = round_up(8 * I, 256), o_Gm = o_Fref + round_up(8 * I, 256);
    const size_t o_Gref = o_Gm + round_up(8 * (int64_t)Jp, 256), o_beta = o_Gref + round_up(8 * (int64_t)Jp, 256);
    const size_t o_cp = o_beta + round_up(8 * (int64_t)Jp, 256), o_ep = o_cp + round_up(4 * (int64_t)V * Jp, 256);
    const size_t o_st = o_ep + round_up(16 * (int64_t)V, 256), total = o_st + 256;
    char* base = (char*)scratch(ctx, SLOT_SCAL, total, &st);
    if (st) return st;
    float2* Fm = (float2*)(base + o_Fm);
    float2* Fref = (float2*)(base + o_Fref);
    double* Gm = (double*)(base + o_Gm);
    double* Gref = (double*)(base + o_Gref);
    float* beta = (float*)(base + o_beta);
    LpState* lst = (LpState*)(base + o_st);
    LpState* hls = (LpState*)host_staging(ctx, sizeof(LpState) + sizeof(SolveSummary), &st);
    if (st) return st;
    // phase events (timing mode only): [0] before iteration 1, then a pair around each loop
    // launch, and the last one after the finalize
    const bool timing = ctx->timing;
    cudaEvent_t tev[2 + 2 * 8] = {};
    int ntev = 0;
    auto mark = [&](void) {
        if (!timing || ntev >= (int)(sizeof(tev) / sizeof(tev[0]))) return;
        if (cudaEventCreate(&tev[ntev]) == cudaSuccess) cudaEventRecord(tev[ntev++], s);
        else cudaGetLastError();
    };
    struct EvGuard {
        cudaEvent_t* e;
        int* n;
        ~EvGuard() {
            for (int i = 0; i < *n; ++i) cudaEventDestroy(e[i]);
        }
    } evguard{tev, &ntev};
    int loop_reads = 0;
    mark();
    // iteration 1 in the log domain from C
    int dstat = 0;
    st = f32_first_iteration(ctx, a, Fm, Gm, &dstat);
    if (st) return st;
    if (dstat != DEV_OK) {
        std::memset(sum_host, 0, sizeof(*sum_host));
        sum_host->status = dstat == DEV_ENUMERIC ? OT_ENUMERIC_INTERNAL : dstat;
        return OT_OK;
    }
    float k_hi, k_lo;
    split_k(LOG2E / a.eps, &k_hi, &k_lo);
    // default thresholds: FP32 only guards the range; BF16 keeps FP32's exponent range; FP16
    // flushes entries below 2^-24 of a row, so its kernel is rebuilt before scalings move far
    const double tau_default = std::is_same<T, float>::value ? 30.0 : (std::is_same<T, __half>::value ? 8.0 : 20.0);
    const double tau = absorb_log2 > 0 ? absorb_log2 : tau_default;
    int iters = 1, converged = 0, absorptions = 0;
    double err = 0.0;
    const int bgrid = (int)std::max<int64_t>(1, std::min<int64_t>((I + 7) / 8, 8LL * ctx->num_sms));
    const size_t build_smem = 2 * sizeof(float) * (size_t)Jp;  // G pairs
    if (build_smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(lp_build<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)build_smem);
        if (e != cudaSuccess) return cuda_error(ctx, e, "lp_build attribute");
    }
    for (int launch = 0;; ++launch) {
        if (iters >= a.max_iter) break;  // the first iteration's plan is the answer
        lp_build<T><<<bgrid, 256, build_smem, s>>>(a.C, a.ld, K, ldk, I, J, Jp, Fm, Gm, Fref, Gref, k_hi,
                                                           k_lo);
        cudaError_t e = cudaMemsetAsync(lst, 0, sizeof(LpState), s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "memset");
        LpParams P;
        P.K = K;
        P.ldk = ldk;
        P.I = I;
        P.J = J;
        P.Jp = Jp;
        P.V = V;
        P.p = a.p;
        P.q = a.q;
        P.Fref = Fref;
        P.Gref = Gref;
        P.beta = beta;
        P.colpart = (float*)(base + o_cp);
        P.errpart = (double*)(base + o_ep);
        P.Fm = Fm;
        P.Gm = Gm;
        P.st = lst;
        P.tol = a.tol;
        P.max_iter = a.max_iter;
        P.it0 = iters;
        P.tau = (float)tau;
        P.spin = ctx->spin_limit;
        void* args[] = {&P, &S};
        mark();
        e = cudaLaunchCooperativeKernel(kk.fn, dim3(grid), dim3(32 * (kk.ncw + 1)), args, smem, s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "stored-kernel loop launch");
        mark();
        ctx->launches += 2;
        e = cudaMemcpyAsync(hls, lst, sizeof(LpState), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "stored-kernel loop");
        if (hls->status != DEV_OK) {
            std::memset(sum_host, 0, sizeof(*sum_host));
            sum_host->status = hls->status == DEV_ENUMERIC ? OT_ENUMERIC_INTERNAL : hls->status;
            sum_host->iters = hls->iters;
            return OT_OK;
        }
        loop_reads += hls->iters + 1 - iters;  // the launch read K~ once per iteration and once to test
        iters = hls->iters;
        err = hls->err;
        converged = hls->converged;
        if (hls->exit_reason != 1) break;
        ++absorptions;  // Fm, Gm hold the plan of iteration `iters`: rebuild there
    }
    st = f32_finalize_on(ctx, a, Fm, Gm, iters, err, converged, sum_host);
    if (st) return st;
    sum_host->absorptions = absorptions;
    mark();
    if (timing && ntev >= 4 && cudaEventSynchronize(tev[ntev - 1]) == cudaSuccess) {
        // init: iteration 1 and the first kernel build; loop: the persistent loop launches;
        // finalize: everything after the last loop launch (rebuilds between launches count as loop)
        float a0 = 0.f, lp = 0.f, fin = 0.f, x = 0.f;
        cudaEventElapsedTime(&a0, tev[0], tev[1]);
        for (int i = 1; i + 1 < ntev - 1; i += 2) {
            if (cudaEventElapsedTime(&x, tev[i], tev[i + 1]) == cudaSuccess) lp += x;
        }
        cudaEventElapsedTime(&fin, tev[ntev - 2], tev[ntev - 1]);
        ot_assoc_timings t = {};
        t.init_ms = a0;
        t.loop_ms = lp;
        t.finalize_ms = fin;
        t.sweeps = loop_reads;
        t.valid = 1;
        ctx->last_timings = t;
    }
    cudaGetLastError();
    return OT_OK;
}

}  // namespace ota
