// Several solves of Algorithm 1 on ONE cost matrix in one persistent launch (an eps sweep:
// the same C, p and q at up to MS_MAX regularisations).
//
// A sweep is bound by reading C from HBM; solves that share C can share the read.  Each
// solve keeps its own potentials (row potentials in shared memory, column potentials,
// partials and loop state in its own scratch) and follows exactly the single-solve
// algorithm (sk_core.cuh): setup, the exact log-domain first iteration, plan-scale sweeps
// with the one-sweep-late loop test, the finalize sweep.  The first iterations and the
// finalize sweeps run one solve after the other (their per-column state does not fit the
// registers of several solves); the plan-scale sweeps run fused: every staged row of C is
// used by every solve that is still iterating, and the grid barriers of an iteration serve
// all of them.  A solve whose loop test stops it keeps its potentials and leaves the fused
// sweeps; the launch ends when the last one stops.  Partitions, team order and every
// reduction order are those of a single solve with the same team width, so each solve's
// result does not depend on which other solves share the launch.
#pragma once

#include "sk_core.cuh"

namespace ota {

static constexpr int MS_MAX = 3;

struct MultiParams {
    SolveParams P[MS_MAX];  // C, ld, I, J, Jp, V, p, q, g_warm, input_bad equal in all; the
                            // rest (k, tol, scratch, outputs, loop state) per solve
    int n;
    LoopState* grp;         // barrier counter and status word of the launch
};

// Shared-memory layout: StreamCfg offsets with the column potentials of solve s at
// off_G + 8 Jp s (FP32 pairs: Jp high parts, then Jp low parts) and its row potential
// buffers at off_F + 16 rmax s.
inline bool plan_multi(int nteams, int n, int64_t I, int Jp, int64_t ld, int nb, int stage_target, size_t budget,
                       StreamCfg* S, size_t* smem, int* Vout) {
    const size_t comb = (size_t)((nteams + 1) / 2) * Jp * sizeof(float);
    const size_t row_bytes = (size_t)ld * sizeof(float);
    const size_t per = (size_t)nteams * row_bytes;
    const int rpt = (int)(stage_target / per > 1 ? stage_target / per : 1);
    const int rs = nteams * rpt;
    const int V = parts_for(I, rs);
    int64_t rmax = 0;
    for (int b = 0; b < nb; ++b) {
        int64_t r0, r1;
        cta_rows(I, rs, V, b, nb, &r0, &r1);
        rmax = r1 - r0 > rmax ? r1 - r0 : rmax;
    }
    if (rmax < 1) rmax = 1;
    auto up = [](size_t x, size_t m) { return (x + m - 1) / m * m; };
    const size_t off_G = up(SMEM_HDR + comb, 16);
    const size_t off_F = up(off_G + (size_t)2 * n * Jp * sizeof(float), 16);
    const size_t off_P = off_F + (size_t)n * 2 * rmax * sizeof(float2);
    const size_t off_ring = up(off_P + (size_t)rmax * sizeof(float), 128);
    const size_t stage = (size_t)rs * row_bytes;
    const size_t room = off_ring < budget ? (budget - off_ring) / stage : 0;
    const int stages = (int)(room < (size_t)MAX_STAGES ? room : (size_t)MAX_STAGES);
    if (stages < 2) return false;
    S->rpt = rpt;
    S->rows_per_stage = rs;
    S->stages = stages;
    S->stage_floats = (int)(stage / sizeof(float));
    S->rmax = (int)rmax;
    S->off_G = (int)off_G;
    S->off_F = (int)off_F;
    S->off_P = (int)off_P;
    S->off_ring = (int)off_ring;
    *smem = off_ring + (size_t)stages * stage;
    *Vout = V;
    return true;
}

// The exact first iteration of one solve (sweep 1 of sk_consumers): row log-sum-exp, then a
// column (max, sum) pair per lane merged per partition, the G^1 update after a grid barrier.
// F'^1 goes to F1, G^1 to P.G + Jp and Gs.  Returns false when a wait gave up or the solve
// broke down (status set).
template <int TW, int VPT>
__device__ __forceinline__ bool ms_first_sweep(const SolveParams& P, const StreamCfg& S, GroupCtx& g, SkShared* sh,
                                               unsigned char* dyn, float* Gs, float2* F1, const float* Ps,
                                               int nrow, int v0, int v1, uint32_t& cseq, int& par) {
    constexpr int NCW = Cons<TW>::NCW;
    constexpr int TT = 32 * TW, NTEAMS = NCW / TW, NC = NCW * 32;
    constexpr int HALF = (NTEAMS + 1) / 2;
    uint64_t* full = reinterpret_cast<uint64_t*>(dyn);
    uint64_t* empty = full + MAX_STAGES;
    float* comb = reinterpret_cast<float*>(dyn + SMEM_HDR);
    const float* ring = reinterpret_cast<const float*>(dyn + S.off_ring);
    float* red = sh->red;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int J = P.J, Jp = P.Jp, rs_ = S.rows_per_stage, V = P.V, nb = g.nb, b = g.b;
    const int* pend = sh->pend - v0;
    const double* LQ = P.G + 2 * Jp;
    const Team<TW> tm;
    float4 M[VPT], Sm[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        M[v] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
        Sm[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float2* part2 = reinterpret_cast<float2*>(P.colpart);
    int kb = 0;
    for (int vp = v0; vp < v1; ++vp) {
        const int vend = pend[vp];
        for (; kb < vend; ++kb) {
            const int st = (int)(cseq % (uint32_t)S.stages);
            const uint32_t ph = (cseq / (uint32_t)S.stages) & 1u;
            const bool ok = mbar_try_wait(&full[st], ph) || mbar_wait_bounded(&full[st], ph, P.spin, g.abort);
            const int lr0 = kb * rs_;
            const int rows = min(rs_, nrow - lr0);
            const float* stage = ring + (size_t)st * S.stage_floats;
            for (int j = 0; ok && j < S.rpt; ++j) {
                const int rr = tm.team + NTEAMS * j;
                if (rr >= rows) break;
                float4 x[VPT];
                load_row_smem<TW, VPT>(stage + (size_t)rr * P.ld, J, tm.tl, x);
                float m = -INFINITY;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const int col = 4 * (tm.tl + TT * v);
                    float4 gv = col < Jp ? *reinterpret_cast<const float4*>(Gs + col) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < 4; ++c) m = fmaxf(m, fmaf(-comp(x[v], c), P.k_hi, comp(gv, c)));
                }
                m = team_reduce<TW, float, true>(m, red, NTEAMS, tm, par);
                float s = 0.f;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const int col = 4 * (tm.tl + TT * v);
                    float4 gv = col < Jp ? *reinterpret_cast<const float4*>(Gs + col) : make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 gl = col < Jp ? *reinterpret_cast<const float4*>(Gs + Jp + col) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float z = expo2(-m, comp(gl, c), comp(gv, c), comp(x[v], c), P.k_hi, P.k_lo);
                        comp(x[v], c) = z;
                        s += ex2(z);
                    }
                }
                s = team_reduce<TW, float, false>(s, red, NTEAMS, tm, par);
                const float ls = log2f(s);
                if (tm.tl == 0) {
                    float hi, lo;
                    two_sum(m, ls, hi, lo);
                    F1[lr0 + rr] = make_float2(-hi, -lo);
                }
                const float cst = log2f(Ps[lr0 + rr]) - ls;
#pragma unroll
                for (int v = 0; v < VPT; ++v)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float u = comp(x[v], c) + cst;
                        float& Mc = comp(M[v], c);
                        float& Sc = comp(Sm[v], c);
                        const float mn = fmaxf(fmaxf(Mc, u), -1e30f);
                        Sc = fmaf(Sc, ex2(Mc - mn), ex2(u - mn));
                        Mc = mn;
                    }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
            ++cseq;
        }
        // end of partition vp: teams' (max, sum) pairs merged in team order
        for (int round = 0; round < 2; ++round) {
            if ((tm.team < HALF) == (round == 0)) {
                const int slot = round == 0 ? tm.team : tm.team - HALF;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const int col = 4 * (tm.tl + TT * v);
                    if (col < Jp) {
                        float4* d = reinterpret_cast<float4*>(comb + slot * Jp + col);
                        if (round == 0) {
                            *d = M[v];
                        } else {
                            float4 o = *d;
                            o.x = fmaxf(o.x, M[v].x);
                            o.y = fmaxf(o.y, M[v].y);
                            o.z = fmaxf(o.z, M[v].z);
                            o.w = fmaxf(o.w, M[v].w);
                            *d = o;
                        }
                    }
                }
            }
            bar_named(CONS_BAR, NC);
        }
        for (int j = tid; j < Jp; j += NC) {
            float mm = comb[j];
            for (int t = 1; t < HALF; ++t) mm = fmaxf(mm, comb[t * Jp + j]);
            Gs[j] = mm;
        }
        bar_named(CONS_BAR, NC);
        for (int round = 0; round < 2; ++round) {
            if ((tm.team < HALF) == (round == 0)) {
                const int slot = round == 0 ? tm.team : tm.team - HALF;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const int col = 4 * (tm.tl + TT * v);
                    if (col < Jp) {
                        float4 sc;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float Mc = comp(M[v], c), mm = Gs[col + c];
                            comp(sc, c) = Mc > -INFINITY ? comp(Sm[v], c) * ex2(Mc - mm) : 0.f;
                        }
                        float4* d = reinterpret_cast<float4*>(comb + slot * Jp + col);
                        if (round == 0) {
                            *d = sc;
                        } else {
                            float4 o = *d;
                            o.x += sc.x;
                            o.y += sc.y;
                            o.z += sc.z;
                            o.w += sc.w;
                            *d = o;
                        }
                    }
                }
            }
            bar_named(CONS_BAR, NC);
        }
        for (int j = tid; j < J; j += NC) {
            float ss = comb[j];
            for (int t = 1; t < HALF; ++t) ss += comb[t * Jp + j];
            part2[(int64_t)vp * Jp + j] = make_float2(Gs[j], ss);
        }
        bar_named(CONS_BAR, NC);
        load_G_smem(P.G, J, Jp, Gs, tid, NC);
        bar_named(CONS_BAR, NC);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            M[v] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
            Sm[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    if (!grid_barrier_named(g.bar, (unsigned)nb * ++g.gen, g.abort, P.spin, CONS_BAR, NC, &sh->s_ok)) return false;
    {
        const int gw = b * NCW + warp, nw = nb * NCW;
        for (int j = gw; j < J; j += nw) {
            float mm = -INFINITY;
            for (int bb = lane; bb < V; bb += 32) mm = fmaxf(mm, part2[(int64_t)bb * Jp + j].x);
            mm = warp_max(mm);
            double ss = 0.0;
            if (mm > -INFINITY)
                for (int bb = lane; bb < V; bb += 32) {
                    const float2 o = part2[(int64_t)bb * Jp + j];
                    if (o.x > -INFINITY) ss += (double)o.y * (double)ex2(o.x - mm);
                }
            ss = warp_sum(ss);
            if (lane == 0) {
                if (!(ss > 0.0) || !isfinite(ss)) {
                    atomicCAS(g.status, DEV_OK, DEV_ENUMERIC);
                } else {
                    P.G[Jp + j] = P.G[j] + LQ[j] - ((double)mm + log2(ss));
                }
            }
        }
    }
    if (!grid_barrier_named(g.bar, (unsigned)nb * ++g.gen, g.abort, P.spin, CONS_BAR, NC, &sh->s_ok)) return false;
    if (ld_volatile_i32(g.status) != DEV_OK) return false;
    load_G_smem(P.G + Jp, J, Jp, Gs, tid, NC);
    bar_named(CONS_BAR, NC);
    return true;
}

// The consumer warps of a multi-solve launch.  ret_par[s] receives the row potential buffer
// of solve s's returned plan.  Returns false when the launch failed (status set).
// NS: solves the fused sweeps can hold (accumulator registers); RC: the cell values of a row
// are computed twice per solve (once for the row sum, once for the column partials) instead
// of being kept, which frees a row's worth of registers for wide rows at one more ex2 a cell.
template <int TW, int VPT, int NS, bool RC>
__device__ __forceinline__ bool ms_consumers(const MultiParams& M, const StreamCfg& S, GroupCtx& g, SkShared* sh,
                                             unsigned char* dyn, int64_t r0, int64_t r1) {
    constexpr int NCW = Cons<TW>::NCW;
    constexpr int TT = 32 * TW, NTEAMS = NCW / TW, NC = NCW * 32;
    const SolveParams& P0 = M.P[0];
    uint64_t* full = reinterpret_cast<uint64_t*>(dyn);
    uint64_t* empty = full + MAX_STAGES;
    float* comb = reinterpret_cast<float*>(dyn + SMEM_HDR);
    float* Gbase = reinterpret_cast<float*>(dyn + S.off_G);
    float2* Fbase = reinterpret_cast<float2*>(dyn + S.off_F);
    float* Ps = reinterpret_cast<float*>(dyn + S.off_P);
    const float* ring = reinterpret_cast<const float*>(dyn + S.off_ring);
    float* red = sh->red;
    float* errf = sh->errf;
    double(*sh_sum)[2] = sh->sh_sum;
    volatile int& s_stop = sh->s_stop;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int nb = g.nb, b = g.b, n = M.n;
    const int V = P0.V, rs_ = S.rows_per_stage;
    const int J = P0.J, Jp = P0.Jp;
    int v0, v1;
    cta_parts(V, b, nb, &v0, &v1);
    const int nrow = (int)max((int64_t)0, r1 - r0);
    int* status = g.status;
    for (int v = v0 + tid; v < v1; v += NC) sh->pend[v - v0] = (int)((part_row(P0.I, rs_, V, v + 1) - r0 + rs_ - 1) / rs_);
    const int* pend = sh->pend - v0;
#define OTA_MS_BARRIER()                                                                          \
    do {                                                                                          \
        if (!grid_barrier_named(g.bar, (unsigned)nb * ++g.gen, g.abort, P0.spin, CONS_BAR, NC, &sh->s_ok)) { \
            if (tid == 0) s_stop = 1;                                                             \
            return false;                                                                         \
        }                                                                                         \
    } while (0)

    // ---- setup (shared by the solves): sums of p per partition, q, checks, starting G -----
    {
        int bad = 0;
        for (int v = v0; v < v1; ++v) {
            const int a = (int)(part_row(P0.I, rs_, V, v) - r0), e = (int)(part_row(P0.I, rs_, V, v + 1) - r0);
            double sp = 0.0;
            for (int r = a + tid; r < e; r += NC) {
                const float x = __ldg(P0.p + r0 + r);
                bad |= !(x > 0.0f) || !isfinite(x);
                sp += (double)x;
                Ps[r] = x;
            }
            sp = warp_sum(sp);
            if (lane == 0) sh_sum[warp][0] = sp;
            bar_named(CONS_BAR, NC);
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < NCW; ++w) t += sh_sum[w][0];
                P0.errpart[v] = t;
            }
            bar_named(CONS_BAR, NC);
        }
        const int gw = b * NCW + warp, nw = nb * NCW;
        for (int s = 0; s < n; ++s)
            for (int j = gw * 32 + lane; j < J; j += nw * 32) {
                const double g0 = M.P[s].g_warm ? M.P[s].g_warm[j] * M.P[s].k : 0.0;
                bad |= !isfinite(g0);
                M.P[s].G[j] = g0;
            }
        if (b == 0 && tid == 0 && P0.input_bad && *P0.input_bad) bad = 1;
        if (bad) atomicOr(&sh->s_bad, 1);
        bar_named(CONS_BAR, NC);
        if (tid == 0 && sh->s_bad) atomicCAS(status, DEV_OK, DEV_EINVAL);
    }
    OTA_MS_BARRIER();
    if (ld_volatile_i32(status) != DEV_OK) {
        if (tid == 0) s_stop = 1;
        return false;
    }
    double sp = 0.0, sq = 0.0;
    {
        double a = 0.0, c = 0.0;
        int badq = 0;
        for (int bb = tid; bb < V; bb += NC) a += P0.errpart[bb];
        for (int j = tid; j < J; j += NC) {
            const float x = __ldcg(P0.q + j);
            badq |= !(x > 0.0f) || !isfinite(x);
            c += (double)x;
        }
        a = warp_sum(a);
        c = warp_sum(c);
        if (tid == 0) sh->s_bad = 0;
        bar_named(CONS_BAR, NC);
        if (lane == 0) {
            sh_sum[warp][0] = a;
            sh_sum[warp][1] = c;
        }
        if (badq) atomicOr(&sh->s_bad, 1);
        bar_named(CONS_BAR, NC);
        for (int w = 0; w < NCW; ++w) {
            sp += sh_sum[w][0];
            sq += sh_sum[w][1];
        }
        if (sh->s_bad || !(fabs(sp - sq) <= 1e-5 * sp)) {
            if (b == 0 && tid == 0) atomicCAS(status, DEV_OK, DEV_EINVAL);
            if (tid == 0) s_stop = 1;
            return false;
        }
        if (b == 0 && tid == 0)
            for (int s = 0; s < n; ++s) {
                DevScalars* d = M.P[s].sc;
                d->sp = sp;
                d->sq = sq;
                d->inv_sp = 1.0 / sp;
                d->inv_sq = 1.0 / sq;
                d->inv_sp_f = (float)(1.0 / sp);
                d->status = DEV_OK;
            }
    }
    {
        const double inv_sq = 1.0 / sq;
        const int gw = b * NCW + warp, nw = nb * NCW;
        for (int s = 0; s < n; ++s) {
            double* LQ = M.P[s].G + 2 * Jp;
            for (int j = gw * 32 + lane; j < J; j += nw * 32) LQ[j] = log2((double)__ldcg(P0.q + j) * inv_sq);
        }
        const float inv_sp_f = (float)(1.0 / sp);
        for (int r = tid; r < nrow; r += NC) Ps[r] *= inv_sp_f;
        for (int s = 0; s < n; ++s) load_G_smem(M.P[s].G, J, Jp, Gbase + (size_t)2 * s * Jp, tid, NC);
        bar_named(CONS_BAR, NC);
    }
    // LQ of solve s is read after the first grid barrier of its first iteration
    const Team<TW> tm;
    uint32_t cseq = 0;
    int par = 0;

    // ---- the exact first iteration, one solve after the other ---------------------------
    for (int s = 0; s < n; ++s) {
        if (!ms_first_sweep<TW, VPT>(M.P[s], S, g, sh, dyn, Gbase + (size_t)2 * s * Jp,
                                      Fbase + (size_t)s * 2 * S.rmax + S.rmax, Ps, nrow, v0, v1, cseq, par)) {
            if (tid == 0) s_stop = 1;
            return false;
        }
    }

    // ---- fused plan-scale sweeps -----------------------------------------------------------
    unsigned active = (1u << n) - 1u;
    int retp[MS_MAX] = {0, 0, 0};
    for (int it = 2;; ++it) {
        float4 acc[NS][VPT];
        float errt[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            errt[s] = 0.f;
#pragma unroll
            for (int v = 0; v < VPT; ++v) acc[s][v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        int kb = 0;
        for (int vp = v0; vp < v1; ++vp) {
            const int vend = pend[vp];
            for (; kb < vend; ++kb) {
                const int st = (int)(cseq % (uint32_t)S.stages);
                const uint32_t ph = (cseq / (uint32_t)S.stages) & 1u;
                const bool ok = mbar_try_wait(&full[st], ph) || mbar_wait_bounded(&full[st], ph, P0.spin, g.abort);
                const int lr0 = kb * rs_;
                const int rows = min(rs_, nrow - lr0);
                const float* stage = ring + (size_t)st * S.stage_floats;
                for (int jr = 0; ok && jr < S.rpt; ++jr) {
                    const int rr = tm.team + NTEAMS * jr;
                    if (rr >= rows) break;
                    const int lr = lr0 + rr;
                    float4 x[VPT];
                    load_row_smem<TW, VPT>(stage + (size_t)rr * P0.ld, J, tm.tl, x);
                    const float ph_ = Ps[lr];
                    if constexpr (RC) {
                        float dd[NS];
                        float2 FF[NS];
#pragma unroll
                        for (int s = 0; s < NS; ++s) {
                            dd[s] = 0.f;
                            FF[s] = make_float2(0.f, 0.f);
                            if (!((active >> s) & 1u)) continue;
                            const SolveParams& P = M.P[s];
                            const float* Gs = Gbase + (size_t)2 * s * Jp;
                            const float2* Fold = Fbase + (size_t)s * 2 * S.rmax + ((it - 1) & 1) * S.rmax;
                            float2* Fnew = Fbase + (size_t)s * 2 * S.rmax + (it & 1) * S.rmax;
                            const float2 F = Fold[lr];
                            FF[s] = F;
                            float rsum = 0.f;
#pragma unroll
                            for (int v = 0; v < VPT; ++v) {
                                const int col = 4 * (tm.tl + TT * v);
                                if (chunk_inside<TW, VPT>(v) || col < J) {
                                    float4 gv = *reinterpret_cast<const float4*>(Gs + col);
                                    float4 gl = *reinterpret_cast<const float4*>(Gs + Jp + col);
#pragma unroll
                                    for (int c = 0; c < 4; ++c)
                                        rsum += ex2(expo2(F.x, F.y + comp(gl, c), comp(gv, c), comp(x[v], c), P.k_hi,
                                                          P.k_lo));
                                }
                            }
                            rsum = team_reduce<TW, float, false>(rsum, red, NTEAMS, tm, par);
                            const float2 Fn = df_sub(F, log2_corr(rsum));
                            if (tm.tl == 0) Fnew[lr] = Fn;
                            errt[s] = fmaf(ph_, fabsf(rsum - 1.0f), errt[s]);
                            dd[s] = __fdividef(ph_, rsum);
                        }
#pragma unroll
                        for (int s = 0; s < NS; ++s) {
                            if (!((active >> s) & 1u)) continue;
                            const SolveParams& P = M.P[s];
                            const float* Gs = Gbase + (size_t)2 * s * Jp;
                            const float2 F = FF[s];
                            const float d = dd[s];
#pragma unroll
                            for (int v = 0; v < VPT; ++v) {
                                const int col = 4 * (tm.tl + TT * v);
                                if (chunk_inside<TW, VPT>(v) || col < J) {
                                    float4 gv = *reinterpret_cast<const float4*>(Gs + col);
                                    float4 gl = *reinterpret_cast<const float4*>(Gs + Jp + col);
#pragma unroll
                                    for (int c = 0; c < 4; ++c) {
                                        const float t = ex2(expo2(F.x, F.y + comp(gl, c), comp(gv, c), comp(x[v], c),
                                                                  P.k_hi, P.k_lo));
                                        comp(acc[s][v], c) = fmaf(t, d, comp(acc[s][v], c));
                                    }
                                }
                            }
                        }
                        continue;
                    }
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        if (!((active >> s) & 1u)) continue;  // uniform over the launch
                        const SolveParams& P = M.P[s];
                        const float* Gs = Gbase + (size_t)2 * s * Jp;
                        const float2* Fold = Fbase + (size_t)s * 2 * S.rmax + ((it - 1) & 1) * S.rmax;
                        float2* Fnew = Fbase + (size_t)s * 2 * S.rmax + (it & 1) * S.rmax;
                        const float2 F = Fold[lr];
                        float4 t4[VPT];
                        float rsum = 0.f;
#pragma unroll
                        for (int v = 0; v < VPT; ++v) {
                            const int col = 4 * (tm.tl + TT * v);
                            if (chunk_inside<TW, VPT>(v) || col < J) {
                                float4 gv = *reinterpret_cast<const float4*>(Gs + col);
                                float4 gl = *reinterpret_cast<const float4*>(Gs + Jp + col);
#pragma unroll
                                for (int c = 0; c < 4; ++c) {
                                    const float t = ex2(expo2(F.x, F.y + comp(gl, c), comp(gv, c), comp(x[v], c), P.k_hi,
                                                              P.k_lo));
                                    comp(t4[v], c) = t;
                                    rsum += t;
                                }
                            } else {
                                t4[v] = make_float4(0.f, 0.f, 0.f, 0.f);
                            }
                        }
                        rsum = team_reduce<TW, float, false>(rsum, red, NTEAMS, tm, par);
                        const float2 Fn = df_sub(F, log2_corr(rsum));
                        if (tm.tl == 0) Fnew[lr] = Fn;
                        errt[s] = fmaf(ph_, fabsf(rsum - 1.0f), errt[s]);
                        const float d = __fdividef(ph_, rsum);
#pragma unroll
                        for (int v = 0; v < VPT; ++v) {
                            acc[s][v].x = fmaf(t4[v].x, d, acc[s][v].x);
                            acc[s][v].y = fmaf(t4[v].y, d, acc[s][v].y);
                            acc[s][v].z = fmaf(t4[v].z, d, acc[s][v].z);
                            acc[s][v].w = fmaf(t4[v].w, d, acc[s][v].w);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[st]);
                ++cseq;
            }
            // end of partition vp: each active solve's column partials and row residual
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (!((active >> s) & 1u)) continue;
                const SolveParams& P = M.P[s];
                if (tm.tl == 0) errf[tm.team] = errt[s];
                float* cp = P.colpart + (int64_t)vp * Jp;
                cta_col_sum<TW, VPT>(comb, acc[s], J, Jp, tm, [&](int j, float sum) { cp[j] = sum; });
                if (tid == 0) {
                    float2 e = make_float2(errf[0], 0.f);
                    for (int t = 1; t < NTEAMS; ++t) e = df_add(e, errf[t]);
                    reinterpret_cast<float2*>(P.errpart)[vp] = e;
                }
                bar_named(CONS_BAR, NC);  // errf is read by thread 0 above
#pragma unroll
                for (int v = 0; v < VPT; ++v) acc[s][v] = make_float4(0.f, 0.f, 0.f, 0.f);
                errt[s] = 0.f;
            }
        }
        OTA_MS_BARRIER();
        // loop tests (warp 0) and column updates (the other warps) of every active solve
        if (warp == 0) {
            for (int s = 0; s < n; ++s) {
                if (!((active >> s) & 1u)) continue;
                const SolveParams& P = M.P[s];
                const float2* errp = reinterpret_cast<const float2*>(P.errpart);
                float2 e = make_float2(0.f, 0.f);
                for (int bb = lane; bb < V; bb += 32) e = df_add2(e, errp[bb]);
                e = warp_sum_df(e);
                if (lane == 0) {
                    const double ed = (double)e.x + (double)e.y;
                    const bool conv = ed <= stop_tol(P.tol);
                    const int stop = conv || (it - 1 >= P.max_iter);
                    if (stop) {
                        atomicOr(&sh->s_dec, 1 << s);
                        if (b == 0) {
                            P.st->iters = it - 1;
                            P.st->err = ed;
                            P.st->converged = conv;
                        }
                    }
                }
            }
        } else {
            const int gw = b * (NCW - 1) + (warp - 1), nw = nb * (NCW - 1);
            for (int s = 0; s < n; ++s) {
                if (!((active >> s) & 1u)) continue;
                const SolveParams& P = M.P[s];
                const double* Gold = P.G + ((it - 1) & 1) * Jp;
                double* Gnew = P.G + (it & 1) * Jp;
                const double* LQ = P.G + 2 * Jp;
                for (int j = gw; j < J; j += nw) {
                    float2 sum = make_float2(0.f, 0.f);
                    for (int bb = lane; bb < V; bb += 32) sum = df_add(sum, P.colpart[(int64_t)bb * Jp + j]);
                    sum = warp_sum_df(sum);
                    if (lane == 0) {
                        if (!(sum.x > 0.f) || !isfinite(sum.x)) {
                            atomicCAS(status, DEV_OK, DEV_ENUMERIC);
                        } else {
                            const float2 ls = df_log2(sum);
                            Gnew[j] = (Gold[j] - (double)ls.x) + (LQ[j] - (double)ls.y);
                        }
                    }
                }
            }
        }
        bar_named(CONS_BAR, NC);
        const unsigned stopped = (unsigned)sh->s_dec & active;
        for (int s = 0; s < n; ++s)
            if ((stopped >> s) & 1u) retp[s] = (it - 1) & 1;
        active &= ~stopped;
        bar_named(CONS_BAR, NC);  // every thread has read s_dec
        if (tid == 0) sh->s_dec = 0;
        if (!active) break;
        OTA_MS_BARRIER();
        if (ld_volatile_i32(status) != DEV_OK) {
            if (tid == 0) s_stop = 1;
            return false;
        }
        for (int s = 0; s < n; ++s)
            if ((active >> s) & 1u) load_G_smem(M.P[s].G + (it & 1) * Jp, J, Jp, Gbase + (size_t)2 * s * Jp, tid, NC);
        bar_named(CONS_BAR, NC);
    }
    if (ld_volatile_i32(status) != DEV_OK) {
        if (tid == 0) s_stop = 1;
        return false;
    }
    // ---- finalize sweeps, one solve after the other ---------------------------------------
    for (int s = 0; s < n; ++s) {
        StreamCfg Ss = S;
        Ss.off_G = S.off_G + (int)(sizeof(float) * (size_t)2 * s * Jp);
        const float2* Fold = Fbase + (size_t)s * 2 * S.rmax + retp[s] * S.rmax;
        sk_finalize_sweep<TW, VPT>(M.P[s], Ss, sh, dyn, r0, nrow, v0, v1, Fold, cseq, g.abort);
        bar_named(CONS_BAR, NC);
    }
    if (tid == 0) s_stop = 1;
    return true;
#undef OTA_MS_BARRIER
}

}  // namespace ota
