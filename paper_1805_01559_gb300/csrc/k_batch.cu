// Batched ragged Sinkhorn: many independent instances of Algorithm 1 (Sec. III-B) in one
// persistent cooperative launch.
//
// The launch holds one CTA per SM.  Its work is split into phases; in phase k the CTAs form
// groups of gsize_k CTAs (gsize_k divides the grid), and every group takes instances from
// the phase's queue (an atomic counter over the phase's instances, largest first) until the
// queue is empty.  A group solves an instance exactly as the single-instance kernel does --
// the same consumer code (sk_core.cuh) with the group in place of the grid -- then, in the
// same launch, finalizes it: plan potentials in natural units, FP64 reductions of the row
// and column residuals, the per-RRH loads rho_j and the transport cost.  Phases end with a
// grid barrier.  Which group size and which stage size (rows of C per bulk copy) an
// instance gets depends on its size bucket; the autotuner below measures the candidates.
//
// A failed instance (bad marginals, numerical breakdown) only ends that instance; a wait
// that gives up raises the launch's abort word and every CTA leaves.  Every wait is bounded.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ot_common.cuh"
#include "sk_core.cuh"
#include "ot_internal.h"

namespace ota {

static constexpr int BT_NCW = Cons<1>::NCW;  // consumer warps (one-warp teams)
static constexpr int BT_NT = Cons<1>::NT;    // + the producer warp
static constexpr int BT_NW = BT_NT / 32;
static constexpr int BT_MAX_FIN_TEAMS = 8;

// One instance as the kernel sees it (host-written).
struct BInst {
    SolveParams P;  // C, ld, I, J, Jp, p, q, g_warm, k, k_hi, k_lo, tol, max_iter (scratch filled per group)
    StreamCfg S;    // stage geometry and shared-memory layout at this instance's group size
    int vpt;        // float4 chunks per lane (J4 <= 32 * vpt)
    int fin_teams;  // finalize teams that fit next to the row potentials
    double eps_ln2;
    double* f_out;
    double* g_out;
    double* rrh_load;
    float* pi;
    int64_t pi_ld;
};

// Result of one instance (device-written).
struct BRes {
    double cost, err_row, err_col, err_loop;
    int iters, converged, status, done;
};

struct BPhase {
    int gsize, ngroups, first, count;
};

// Scratch of one group (sized for the largest instance of its phase).
struct BGroup {
    DevScalars* sc;
    LoopState* ls;
    double* G;         // [3][Jp]
    float* colpart;    // [gsize][2 * Jp]
    double* errpart;   // [gsize] (x2)
    double2* fpart;    // [gsize][Jp] finalize column partials
    double* fred;      // [gsize][BT_NW][2] finalize totals per warp; then [gsize] row residuals
};

struct BCtl {
    unsigned grid_bar;
    int abort;
    unsigned next[16];
};

struct BatchParams {
    const BInst* inst;
    BRes* res;
    const int* order;  // instance indices, phase by phase (largest first within a phase)
    const BPhase* phases;
    int nphases;
    const BGroup* groups;  // phase-major
    const int* goff;       // first group of each phase
    BCtl* ctl;
    unsigned* gbar;        // per group (all phases): barrier counter
    int* gcur;             // per group: the instance index the leader fetched
    long long spin;
};

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Group barrier for all threads of the CTA; only thread 0 advances the generation.
__device__ __forceinline__ bool group_sync(unsigned* bar, unsigned nb, unsigned* s_gen, int* abort, long long spin) {
    unsigned target = 0;
    if (threadIdx.x == 0) target = nb * ++(*s_gen);
    return grid_barrier(bar, target, abort, spin);
}

// Finalize one instance on the group's rows (all threads of the CTA; the producer is idle).
// Teams of one warp walk the CTA's rows; each lane adds p^ t and p^ C t of its cells, row by
// row, into its team's FP32-pair accumulators in shared memory (the stage ring's space; each
// lane owns its columns); CTAs combine teams in order and the group combines CTAs in order,
// in FP64.
template <int VPT>
__device__ __forceinline__ bool bt_finalize(const BInst& D, const SolveParams& P, const BGroup& grp, int rank, int gsize,
                            int64_t r0, int64_t r1, int par, unsigned char* dyn, unsigned* gbar, unsigned* s_gen,
                            int* abort, long long spin, BRes* out) {
    const StreamCfg& S = D.S;
    const int J = P.J, Jp = P.Jp;
    const int NTM = D.fin_teams;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* accs = reinterpret_cast<float4*>(dyn + S.off_ring);  // [NTM][Jp]
    const float2* Fr = reinterpret_cast<const float2*>(dyn + S.off_F) + par * S.rmax;
    const double* Gk = P.G + par * Jp;
    __shared__ float s_err[BT_NW];
    for (int q = threadIdx.x; q < NTM * Jp; q += blockDim.x) accs[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const float inv_sp_f = P.sc->inv_sp_f;
    if (warp < NTM) {
        float4* myacc = accs + (size_t)warp * Jp;
        float4 g[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int col = 4 * (lane + 32 * v);
#pragma unroll
            for (int c = 0; c < 4; ++c) comp(g[v], c) = (col + c < J) ? (float)Gk[col + c] : 0.0f;
        }
        float errt = 0.f;
        // no prefetch of the next row: the registers are needed (13 warps: 128 per thread);
        // the loads of all teams in flight still cover the memory latency
        for (int64_t i = r0 + warp; i < r1; i += NTM) {
            float4 x[VPT];
            load_row<1, VPT>(P.C + i * P.ld, J, lane, x);
            const float2 F = Fr[i - r0];
            const float pf = __ldg(P.p + i);
            const float phf = pf * inv_sp_f;
            float rs = 0.f;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int col = 4 * (lane + 32 * v);
                if (col < J) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (col + c < J) {
                            const float cost = comp(x[v], c);
                            const float t = ex2(expo(F.x, F.y + comp(g[v], c), cost, P.k_hi, P.k_lo));
                            const float ct = t > 0.f ? cost * t : 0.f;
                            rs += t;
                            float4 a = myacc[col + c];
                            const float2 s2 = df_add(make_float2(a.x, a.y), phf * t);
                            const float2 r2 = df_add(make_float2(a.z, a.w), phf * ct);
                            myacc[col + c] = make_float4(s2.x, s2.y, r2.x, r2.y);
                            if (D.pi) D.pi[i * D.pi_ld + col + c] = pf * t;
                        }
                    }
                }
            }
            float se = 0.f;
            warp_sum_pair(rs, se);
            errt = fmaf(phf, fabsf((rs - 1.0f) + se), errt);
            if (lane == 0) D.f_out[i] = D.eps_ln2 * ((double)F.x + (double)F.y + log2((double)pf));
        }
        if (lane == 0) s_err[warp] = errt;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        float4 a = accs[j];
        float2 s = make_float2(a.x, a.y), r = make_float2(a.z, a.w);
        for (int t = 1; t < NTM; ++t) {
            const float4 o = accs[(size_t)t * Jp + j];
            s = df_add2(s, make_float2(o.x, o.y));
            r = df_add2(r, make_float2(o.z, o.w));
        }
        grp.fpart[(int64_t)rank * Jp + j] = make_double2((double)s.x + (double)s.y, (double)r.x + (double)r.y);
    }
    double* rowerr = grp.fred + (size_t)gsize * BT_NW * 2;
    if (threadIdx.x == 0) {
        float2 e = make_float2(s_err[0], 0.f);
        for (int t = 1; t < NTM; ++t) e = df_add(e, s_err[t]);
        rowerr[rank] = (double)e.x + (double)e.y;
    }
    // the next instance's bulk copies write where the accumulators were
    fence_proxy_async_smem();
    if (!group_sync(gbar, gsize, s_gen, abort, spin)) return false;
    // columns: one warp per column over the group's CTAs
    {
        const double inv_sq = P.sc->inv_sq, sp = P.sc->sp;
        double ec = 0.0, co = 0.0;
        const int gw = rank * BT_NW + warp, nw = gsize * BT_NW;
        for (int j = gw; j < J; j += nw) {
            double s = 0.0, r = 0.0;
            for (int bb = lane; bb < gsize; bb += 32) {
                const double2 v = grp.fpart[(int64_t)bb * Jp + j];
                s += v.x;
                r += v.y;
            }
            s = warp_sum(s);
            r = warp_sum(r);
            if (lane == 0) {
                ec += fabs(s - (double)__ldg(P.q + j) * inv_sq);
                co += r;
                if (D.rrh_load) D.rrh_load[j] = r * sp;
                D.g_out[j] = D.eps_ln2 * Gk[j];
            }
        }
        if (lane == 0) {
            grp.fred[((size_t)rank * BT_NW + warp) * 2 + 0] = ec;
            grp.fred[((size_t)rank * BT_NW + warp) * 2 + 1] = co;
        }
    }
    if (!group_sync(gbar, gsize, s_gen, abort, spin)) return false;
    if (rank == 0 && threadIdx.x == 0) {
        double ec = 0.0, co = 0.0, er = 0.0;
        for (int k = 0; k < gsize * BT_NW; ++k) {
            ec += grp.fred[2 * k];
            co += grp.fred[2 * k + 1];
        }
        for (int k = 0; k < gsize; ++k) er += rowerr[k];
        out->cost = co * P.sc->sp;
        out->err_row = er;
        out->err_col = ec;
        out->err_loop = grp.ls->err;
        out->iters = grp.ls->iters;
        out->converged = grp.ls->converged;
        out->done = 1;  // out->status holds whatever the solve reported (DEV_OK normally)
    }
    return true;
}

// One instance on this CTA's group: (re)arm the stage barriers, stream and sweep, finalize.
// Returns false when the launch must end (a wait gave up).
template <int VPT>
__device__ __forceinline__ bool bt_instance(const BatchParams& B, int ii, const BGroup& grp, int rank, int gsize, unsigned* gbar,
                            unsigned* s_gen, int* s_nbar, SkShared* sh, unsigned char* dyn) {
    const BInst& D = B.inst[ii];
    SolveParams P = D.P;
    P.sc = grp.sc;
    P.st = grp.ls;
    P.G = grp.G;
    P.colpart = grp.colpart;
    P.errpart = grp.errpart;
    P.F_out = nullptr;
    P.input_bad = nullptr;
    P.spin = B.spin;
    const StreamCfg S = D.S;
    uint64_t* full = reinterpret_cast<uint64_t*>(dyn);
    uint64_t* empty = full + MAX_STAGES;
    float* ring = reinterpret_cast<float*>(dyn + S.off_ring);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* abort = &B.ctl->abort;
    int64_t r0, r1;
    cta_rows(P.I, S.rows_per_stage, rank, gsize, &r0, &r1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < *s_nbar; ++s) {
            mbar_inval(&full[s]);
            mbar_inval(&empty[s]);
        }
        for (int s = 0; s < S.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], BT_NCW);
        }
        *s_nbar = S.stages;
        sh->s_stop = 0;
        sh->s_bad = 0;
        mbar_fence_init();
    }
    __shared__ int s_res;
    __syncthreads();
    if (warp == BT_NCW) {
        if (lane == 0) stream_rows_producer(P.C, P.ld, r0, r1, S, ring, full, empty, &sh->s_stop, abort, B.spin);
    } else {
        // the instance's status word is its result slot (zeroed = DEV_OK before the launch):
        // a group's shared words are reused by the next instance while a slow CTA may still be
        // reading this one's status after the barrier that ended it
        GroupCtx g{gsize, rank, gbar, *s_gen, abort, &B.res[ii].status};
        int par = 0;
        const bool ok = sk_consumers<1, VPT>(P, S, g, sh, dyn, r0, r1, &par);
        if (threadIdx.x == 0) {
            *s_gen = g.gen;
            s_res = ok ? 1 + par : 0;
        }
    }
    __syncthreads();  // the producer has drained its copies
    if (ld_volatile_i32(abort) != DEV_OK) return false;
    if (s_res == 0) {  // the instance failed (the same in every CTA of the group)
        if (rank == 0 && threadIdx.x == 0) {
            BRes* out = B.res + ii;
            out->iters = 0;
            out->converged = 0;
            out->done = 1;
        }
        return true;
    }
    return bt_finalize<VPT>(D, P, grp, rank, gsize, r0, r1, s_res - 1, dyn, gbar, s_gen, abort, B.spin,
                            B.res + ii);
}

__global__ void __launch_bounds__(BT_NT, 1) sk_batch(BatchParams B) {
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ SkShared sh;
    __shared__ unsigned s_gen, s_ggen;
    __shared__ int s_idx, s_nbar;
    if (threadIdx.x == 0) {
        s_ggen = 0;
        s_nbar = 0;
    }
    __syncthreads();
    for (int ph = 0; ph < B.nphases; ++ph) {
        const BPhase PH = B.phases[ph];
        const int grp_i = blockIdx.x / PH.gsize, rank = blockIdx.x % PH.gsize;
        if (grp_i < PH.ngroups) {
            const int gi = B.goff[ph] + grp_i;
            const BGroup grp = B.groups[gi];
            unsigned* gbar = B.gbar + gi;
            if (threadIdx.x == 0) s_gen = 0;
            for (;;) {
                if (rank == 0 && threadIdx.x == 0) B.gcur[gi] = (int)atomicAdd(&B.ctl->next[ph], 1u);
                if (!group_sync(gbar, PH.gsize, &s_gen, &B.ctl->abort, B.spin)) return;
                if (threadIdx.x == 0) s_idx = ld_volatile_i32(B.gcur + gi);
                __syncthreads();
                const int k = s_idx;
                if (k >= PH.count) break;
                const int ii = B.order[PH.first + k];
                bool go = true;
                switch (B.inst[ii].vpt) {
                    case 1: go = bt_instance<1>(B, ii, grp, rank, PH.gsize, gbar, &s_gen, &s_nbar, &sh, dyn); break;
                    case 2: go = bt_instance<2>(B, ii, grp, rank, PH.gsize, gbar, &s_gen, &s_nbar, &sh, dyn); break;
                    case 3: go = bt_instance<3>(B, ii, grp, rank, PH.gsize, gbar, &s_gen, &s_nbar, &sh, dyn); break;
                    case 4: go = bt_instance<4>(B, ii, grp, rank, PH.gsize, gbar, &s_gen, &s_nbar, &sh, dyn); break;
                    case 5: go = bt_instance<5>(B, ii, grp, rank, PH.gsize, gbar, &s_gen, &s_nbar, &sh, dyn); break;
                    case 6: go = bt_instance<6>(B, ii, grp, rank, PH.gsize, gbar, &s_gen, &s_nbar, &sh, dyn); break;
                    case 7: go = bt_instance<7>(B, ii, grp, rank, PH.gsize, gbar, &s_gen, &s_nbar, &sh, dyn); break;
                    default: go = bt_instance<8>(B, ii, grp, rank, PH.gsize, gbar, &s_gen, &s_nbar, &sh, dyn); break;
                }
                if (!go) return;
            }
        }
        unsigned target = 0;
        if (threadIdx.x == 0) target = gridDim.x * ++s_ggen;
        if (!grid_barrier(&B.ctl->grid_bar, target, &B.ctl->abort, B.spin)) return;
    }
}

// ------------------------------------------------------------------------------------------
// Host side: size buckets, stage planning, schedule, autotuner, captured graph.
// ------------------------------------------------------------------------------------------
namespace {

constexpr size_t SMEM_BUDGET = 232448 - 4096;  // 227 KB per block minus static shared memory
constexpr int MAX_J_BATCH = 1024;              // one-warp teams: J4 <= 32 * 8

int vpt_for(int J) { return std::max(1, (int)((round_up(J, 4) / 4 + 31) / 32)); }

// Stage geometry and shared-memory layout of one instance solved by nb CTAs.
bool plan_stream(int64_t I, int Jp, int64_t ld, int nb, int stage_target, StreamCfg* S, size_t* smem,
                 int* fin_teams) {
    constexpr int NTEAMS = BT_NCW;
    const size_t comb = (size_t)((NTEAMS + 1) / 2) * Jp * sizeof(float);
    const size_t row_bytes = (size_t)ld * sizeof(float);
    int rpt = (int)std::max<size_t>(1, (size_t)stage_target / ((size_t)NTEAMS * row_bytes));
    for (;;) {
        const int rs = NTEAMS * rpt;
        const int64_t blocks = (I + rs - 1) / rs;
        const int64_t bpc = (blocks + nb - 1) / nb;
        const int rmax = (int)std::min<int64_t>(bpc * rs, I);
        const size_t off_G = round_up(SMEM_HDR + comb, 16);
        const size_t off_F = round_up(off_G + (size_t)Jp * sizeof(float), 16);
        const size_t off_P = off_F + (size_t)2 * rmax * sizeof(float2);
        const size_t off_ring = round_up(off_P + (size_t)rmax * sizeof(float), 128);
        const size_t stage = (size_t)rs * row_bytes;
        const int stages =
            off_ring < SMEM_BUDGET ? (int)std::min<size_t>(MAX_STAGES, (SMEM_BUDGET - off_ring) / stage) : 0;
        int ft = 0;
        for (int t = BT_MAX_FIN_TEAMS; t >= 1 && !ft; t /= 2)
            if (off_ring + (size_t)t * Jp * sizeof(float4) <= SMEM_BUDGET) ft = t;
        if (ft && (stages >= 3 || (stages >= 2 && rpt == 1))) {
            S->rpt = rpt;
            S->rows_per_stage = rs;
            S->stages = stages;
            S->stage_floats = (int)(stage / sizeof(float));
            S->rmax = rmax;
            S->off_G = (int)off_G;
            S->off_F = (int)off_F;
            S->off_P = (int)off_P;
            S->off_ring = (int)off_ring;
            *smem = off_ring + std::max((size_t)stages * stage, (size_t)ft * Jp * sizeof(float4));
            *fin_teams = ft;
            return true;
        }
        if (rpt == 1) return false;
        rpt = std::max(1, rpt / 2);
    }
}

std::vector<int> divisors(int n) {
    std::vector<int> d;
    for (int k = 1; k <= n; ++k)
        if (n % k == 0) d.push_back(k);
    return d;
}

// Default schedule before tuning: about 2^18 cells per CTA, at most one row block per CTA.
int default_gsize(int64_t I, int J, int num_sms) {
    const double cells = (double)I * J;
    const int64_t blocks = (I + BT_NCW - 1) / BT_NCW;
    int best = 1;
    for (int d : divisors(num_sms))
        if (d <= cells / 262144.0 && d <= blocks) best = d;
    return best;
}

}  // namespace

int batch_bucket(int64_t I, int J) {
    const double cells = (double)I * J;
    int c = 0;
    if (cells >= 524288.0) c = 1;
    if (cells >= 2097152.0) c = 2;
    if (cells >= 8388608.0) c = 3;
    if (cells >= 33554432.0) c = 4;
    const int jc = J <= 256 ? 0 : (J <= 512 ? 1 : 2);
    return c * 3 + jc;
}

}  // namespace ota

// ------------------------------------------------------------------------------------------
// The batch object: planned schedule, device tables, captured graph.
// ------------------------------------------------------------------------------------------
struct ot_assoc_batch {
    ot_assoc_ctx* ctx = nullptr;
    int n = 0;
    std::vector<ot_assoc_instance> inst;
    // host mirrors
    ota::BInst* h_inst = nullptr;  // pinned: copied to the device by the graph on every launch
    ota::BRes* h_res = nullptr;    // pinned: copied back by the graph
    std::vector<int> h_order;
    std::vector<ota::BPhase> h_phases;
    std::vector<ota::BGroup> h_groups;
    std::vector<int> h_goff;
    // device memory (one allocation)
    void* dmem = nullptr;
    size_t dbytes = 0;
    ota::BInst* d_inst = nullptr;
    ota::BRes* d_res = nullptr;
    ota::BCtl* d_ctl = nullptr;
    unsigned* d_gbar = nullptr;
    int* d_gcur = nullptr;
    size_t zero_bytes = 0;  // control words cleared before each launch (ctl, gbar, gcur)
    ota::BatchParams params{};
    size_t smem = 0;
    int grid = 0;
    cudaStream_t stream = nullptr;  // capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int use_graph = 1;
};

namespace ota {

static ot_status batch_check(ot_assoc_ctx* ctx, const ot_assoc_instance& a, int k) {
    if (!a.C || !a.p || !a.q || !a.f || !a.g) return set_error(ctx, OT_EINVAL, "instance %d: null pointer", k);
    if (a.I <= 0 || a.J <= 0) return set_error(ctx, OT_EINVAL, "instance %d: I and J must be positive", k);
    if (a.J > MAX_J_BATCH) return set_error(ctx, OT_EUNSUPPORTED, "instance %d: J=%d above 1024 (batched)", k, a.J);
    const int64_t ld = a.ld ? a.ld : a.J;
    if (ld < a.J || ld % 4 != 0 || ((uintptr_t)a.C & 15u))
        return set_error(ctx, OT_EINVAL, "instance %d: C must be 16-byte aligned with ld %% 4 == 0 and ld >= J", k);
    if (!(a.eps > 0.0) || !std::isfinite(a.eps)) return set_error(ctx, OT_EINVAL, "instance %d: eps", k);
    if (!(a.tol >= 0.0)) return set_error(ctx, OT_EINVAL, "instance %d: tol", k);
    if (a.max_iter < 1) return set_error(ctx, OT_EINVAL, "instance %d: max_iter", k);
    if (a.pi && a.pi_ld != 0 && a.pi_ld < a.J) return set_error(ctx, OT_EINVAL, "instance %d: pi_ld < J", k);
    return OT_OK;
}

// Fill the descriptor fields that depend only on the instance's values (not its shape).
static void fill_values(BInst* d, const ot_assoc_instance& a) {
    SolveParams& P = d->P;
    P.C = a.C;
    P.ld = a.ld ? a.ld : a.J;
    P.I = a.I;
    P.J = a.J;
    P.Jp = (int)round_up(a.J, 4);
    P.p = a.p;
    P.q = a.q;
    P.g_warm = a.warm_start ? a.g : nullptr;
    P.k = LOG2E / a.eps;
    split_k(P.k, &P.k_hi, &P.k_lo);
    P.tol = a.tol;
    P.max_iter = a.max_iter;
    d->eps_ln2 = a.eps * LN2;
    d->f_out = a.f;
    d->g_out = a.g;
    d->rrh_load = a.rrh_load;
    d->pi = a.pi;
    d->pi_ld = a.pi ? (a.pi_ld ? a.pi_ld : a.J) : 0;
}

static void batch_free(ot_assoc_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->dmem) {
        cudaFree(b->dmem);
        b->ctx->held -= b->dbytes;
    }
    if (b->h_inst) cudaFreeHost(b->h_inst);
    if (b->h_res) cudaFreeHost(b->h_res);
    b->exec = nullptr;
    b->graph = nullptr;
    b->stream = nullptr;
    b->dmem = nullptr;
    b->h_inst = nullptr;
    b->h_res = nullptr;
}

// Group size and stage target of an instance: the tuned entry of its bucket, else defaults.
static void choose(const ot_assoc_ctx* ctx, int64_t I, int J, int* gsize, int* stage) {
    const int bk = batch_bucket(I, J);
    const TuneEntry& t = ctx->tune[bk];
    *gsize = t.gsize > 0 ? t.gsize : default_gsize(I, J, ctx->num_sms);
    *stage = t.stage > 0 ? t.stage : 24576;
    const int64_t blocks = (I + BT_NCW - 1) / BT_NCW;
    while (*gsize > 1 && *gsize > blocks) {  // every CTA of a group owns at least one row block
        int next = 1;
        for (int d : divisors(ctx->num_sms))
            if (d < *gsize) next = d;
        *gsize = next;
    }
}

// Plan the schedule and device layout; forced_gsize / forced_stage (> 0) override the choice
// for every instance (used by the autotuner).
static ot_status batch_plan(ot_assoc_batch* b, int forced_gsize, int forced_stage) {
    ot_assoc_ctx* ctx = b->ctx;
    const int n = b->n;
    const int nsm = ctx->num_sms;
    std::vector<int> gs(n), stg(n);
    std::vector<BInst> d(n);
    size_t smem = 0;
    for (int k = 0; k < n; ++k) {
        const ot_assoc_instance& a = b->inst[k];
        int g, st;
        choose(ctx, a.I, a.J, &g, &st);
        if (forced_gsize > 0) g = forced_gsize;
        if (forced_stage > 0) st = forced_stage;
        std::memset(&d[k], 0, sizeof(BInst));
        fill_values(&d[k], a);
        d[k].vpt = vpt_for(a.J);
        size_t sm = 0;
        int ft = 0;
        // grow the group until the CTA's share of the rows fits next to two stages
        bool ok = false;
        for (;;) {
            if (plan_stream(a.I, d[k].P.Jp, d[k].P.ld, g, st, &d[k].S, &sm, &ft)) {
                ok = true;
                break;
            }
            int next = 0;
            for (int dv : divisors(nsm))
                if (dv > g) {
                    next = dv;
                    break;
                }
            if (!next) break;
            g = next;
        }
        if (!ok) return set_error(ctx, OT_EUNSUPPORTED, "instance %d (I=%lld J=%d) does not fit the shared memory", k,
                                  (long long)a.I, a.J);
        d[k].fin_teams = ft;
        gs[k] = g;
        stg[k] = st;
        smem = std::max(smem, sm);
    }
    // phases: one per group size, largest groups first; inside a phase, largest instances first
    std::vector<int> sizes(gs.begin(), gs.end());
    std::sort(sizes.begin(), sizes.end(), std::greater<int>());
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    if ((int)sizes.size() > 16) return set_error(ctx, OT_EUNSUPPORTED, "too many phases");
    b->h_phases.clear();
    b->h_order.clear();
    b->h_goff.clear();
    int ngroups_total = 0;
    std::vector<size_t> phase_jp, phase_gsz;
    for (int g : sizes) {
        BPhase ph;
        ph.gsize = g;
        ph.ngroups = nsm / g;
        ph.first = (int)b->h_order.size();
        std::vector<int> idx;
        int jpmax = 4;
        for (int k = 0; k < n; ++k)
            if (gs[k] == g) {
                idx.push_back(k);
                jpmax = std::max(jpmax, d[k].P.Jp);
            }
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
            return (double)b->inst[x].I * b->inst[x].J > (double)b->inst[y].I * b->inst[y].J;
        });
        ph.count = (int)idx.size();
        b->h_order.insert(b->h_order.end(), idx.begin(), idx.end());
        b->h_goff.push_back(ngroups_total);
        ngroups_total += ph.ngroups;
        b->h_phases.push_back(ph);
        phase_jp.push_back((size_t)jpmax);
        phase_gsz.push_back((size_t)g);
    }
    // device layout: [inst][res][ctl][gbar][gcur][order][phases][goff][groups][group scratch...]
    auto al = [](size_t x) { return (size_t)round_up((int64_t)x, 256); };
    size_t off = 0;
    const size_t o_inst = off;
    off = al(off + sizeof(BInst) * n);
    const size_t o_res = off;
    off = al(off + sizeof(BRes) * n);
    const size_t o_ctl = off;
    off = al(off + sizeof(BCtl));
    const size_t o_gbar = off;
    off = al(off + sizeof(unsigned) * ngroups_total);
    const size_t o_gcur = off;
    off = al(off + sizeof(int) * ngroups_total);
    const size_t zero_end = off;
    const size_t o_order = off;
    off = al(off + sizeof(int) * n);
    const size_t o_phases = off;
    off = al(off + sizeof(BPhase) * b->h_phases.size());
    const size_t o_goff = off;
    off = al(off + sizeof(int) * b->h_goff.size());
    const size_t o_groups = off;
    off = al(off + sizeof(BGroup) * ngroups_total);
    std::vector<size_t> g_off(ngroups_total);
    std::vector<size_t> g_sizes(ngroups_total);
    {
        int gi = 0;
        for (size_t p = 0; p < b->h_phases.size(); ++p) {
            const size_t Jp = phase_jp[p], nb = phase_gsz[p];
            const size_t bytes = 1024 + al(3 * Jp * 8) + al(nb * 2 * Jp * 4) + al(nb * 16) + al(nb * Jp * 16) +
                                 al(nb * BT_NW * 16 + nb * 8);
            for (int q = 0; q < b->h_phases[p].ngroups; ++q, ++gi) {
                g_off[gi] = off;
                g_sizes[gi] = bytes;
                off = al(off + bytes);
            }
        }
    }
    const size_t total = off;
    // (re)allocate
    batch_free(b);
    if (ctx->budget && ctx->held + total > ctx->budget)
        return set_error(ctx, OT_ENOMEM, "batch tables need %zu bytes: over the HBM budget", total);
    cudaError_t e = cudaMalloc(&b->dmem, total);
    if (e != cudaSuccess) return cuda_error(ctx, e, "cudaMalloc (batch)");
    b->dbytes = total;
    ctx->held += total;
    e = cudaMallocHost((void**)&b->h_inst, sizeof(BInst) * n);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_res, sizeof(BRes) * n);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_error(ctx, e, "cudaMallocHost (batch)");
    }
    char* base = (char*)b->dmem;
    b->d_inst = (BInst*)(base + o_inst);
    b->d_res = (BRes*)(base + o_res);
    b->d_ctl = (BCtl*)(base + o_ctl);
    b->d_gbar = (unsigned*)(base + o_gbar);
    b->d_gcur = (int*)(base + o_gcur);
    b->zero_bytes = zero_end - o_res;
    b->h_groups.resize(ngroups_total);
    {
        int gi = 0;
        for (size_t p = 0; p < b->h_phases.size(); ++p) {
            const size_t Jp = phase_jp[p], nb = phase_gsz[p];
            for (int q = 0; q < b->h_phases[p].ngroups; ++q, ++gi) {
                char* g = base + g_off[gi];
                BGroup& G = b->h_groups[gi];
                G.sc = (DevScalars*)g;
                G.ls = (LoopState*)(g + 512);
                size_t o = 1024;
                G.G = (double*)(g + o);
                o += al(3 * Jp * 8);
                G.colpart = (float*)(g + o);
                o += al(nb * 2 * Jp * 4);
                G.errpart = (double*)(g + o);
                o += al(nb * 16);
                G.fpart = (double2*)(g + o);
                o += al(nb * Jp * 16);
                G.fred = (double*)(g + o);
            }
        }
    }
    std::memcpy(b->h_inst, d.data(), sizeof(BInst) * n);
    e = cudaMemcpy(base + o_order, b->h_order.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + o_phases, b->h_phases.data(), sizeof(BPhase) * b->h_phases.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + o_goff, b->h_goff.data(), sizeof(int) * b->h_goff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + o_groups, b->h_groups.data(), sizeof(BGroup) * ngroups_total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_error(ctx, e, "batch table upload");
    }
    BatchParams& BP = b->params;
    BP.inst = b->d_inst;
    BP.res = b->d_res;
    BP.order = (const int*)(base + o_order);
    BP.phases = (const BPhase*)(base + o_phases);
    BP.nphases = (int)b->h_phases.size();
    BP.groups = (const BGroup*)(base + o_groups);
    BP.goff = (const int*)(base + o_goff);
    BP.ctl = b->d_ctl;
    BP.gbar = b->d_gbar;
    BP.gcur = b->d_gcur;
    BP.spin = ctx->spin_limit;
    b->smem = smem;
    b->grid = nsm;
    if (cudaFuncSetAttribute((const void*)sk_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return set_error(ctx, OT_ECUDA, "batched kernel: %zu bytes of shared memory refused", smem);
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)sk_batch, BT_NT, smem) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        batch_free(b);
        return set_error(ctx, OT_EUNSUPPORTED, "batched kernel cannot be resident");
    }
    return OT_OK;
}

// Enqueue one run: descriptors in, control words cleared, the persistent kernel, results out.
static cudaError_t batch_enqueue(ot_assoc_batch* b, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(b->d_inst, b->h_inst, sizeof(BInst) * b->n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->d_res, 0, b->zero_bytes, s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(BT_NT);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, sk_batch, b->params);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(b->h_res, b->d_res, sizeof(BRes) * b->n, cudaMemcpyDeviceToHost, s);
}

static ot_status batch_capture(ot_assoc_batch* b) {
    ot_assoc_ctx* ctx = b->ctx;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (!b->stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_error(ctx, e, "stream for capture");
    }
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_error(ctx, e, "begin capture");
    cudaError_t e2 = batch_enqueue(b, b->stream);
    e = cudaStreamEndCapture(b->stream, &b->graph);
    if (e2 != cudaSuccess) return cuda_error(ctx, e2, "batched launch capture");
    if (e != cudaSuccess) return cuda_error(ctx, e, "end capture");
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return cuda_error(ctx, e, "graph instantiate");
    return OT_OK;
}

static ot_status batch_status(ot_assoc_ctx* ctx, const BRes& r, ot_assoc_instance_result* o) {
    o->transport_cost = r.cost;
    o->marg_err_row = r.err_row;
    o->marg_err_col = r.err_col;
    o->err_loop = r.err_loop;
    o->iters = r.iters;
    int st;
    if (!r.done) st = OT_ETIMEOUT;
    else if (r.status == DEV_EINVAL) st = OT_EINVAL;
    else if (r.status == DEV_ENUMERIC) st = OT_EINVAL;
    else if (r.status == DEV_ETIMEOUT) st = OT_ETIMEOUT;
    else if (r.status != DEV_OK) st = OT_ECUDA;
    else st = r.converged ? OT_OK : OT_NOT_CONVERGED;
    o->status = st;
    o->converged = r.converged;
    o->reserved = 0;
    (void)ctx;
    return (ot_status)st;
}

ot_status batch_create(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int n, int flags, ot_assoc_batch** out,
                       int forced_gsize, int forced_stage) {
    *out = nullptr;
    if (n <= 0 || !inst) return set_error(ctx, OT_EINVAL, "empty batch");
    for (int k = 0; k < n; ++k) {
        ot_status st = batch_check(ctx, inst[k], k);
        if (st) return st;
    }
    ot_assoc_batch* b = new ot_assoc_batch;
    b->ctx = ctx;
    b->n = n;
    b->inst.assign(inst, inst + n);
    b->use_graph = !(flags & OT_BATCH_NO_GRAPH);
    ot_status st = batch_plan(b, forced_gsize, forced_stage);
    if (!st && b->use_graph) st = batch_capture(b);
    if (st) {
        batch_free(b);
        delete b;
        return st;
    }
    *out = b;
    return OT_OK;
}

ot_status batch_launch(ot_assoc_batch* b, cudaStream_t s) {
    ot_assoc_ctx* ctx = b->ctx;
    cudaError_t e;
    if (b->use_graph) {
        e = cudaGraphLaunch(b->exec, s);
    } else {
        e = batch_enqueue(b, s);
    }
    if (e != cudaSuccess) return cuda_error(ctx, e, "batched launch");
    ctx->launches += 1;
    return OT_OK;
}

ot_status batch_wait(ot_assoc_batch* b, cudaStream_t s, ot_assoc_instance_result* res) {
    ot_assoc_ctx* ctx = b->ctx;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "batched solve");
    int aborted = 0;
    for (int k = 0; k < b->n; ++k) {
        ot_assoc_instance_result tmp;
        batch_status(ctx, b->h_res[k], res ? &res[k] : &tmp);
        if (!b->h_res[k].done) aborted = 1;
    }
    if (aborted) return set_error(ctx, OT_ETIMEOUT, "a device-side wait of the batched launch exceeded its spin limit");
    ctx->err.clear();
    return OT_OK;
}

void batch_destroy(ot_assoc_batch* b) {
    if (!b) return;
    DeviceGuardLite g(b->ctx->device);
    batch_free(b);
    delete b;
}

ot_status batch_set(ot_assoc_batch* b, int k, const ot_assoc_instance* a) {
    ot_assoc_ctx* ctx = b->ctx;
    if (k < 0 || k >= b->n || !a) return set_error(ctx, OT_EINVAL, "bad instance index");
    ot_status st = batch_check(ctx, *a, k);
    if (st) return st;
    const ot_assoc_instance& o = b->inst[k];
    const int64_t ld_o = o.ld ? o.ld : o.J, ld_a = a->ld ? a->ld : a->J;
    if (a->I != o.I || a->J != o.J || ld_a != ld_o)
        return set_error(ctx, OT_EINVAL, "instance %d: shape (I, J, ld) differs from the planned one", k);
    b->inst[k] = *a;
    fill_values(&b->h_inst[k], *a);
    return OT_OK;
}

// ------------------------------------------------------------------------------------------
// Autotuner.  For each size bucket present in `inst`, time the candidate (group size, stage
// size) pairs on that bucket's instances (replicated so that every group of the phase has
// work), with a fixed number of iterations and outputs sent to scratch, and keep the pair
// with the highest cells * iterations / s.  Results go into the context's tuning table.
// ------------------------------------------------------------------------------------------
ot_status batch_autotune(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int n, int iters, cudaStream_t s) {
    if (iters < 3) iters = 3;
    std::vector<std::vector<int>> by_bucket(TUNE_BUCKETS);
    for (int k = 0; k < n; ++k) {
        ot_status st = batch_check(ctx, inst[k], k);
        if (st) return st;
        by_bucket[batch_bucket(inst[k].I, inst[k].J)].push_back(k);
    }
    const std::vector<int> divs = divisors(ctx->num_sms);
    const int stages[3] = {12288, 24576, 49152};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return set_error(ctx, OT_ECUDA, "autotune events");
    }
    ot_status result = OT_OK;
    for (int bk = 0; bk < TUNE_BUCKETS && !result; ++bk) {
        if (by_bucket[bk].empty()) continue;
        // sample: up to 4 instances of the bucket; their largest Jp and I size the scratch
        std::vector<int> sample(by_bucket[bk].begin(), by_bucket[bk].begin() + std::min<size_t>(4, by_bucket[bk].size()));
        int64_t Imax = 0;
        int Jmax = 0;
        int64_t blocks_min = INT64_MAX;
        for (int k : sample) {
            Imax = std::max(Imax, inst[k].I);
            Jmax = std::max(Jmax, inst[k].J);
            blocks_min = std::min(blocks_min, (inst[k].I + BT_NCW - 1) / BT_NCW);
        }
        const int g0 = default_gsize(inst[sample[0]].I, inst[sample[0]].J, ctx->num_sms);
        double best_rate = -1.0;
        TuneEntry best = {};
        for (int gsz : divs) {
            if (gsz > blocks_min || gsz * 8 < g0 || gsz > g0 * 8) continue;
            const int ngroups = ctx->num_sms / gsz;
            const int reps = std::max<int>(2 * ngroups, (int)sample.size());
            std::vector<ot_assoc_instance> tb(reps);
            // outputs to scratch: f, g per replica (never the caller's buffers)
            ot_status st = OT_OK;
            const size_t per = (size_t)round_up(Imax, 32) + (size_t)round_up(Jmax, 32);
            double* outbuf = (double*)scratch(ctx, SLOT_TUNE, sizeof(double) * per * reps, &st);
            if (st) {
                result = st;
                break;
            }
            double cells_iter = 0.0;
            for (int r = 0; r < reps; ++r) {
                tb[r] = inst[sample[r % sample.size()]];
                tb[r].f = outbuf + per * r;
                tb[r].g = outbuf + per * r + round_up(Imax, 32);
                tb[r].rrh_load = nullptr;
                tb[r].pi = nullptr;
                tb[r].warm_start = 0;
                tb[r].tol = 0.0;
                tb[r].max_iter = iters;
                cells_iter += (double)tb[r].I * tb[r].J * (iters + 1);
            }
            for (int stg : stages) {
                ot_assoc_batch* b = nullptr;
                st = batch_create(ctx, tb.data(), reps, OT_BATCH_NO_GRAPH, &b, gsz, stg);
                if (st == OT_EUNSUPPORTED) {
                    ctx->err.clear();
                    continue;
                }
                if (st) {
                    result = st;
                    break;
                }
                float ms = 0.f;
                st = batch_launch(b, s);  // warm-up
                if (!st) st = batch_wait(b, s, nullptr);
                if (!st) {
                    cudaEventRecord(e0, s);
                    st = batch_launch(b, s);
                    cudaEventRecord(e1, s);
                    if (!st) st = batch_wait(b, s, nullptr);
                    if (!st && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        cudaGetLastError();
                        ms = 0.f;
                    }
                }
                batch_destroy(b);
                if (st) {
                    result = st;
                    break;
                }
                const double rate = ms > 0.f ? cells_iter / (ms * 1e-3) : 0.0;
                if (rate > best_rate) {
                    best_rate = rate;
                    best.gsize = gsz;
                    best.stage = stg;
                    best.rate = rate;
                }
            }
            if (result) break;
        }
        if (!result && best.gsize > 0) ctx->tune[bk] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return result;
}

}  // namespace ota
