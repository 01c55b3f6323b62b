// Device code shared by the batched and the serving persistent kernels: a group of CTAs
// solves one instance (Algorithm 1 of the paper, Sec. III-B) with the solver core and
// finalizes it in the same launch.
#pragma once

#include <cuda_runtime.h>

#include "ot_common.cuh"
#include "sk_core.cuh"
#include "ot_internal.h"

namespace ota {

static constexpr int BT_NCW = Cons<1>::NCW;  // consumer warps (one-warp teams)
static constexpr int BT_NT = Cons<1>::NT;    // + the producer warp
static constexpr int BT_NW = BT_NT / 32;

// One instance as the kernel sees it (host-written).
struct BInst {
    SolveParams P;  // C, ld, I, J, Jp, p, q, g_warm, k, k_hi, k_lo, tol, max_iter (scratch filled per group)
    StreamCfg S;    // stage geometry and shared-memory layout at this instance's group size
    int vpt;        // float4 chunks per lane (J4 <= 32 * vpt)
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

// Scratch of one group (sized for the largest instance of its phase).
struct BGroup {
    DevScalars* sc;
    LoopState* ls;
    double* G;         // gstate_words(Jp)
    float* colpart;    // [V][2 * Jp]
    double* errpart;   // [V] (x2)
    double2* fpart;    // [V][Jp] finalize column partials
    double* fred;      // [gsize][BT_NW][2] finalize totals per warp; then [V] row residuals
    int phase;         // the queue this group takes instances from
    int first_cta;     // the group is CTAs [first_cta, first_cta + gsize)
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

// Finish one instance after the solver's finalize sweep (which left per-CTA FP64 column
// partials and row residuals in the group's scratch): one warp per column over the group's
// CTAs in order, then the group's leader forms the totals.
__device__ __forceinline__ bool bt_finalize(const BInst& D, const SolveParams& P, const BGroup& grp, int rank,
                                            int gsize, int par, unsigned* gbar, unsigned* s_gen, int* abort,
                                            long long spin, BRes* out) {
    const int J = P.J, Jp = P.Jp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* Gk = P.G + par * Jp;
    if (!group_sync(gbar, gsize, s_gen, abort, spin)) return false;
    {
        const double inv_sq = P.sc->inv_sq, sp = P.sc->sp;
        double ec = 0.0, co = 0.0;
        const int gw = rank * BT_NW + warp, nw = gsize * BT_NW;
        for (int j = gw; j < J; j += nw) {
            double s = 0.0, r = 0.0;
            for (int bb = lane; bb < P.V; bb += 32) {
                const double2 v = grp.fpart[(int64_t)bb * Jp + j];
                s += v.x;
                r += v.y;
            }
            s = warp_sum(s);
            r = warp_sum(r);
            if (lane == 0) {
                ec += fabs(s - (double)__ldcg(P.q + j) * inv_sq);
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
        const double* rowerr = grp.fred + (size_t)gsize * BT_NW * 2;
        double ec = 0.0, co = 0.0, er = 0.0;
        for (int k = 0; k < gsize * BT_NW; ++k) {
            ec += grp.fred[2 * k];
            co += grp.fred[2 * k + 1];
        }
        for (int k = 0; k < P.V; ++k) er += rowerr[k];
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
__device__ __noinline__ bool bt_instance(const BInst& D, BRes* out, int* abort, long long spin, const BGroup& grp,
                                            int rank, int gsize, unsigned* gbar, unsigned* s_gen, int* s_nbar,
                                            SkShared* sh, unsigned char* dyn) {
    // the instance's parameters with the group's scratch, in shared memory: the solver reads
    // its fields from there as a single-instance kernel reads its parameter block, instead of
    // holding a copy in registers
    __shared__ SolveParams s_P;
    if (threadIdx.x == 0) {
        SolveParams P = D.P;
        P.sc = grp.sc;
        P.st = grp.ls;
        P.G = grp.G;
        P.colpart = grp.colpart;
        P.errpart = grp.errpart;
        P.F_out = nullptr;
        P.spin = spin;
        P.fpart = grp.fpart;
        P.epart = grp.fred + (size_t)gsize * BT_NW * 2;
        P.pi = D.pi;
        P.pi_ld = D.pi_ld;
        P.f_nat = D.f_out;
        P.eps_ln2 = D.eps_ln2;
        P.F_in = nullptr;
        P.G_in = nullptr;
        P.dev_xy = nullptr;
        P.rrh_xy = nullptr;
        s_P = P;
    }
    __syncthreads();
    const SolveParams& P = s_P;
    const StreamCfg S = D.S;
    uint64_t* full = reinterpret_cast<uint64_t*>(dyn);
    uint64_t* empty = full + MAX_STAGES;
    float* ring = reinterpret_cast<float*>(dyn + S.off_ring);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t r0, r1;
    cta_rows(P.I, S.rows_per_stage, P.V, rank, gsize, &r0, &r1);
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
        if (lane == 0) stream_rows_producer(P.C, P.ld, r0, r1, S, ring, full, empty, &sh->s_stop, abort, spin);
    } else {
        // the instance's status word is its result slot (zeroed = DEV_OK before the launch):
        // a group's shared words are reused by the next instance while a slow CTA may still be
        // reading this one's status after the barrier that ended it
        GroupCtx g{gsize, rank, gbar, *s_gen, abort, &out->status};
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
            out->iters = 0;
            out->converged = 0;
            out->done = 1;
        }
        return true;
    }
    return bt_finalize(D, P, grp, rank, gsize, s_res - 1, gbar, s_gen, abort, spin, out);
}

// One instance by the group, dispatched on its chunks per lane.
__device__ __forceinline__ bool bt_run(const BInst& D, BRes* out, int* abort, long long spin, const BGroup& grp,
                                       int rank, int gsize, unsigned* gbar, unsigned* s_gen, int* s_nbar, SkShared* sh,
                                       unsigned char* dyn) {
    switch (D.vpt) {
        case 1: return bt_instance<1>(D, out, abort, spin, grp, rank, gsize, gbar, s_gen, s_nbar, sh, dyn);
        case 2: return bt_instance<2>(D, out, abort, spin, grp, rank, gsize, gbar, s_gen, s_nbar, sh, dyn);
        case 3: return bt_instance<3>(D, out, abort, spin, grp, rank, gsize, gbar, s_gen, s_nbar, sh, dyn);
        case 4: return bt_instance<4>(D, out, abort, spin, grp, rank, gsize, gbar, s_gen, s_nbar, sh, dyn);
        case 5: return bt_instance<5>(D, out, abort, spin, grp, rank, gsize, gbar, s_gen, s_nbar, sh, dyn);
        case 6: return bt_instance<6>(D, out, abort, spin, grp, rank, gsize, gbar, s_gen, s_nbar, sh, dyn);
        case 7: return bt_instance<7>(D, out, abort, spin, grp, rank, gsize, gbar, s_gen, s_nbar, sh, dyn);
        default: return bt_instance<8>(D, out, abort, spin, grp, rank, gsize, gbar, s_gen, s_nbar, sh, dyn);
    }
}

// ---- host helpers ----------------------------------------------------------------------
static constexpr size_t SMEM_BUDGET = 232448 - 4096;  // 227 KB per block minus static shared memory
static constexpr int MAX_J_BATCH = 1024;              // one-warp teams: J4 <= 32 * 8

inline int vpt_for(int J) { return std::max(1, (int)((round_up(J, 4) / 4 + 31) / 32)); }

// Stage geometry and shared-memory layout of one instance solved by nb CTAs.
inline bool plan_stream(int64_t I, int Jp, int64_t ld, int nb, int stage_target, StreamCfg* S, size_t* smem, int* V) {
    return plan_stage(BT_NCW, I, Jp, ld, nb, stage_target, SMEM_BUDGET, S, smem, V);
}

// Fill the descriptor fields that depend only on the instance's values (not its shape).
inline void fill_values(BInst* d, const ot_assoc_instance& a) {
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

}  // namespace ota
