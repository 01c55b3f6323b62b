// Entropic-OT Sinkhorn solver, FP32 log domain (Algorithm 1 of the paper, Sec. III-B).
//
// Notation (log2 units, so every exponential is one MUFU.EX2):
//   k      = log2(e) / eps, split k = k_hi + k_lo (two FP32 numbers, ~2^-48 relative).
//   G_j    = g_j * k                    column potential (b_j = 2^G_j)
//   F'_i   = f_i * k - log2 p_i         row potential relative to the row mass
//   t_ij   = 2^(F'_i + G_j - k C_ij)    = pi_ij / p_i of the current plan
//
// One persistent cooperative launch does the whole iteration:
//   setup      marginal sums and checks, starting column potentials (b = 1 or warm start);
//   sweep 1    the exact log-domain first iteration: a row log-sum-exp with the row maximum
//              factored out, then a column log-sum-exp kept as an online (max, sum) pair per
//              column, so no column can underflow however far the start is;
//   sweeps 2.. every plan pi^(k-1) now has exact columns (sum q_j <= 1) and rows
//              >= p_i min q, so iteration k works on t_ij = pi^(k-1)_ij / p_i directly: one
//              read of C and ONE exp per cell give
//                a-update  r_i = sum_j t_ij,                 F'_i <- F'_i - log2 r_i
//                b-update  s_j = sum_i t_ij p^_i / r_i,      G_j <- G_j + log2 q^_j - log2 s_j
//              and r_i is also the row sum of pi^(k-1): the loop test ("while accuracy") on
//              that plan's row residual is one sweep late, so the previous F' (the other
//              shared-memory buffer) is what a stop returns.
// Each CTA owns a fixed block-aligned range of rows for the whole solve; its row potentials
// (an FP32 hi/lo pair, updated with error-free FP32 two-sums) and p^ live in shared memory.
// A producer warp streams the CTA's rows of C through a ring of shared-memory stages with
// bulk copies (TMA); it runs on into the next sweep while the consumers are in a grid
// barrier (C never changes).  Column partials are combined per CTA in team order and
// across CTAs in CTA order, so reruns are bit-identical.  Every wait is bounded.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "ot_common.cuh"
#include "sk_core.cuh"
#include "sk_multi.cuh"
#include "ot_internal.h"

namespace ota {

template <int TW, int VPT>
__global__ void __launch_bounds__(Cons<TW>::NT, 1) sk_solve(SolveParams P, StreamCfg S) {
    constexpr int NCW = Cons<TW>::NCW;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ SkShared sh;
    uint64_t* full = reinterpret_cast<uint64_t*>(dyn);
    uint64_t* empty = full + MAX_STAGES;
    float* ring = reinterpret_cast<float*>(dyn + S.off_ring);
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
            stream_rows_producer(P.C, P.ld, r0, r1, S, ring, full, empty, &sh.s_stop, &P.st->status, P.spin);
        return;
    }
    GroupCtx g{(int)gridDim.x, (int)blockIdx.x, &P.st->bar, 0u, &P.st->status, &P.st->status};
    int par = 0;
    sk_consumers<TW, VPT>(P, S, g, &sh, dyn, r0, r1, &par);
}

// Euclidean cost formed on the fly (Sec. IV cost choice (i)): no matrix is read, so there is
// no producer warp (the block is the consumer warps alone, which leaves each thread more
// registers); the RRH coordinates are staged once in the ring's space and every sweep forms
// C_ij = ||x_i - x_j|| from them and the device's coordinates.
template <int TW, int VPT>
__global__ void __launch_bounds__(Cons<TW>::NCW * 32, 1) sk_solve_euclid(SolveParams P, StreamCfg S) {
    constexpr int NCW = Cons<TW>::NCW;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ SkShared sh;
    float* rx = reinterpret_cast<float*>(dyn + S.off_ring);
    for (int j = threadIdx.x; j < P.Jp; j += blockDim.x) {
        const float2 r = j < P.J ? P.rrh_xy[j] : make_float2(0.f, 0.f);
        rx[j] = r.x;
        rx[P.Jp + j] = r.y;
    }
    if (threadIdx.x == 0) {
        sh.s_stop = 0;
        sh.s_bad = 0;
    }
    __syncthreads();
    int64_t r0, r1;
    cta_rows(P.I, S.rows_per_stage, P.V, blockIdx.x, gridDim.x, &r0, &r1);
    GroupCtx g{(int)gridDim.x, (int)blockIdx.x, &P.st->bar, 0u, &P.st->status, &P.st->status};
    int par = 0;
    sk_consumers<TW, VPT, true>(P, S, g, &sh, dyn, r0, r1, &par);
}

// Several solves sharing one cost matrix (sk_multi.cuh): the same launch structure.
template <int TW, int VPT, int NS, bool RC>
__global__ void __launch_bounds__(Cons<TW>::NT, 1) sk_solve_multi(MultiParams M, StreamCfg S) {
    constexpr int NCW = Cons<TW>::NCW;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ SkShared sh;
    uint64_t* full = reinterpret_cast<uint64_t*>(dyn);
    uint64_t* empty = full + MAX_STAGES;
    float* ring = reinterpret_cast<float*>(dyn + S.off_ring);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SolveParams& P0 = M.P[0];
    int64_t r0, r1;
    cta_rows(P0.I, S.rows_per_stage, P0.V, blockIdx.x, gridDim.x, &r0, &r1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        sh.s_stop = 0;
        sh.s_bad = 0;
        sh.s_dec = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == NCW) {
        if (lane == 0)
            stream_rows_producer(P0.C, P0.ld, r0, r1, S, ring, full, empty, &sh.s_stop, &M.grp->status, P0.spin);
        return;
    }
    GroupCtx g{(int)gridDim.x, (int)blockIdx.x, &M.grp->bar, 0u, &M.grp->status, &M.grp->status};
    ms_consumers<TW, VPT, NS, RC>(M, S, g, &sh, dyn, r0, r1);
}

// The launch's status into every solve's loop state (the finalize kernels read it there).
__global__ void sk_multi_status(const LoopState* grp, LoopState* a, LoopState* b, LoopState* c) {
    if (threadIdx.x == 0) {
        const int st = grp->status;
        a->status = st;
        if (b) b->status = st;
        if (c) c->status = st;
    }
}

// ------------------------------------------------------------------------------------------
// Finalize: the solver's last sweep (sk_finalize_sweep in sk_core.cuh) leaves per-CTA FP64
// column partials (sum p^ t, sum p^ C t) and row residuals; these kernels finish the column
// marginals, loads rho_j, potentials g in natural units, and the totals.
// ------------------------------------------------------------------------------------------
__global__ void sk_finalize_cols(const double2* __restrict__ fpart, int nb, int Jp, int J,
                                 const float* __restrict__ q, const DevScalars* sc,
                                 const LoopState* st, const double* G, int g_by_parity, double eps_ln2,
                                 double* g_out, double* rrh_load, double2* cols) {
    if (st->status != DEV_OK) return;
    if (g_by_parity) G += (st->iters & 1) * Jp;  // G^k of the returned plan
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
            cols[j] = make_double2(fabs(s - (double)q[j] * sc->inv_sq), r);
            if (rrh_load) rrh_load[j] = r * sc->sp;
            g_out[j] = eps_ln2 * G[j];
        }
    }
}

// Totals: row residual (per-CTA partials), column residual and transport cost = sum_j rho_j.
__global__ void sk_summary(const double* __restrict__ epart, int nb, const double2* __restrict__ cols, int J,
                           const DevScalars* sc, const LoopState* st, SolveSummary* out) {
    __shared__ double sh[3][32];
    double er = 0.0, co = 0.0, ec = 0.0;
    const bool ok = st->status == DEV_OK;
    if (ok) {
        for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) er += epart[bb];
        for (int j = threadIdx.x; j < J; j += blockDim.x) {
            const double2 c = cols[j];
            ec += c.x;
            co += c.y;
        }
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
        out->cost = ok ? c * sc->sp : 0.0;
        out->err_loop = st->err;
        out->iters = st->iters;
        out->converged = st->converged;
        out->status = st->status;
        out->absorptions = 0;
    }
}

// ------------------------------------------------------------------------------------------
// Host side.
// ------------------------------------------------------------------------------------------
namespace {

struct Kernels {
    const void* solve;
    int tw, vpt, ncw;
    int nthreads;  // block size: the consumer warps, plus the producer warp where C is streamed
};

template <int TW, int VPT, bool EUC>
Kernels kernels_for() {
    if constexpr (EUC) return Kernels{(const void*)sk_solve_euclid<TW, VPT>, TW, VPT, Cons<TW>::NCW, Cons<TW>::NCW * 32};
    else return Kernels{(const void*)sk_solve<TW, VPT>, TW, VPT, Cons<TW>::NCW, Cons<TW>::NT};
}

// One-warp teams (TW = 1) get VPT = ceil(J4 / 32) exactly; chunk_inside() relies on it.
template <bool EUC>
bool pick_kernels_t(int J, Kernels* k) {
    const int J4 = (J + 3) / 4;
    if (J4 <= 32) *k = kernels_for<1, 1, EUC>();
    else if (J4 <= 64) *k = kernels_for<1, 2, EUC>();
    else if (J4 <= 96) *k = kernels_for<1, 3, EUC>();
    else if (J4 <= 128) *k = kernels_for<1, 4, EUC>();
    else if (J4 <= 160) *k = kernels_for<1, 5, EUC>();
    else if (J4 <= 192) *k = kernels_for<1, 6, EUC>();
    else if (J4 <= 224) *k = kernels_for<1, 7, EUC>();
    else if (J4 <= 256) *k = kernels_for<1, 8, EUC>();
    else if (J4 <= 512) *k = kernels_for<2, 8, EUC>();
    else if (J4 <= 1024) *k = kernels_for<4, 8, EUC>();
    else if (J4 <= 2048) *k = kernels_for<8, 8, EUC>();
    else return false;
    return true;
}
bool pick_kernels(int J, Kernels* k) { return pick_kernels_t<false>(J, k); }

// Stage geometry, shared-memory layout and grid of the persistent kernel: one CTA per row
// partition (at most one per SM).
struct LoopLaunch {
    StreamCfg cfg;
    size_t smem;
    int grid;
    int V;
};

// Launch plans already made on this host thread (device, kernel and shape as the key): a
// repeated solve of one shape skips the planning and the attribute and occupancy queries.
struct PlanEntry {
    int device = -1;
    const void* fn = nullptr;
    int64_t I = 0, ld = 0;
    int Jp = 0, num_sms = 0, cap = 0;
    LoopLaunch L;
};
static constexpr int PLAN_CACHE = 8;
thread_local PlanEntry t_plans[PLAN_CACHE];
thread_local int t_plan_next = 0;

ot_status plan_solve_uncached(const Kernels& kk, int64_t I, int Jp, int64_t ld, int num_sms, int cap,
                              LoopLaunch* L);

ot_status plan_solve(const Kernels& kk, int64_t I, int Jp, int64_t ld, int num_sms, int cap, LoopLaunch* L) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return plan_solve_uncached(kk, I, Jp, ld, num_sms, cap, L);
    }
    for (const PlanEntry& e : t_plans)
        if (e.fn == kk.solve && e.device == dev && e.I == I && e.Jp == Jp && e.ld == ld && e.num_sms == num_sms &&
            e.cap == cap) {
            *L = e.L;
            return OT_OK;
        }
    const ot_status st = plan_solve_uncached(kk, I, Jp, ld, num_sms, cap, L);
    if (st == OT_OK) {
        PlanEntry& e = t_plans[t_plan_next];
        t_plan_next = (t_plan_next + 1) % PLAN_CACHE;
        e.device = dev;
        e.fn = kk.solve;
        e.I = I;
        e.Jp = Jp;
        e.ld = ld;
        e.num_sms = num_sms;
        e.cap = cap;
        e.L = *L;
    }
    return st;
}

ot_status plan_solve_uncached(const Kernels& kk, int64_t I, int Jp, int64_t ld, int num_sms, int cap,
                              LoopLaunch* L) {
    const int nteams = kk.ncw / kk.tw;
    const size_t budget = 232448 - 2048;  // 227 KB per block minus static shared memory
    StreamCfg S;
    size_t smem = 0;
    int V = 1;
    // the partitions depend on I and the stage rows only; ask with one CTA per partition
    if (!plan_stage(nteams, I, Jp, ld, 1, 24576, (size_t)1 << 40, &S, &smem, &V)) return OT_EUNSUPPORTED;
    const int grid = std::max(1, std::min({V, num_sms, cap}));
    if (!plan_stage(nteams, I, Jp, ld, grid, 24576, budget, &L->cfg, &L->smem, &L->V))
        return OT_EUNSUPPORTED;  // the rows a CTA owns do not fit next to two stages
    L->grid = grid;
    if (allow_max_dynamic_smem(kk.solve, L->smem) != cudaSuccess) {
        cudaGetLastError();
        return OT_ECUDA;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kk.solve, kk.nthreads, L->smem) != cudaSuccess) {
        cudaGetLastError();
        return OT_ECUDA;
    }
    if (occ < 1 || L->grid > occ * num_sms) return OT_EUNSUPPORTED;  // cooperative launch: all co-resident
    return OT_OK;
}

// Device buffers of one solve.
struct SolveBufs {
    DevScalars* sc;
    LoopState* ls;
    SolveSummary* summ;
    double2* cols;    // [Jp]
    double* G;        // gstate_words(Jp)
    double* errpart;  // [2][nb]: loop residual pairs, then the finalize row residuals
    void* colpart;    // [nb][Jp] float2
    double2* fpart;   // [nb][Jp]
};

// What one launch of the persistent kernel does (besides the full solve).
struct SolveMode {
    int init = 0;                // iteration 1 only, no finalize; F'^1 -> F_out, G^1 stays in B.G + Jp
    float2* F_out = nullptr;
    const float2* F_in = nullptr;  // finalize only, on these potentials (F' pairs, G log2 units)
    const double* G_in = nullptr;
    int iters = 0;               // reported with a finalize-only launch
    double err = 0.0;
    int converged = 0;
};

__global__ void sk_set_loop(LoopState* ls, int iters, double err, int converged) {
    if (threadIdx.x == 0) {
        ls->iters = iters;
        ls->err = err;
        ls->converged = converged;
    }
}

// Enqueue the whole solve (or the part `mode` asks for); the caller copies B.summ back.
cudaError_t enqueue_solve(const SolveArgs& a, const Kernels& kk, const LoopLaunch& LL, const SolveBufs& B,
                          long long spin, cudaStream_t s, ot_assoc_ctx* ctx, const SolveMode& mode = SolveMode(),
                          cudaEvent_t kev0 = nullptr, cudaEvent_t kev1 = nullptr) {
    const int J = a.J;
    const int64_t I = a.I;
    const int Jp = (int)round_up(J, 4);
    const double k = LOG2E / a.eps;
    float k_hi, k_lo;
    split_k(k, &k_hi, &k_lo);
    if (ctx) timing_mark(ctx, 0, s);
    cudaError_t e = cudaMemsetAsync(B.sc, 0, 1024, s);  // DevScalars, LoopState, summary
    if (e != cudaSuccess) return e;
    if (mode.F_in) sk_set_loop<<<1, 32, 0, s>>>(B.ls, mode.iters, mode.err, mode.converged);
    SolveParams P;
    P.C = a.C;
    P.ld = a.ld;
    P.I = I;
    P.J = J;
    P.Jp = Jp;
    P.V = LL.V;
    P.p = a.p;
    P.q = a.q;
    P.g_warm = a.warm_start ? a.out->g : nullptr;
    P.input_bad = a.input_bad;
    P.sc = B.sc;
    P.st = B.ls;
    P.G = B.G;
    P.F_out = mode.F_out;
    P.colpart = (float*)B.colpart;
    P.errpart = B.errpart;
    P.k = k;
    P.k_hi = k_hi;
    P.k_lo = k_lo;
    P.tol = mode.init ? 0.0 : a.tol;
    P.max_iter = mode.init ? 1 : a.max_iter;
    P.init_only = mode.init;
    P.spin = spin;
    P.fpart = mode.init ? nullptr : B.fpart;
    P.epart = B.errpart + LL.V;
    P.pi = a.out->pi;
    P.pi_ld = a.out->pi_ld > 0 ? a.out->pi_ld : J;
    P.f_nat = a.out->f;
    P.eps_ln2 = a.eps * LN2;
    P.F_in = mode.F_in;
    P.G_in = mode.G_in;
    P.dev_xy = a.dev_xy;
    P.rrh_xy = a.rrh_xy;
    if (ctx) timing_mark(ctx, 1, s);
    if (kev0) cudaEventRecord(kev0, s);
    {
        void* args[] = {&P, (void*)&LL.cfg};
        e = cudaLaunchCooperativeKernel(kk.solve, dim3(LL.grid), dim3(kk.nthreads), args, LL.smem, s);
        if (e != cudaSuccess) return e;
    }
    if (kev1) cudaEventRecord(kev1, s);
    if (ctx) timing_mark(ctx, 2, s);
    if (!mode.init) {
        const int nb_cols = (int)std::max<int64_t>(1, std::min<int64_t>((J + 15) / 16, 1024));
        const double* G = mode.G_in ? mode.G_in : B.G;
        sk_finalize_cols<<<nb_cols, 512, 0, s>>>(B.fpart, LL.V, Jp, J, a.q, B.sc, B.ls, G, mode.G_in ? 0 : 1,
                                                 a.eps * LN2, a.out->g, a.out->rrh_load, B.cols);
        sk_summary<<<1, 256, 0, s>>>(P.epart, LL.V, B.cols, J, B.sc, B.ls, B.summ);
    }
    if (ctx) timing_mark(ctx, 3, s);
    return cudaGetLastError();
}

// Scratch of a solve in context memory.
ot_status solve_bufs(ot_assoc_ctx* ctx, const LoopLaunch& LL, int Jp, SolveBufs* B) {
    ot_status st = OT_OK;
    B->colpart = scratch(ctx, SLOT_COLPART, sizeof(float2) * (size_t)LL.V * Jp, &st);
    if (st) return st;
    B->fpart = (double2*)scratch(ctx, SLOT_FINPART, sizeof(double2) * (size_t)LL.V * Jp, &st);
    if (st) return st;
    B->G = (double*)scratch(ctx, SLOT_G, gstate_bytes(Jp), &st);
    if (st) return st;
    B->errpart = (double*)scratch(ctx, SLOT_ERRPART, sizeof(double) * 2 * (size_t)LL.V, &st);
    if (st) return st;
    char* state = (char*)scratch(ctx, SLOT_STATE, 4096 + sizeof(double2) * (size_t)Jp, &st);
    if (st) return st;
    B->sc = (DevScalars*)state;
    B->ls = (LoopState*)(state + 256);
    B->summ = (SolveSummary*)(state + 512);
    B->cols = (double2*)(state + 4096);
    return OT_OK;
}

}  // namespace

ot_status enqueue_solve_f32(ot_assoc_ctx* ctx, const SolveArgs& a, SolveSummary* dest, cudaEvent_t kev0,
                            cudaEvent_t kev1) {
    ot_status st = OT_OK;
    const int J = a.J;
    const int64_t I = a.I;
    const int Jp = (int)round_up(J, 4);
    Kernels kk;
    const bool euc = a.dev_xy != nullptr;
    if (!(euc ? pick_kernels_t<true>(J, &kk) : pick_kernels(J, &kk)))
        return set_error(ctx, OT_EUNSUPPORTED, "J=%d above 8192", J);
    LoopLaunch LL;
    st = plan_solve(kk, I, Jp, a.ld, ctx->num_sms, 1 << 30, &LL);
    if (st) return set_error(ctx, st, "solver does not fit the shared memory (I=%lld J=%d)", (long long)I, J);
    SolveBufs B;
    st = solve_bufs(ctx, LL, Jp, &B);
    if (st) return st;
    cudaStream_t s = a.stream;
    cudaError_t e = enqueue_solve(a, kk, LL, B, ctx->spin_limit, s, kev0 ? nullptr : ctx, SolveMode(), kev0, kev1);
    if (e != cudaSuccess) return cuda_error(ctx, e, "solve launch");
    ctx->launches += 3;
    e = cudaMemcpyAsync(dest, B.summ, sizeof(SolveSummary), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "summary copy");
    return OT_OK;
}

// Kernels of the multi-solve launch.  Up to 128 float4 chunks a row, one-warp teams keep
// three solves' accumulators with the row (4 chunks a lane).  Wider rows: two solves on
// one-warp teams with the cell values computed twice (the row stays with the one-warp
// team of a single solve), three solves on wider teams (4 chunks a lane).
template <int TW, int VPT, int NS, bool RC>
Kernels multi_for() {
    return Kernels{(const void*)sk_solve_multi<TW, VPT, NS, RC>, TW, VPT, Cons<TW>::NCW, Cons<TW>::NT};
}
bool pick_multi(int J, int n, Kernels* k) {
    const int J4 = (J + 3) / 4;
    if (J4 <= 32) *k = multi_for<1, 1, 3, false>();
    else if (J4 <= 64) *k = multi_for<1, 2, 3, false>();
    else if (J4 <= 96) *k = multi_for<1, 3, 3, false>();
    else if (J4 <= 128) *k = multi_for<1, 4, 3, false>();
    else if (n <= 2 && J4 <= 160) *k = multi_for<1, 5, 2, true>();
    else if (n <= 2 && J4 <= 192) *k = multi_for<1, 6, 2, true>();
    else if (n <= 2 && J4 <= 224) *k = multi_for<1, 7, 2, true>();
    else if (n <= 2 && J4 <= 256) *k = multi_for<1, 8, 2, true>();
    else if (J4 <= 256) *k = multi_for<2, 4, 3, false>();
    else if (J4 <= 512) *k = multi_for<4, 4, 3, false>();
    else if (J4 <= 1024) *k = multi_for<8, 4, 3, false>();
    else return false;
    return true;
}

ot_status launch_solve_f32(ot_assoc_ctx* ctx, const SolveArgs& a, SolveSummary* sum_host) {
    ot_status st = OT_OK;
    SolveSummary* hsum = (SolveSummary*)host_staging(ctx, sizeof(SolveSummary), &st);
    if (st) return st;
    ctx->last_timings.valid = 0;
    st = enqueue_solve_f32(ctx, a, hsum, nullptr, nullptr);
    if (st) return st;
    cudaError_t e = cudaStreamSynchronize(a.stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "solve");
    *sum_host = *hsum;
    timing_collect(ctx, hsum->iters);
    return OT_OK;
}

// Several solves on one cost matrix (an eps sweep) in one launch; fills sum_host[0..n).
ot_status launch_solve_multi(ot_assoc_ctx* ctx, const SolveArgs& a, int n, const double* eps, const double* tol,
                             ot_assoc_result* const* outs, SolveSummary* sum_host) {
    const int J = a.J;
    const int64_t I = a.I;
    const int Jp = (int)round_up(J, 4);
    Kernels kk;
    if (!pick_multi(J, n, &kk)) return set_error(ctx, OT_EUNSUPPORTED, "J=%d above 4096 (multi-solve)", J);
    const int nteams = kk.ncw / kk.tw;
    StreamCfg S;
    size_t smem = 0;
    int V = 1;
    if (!plan_multi(nteams, n, I, Jp, a.ld, 1, 24576, (size_t)1 << 40, &S, &smem, &V))
        return set_error(ctx, OT_EUNSUPPORTED, "multi-solve: no stage plan");
    const int grid = std::max(1, std::min(V, ctx->num_sms));
    if (!plan_multi(nteams, n, I, Jp, a.ld, grid, 24576, 232448 - 2048, &S, &smem, &V))
        return set_error(ctx, OT_EUNSUPPORTED, "multi-solve: rows do not fit the shared memory (I=%lld J=%d)",
                         (long long)I, J);
    if (allow_max_dynamic_smem(kk.solve, smem) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, OT_ECUDA, "multi-solve kernel: %zu bytes of shared memory refused", smem);
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kk.solve, kk.nthreads, smem) != cudaSuccess ||
        occ < 1 || grid > occ * ctx->num_sms) {
        cudaGetLastError();
        return set_error(ctx, OT_EUNSUPPORTED, "multi-solve kernel cannot be resident");
    }
    // scratch: [grp state][per solve: state 4096 + cols, G, errpart, colpart, fpart]
    auto al = [](size_t x) { return (size_t)round_up((int64_t)x, 256); };
    const size_t st_bytes = al(4096 + sizeof(double2) * (size_t)Jp);
    const size_t per = st_bytes + al(sizeof(double) * 3 * (size_t)Jp) + al(sizeof(double) * 2 * (size_t)V) +
                       al(sizeof(float2) * (size_t)V * Jp) + al(sizeof(double2) * (size_t)V * Jp);
    ot_status st = OT_OK;
    char* base = (char*)scratch(ctx, SLOT_MISC, 256 + per * n, &st);
    if (st) return st;
    SolveSummary* hsum = (SolveSummary*)host_staging(ctx, sizeof(SolveSummary) * n, &st);
    if (st) return st;
    MultiParams M;
    std::memset(&M, 0, sizeof(M));
    M.n = n;
    M.grp = (LoopState*)base;
    struct Bufs {
        DevScalars* sc;
        LoopState* ls;
        SolveSummary* summ;
        double2* cols;
        double* G;
        double* errpart;
        float* colpart;
        double2* fpart;
    } B[MS_MAX];
    cudaStream_t s = a.stream;
    cudaError_t e = cudaMemsetAsync(base, 0, 256, s);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        char* q = base + 256 + per * k;
        e = cudaMemsetAsync(q, 0, 1024, s);
        B[k].sc = (DevScalars*)q;
        B[k].ls = (LoopState*)(q + 256);
        B[k].summ = (SolveSummary*)(q + 512);
        B[k].cols = (double2*)(q + 4096);
        size_t o = st_bytes;
        B[k].G = (double*)(q + o);
        o += al(sizeof(double) * 3 * (size_t)Jp);
        B[k].errpart = (double*)(q + o);
        o += al(sizeof(double) * 2 * (size_t)V);
        B[k].colpart = (float*)(q + o);
        o += al(sizeof(float2) * (size_t)V * Jp);
        B[k].fpart = (double2*)(q + o);
        SolveParams& P = M.P[k];
        const double kk2 = LOG2E / eps[k];
        P.C = a.C;
        P.ld = a.ld;
        P.I = I;
        P.J = J;
        P.Jp = Jp;
        P.V = V;
        P.p = a.p;
        P.q = a.q;
        P.g_warm = nullptr;
        P.input_bad = a.input_bad;
        P.sc = B[k].sc;
        P.st = B[k].ls;
        P.G = B[k].G;
        P.F_out = nullptr;
        P.colpart = B[k].colpart;
        P.errpart = k == 0 ? B[0].errpart : B[k].errpart;
        P.k = kk2;
        split_k(kk2, &P.k_hi, &P.k_lo);
        P.tol = tol[k];
        P.max_iter = a.max_iter;
        P.spin = ctx->spin_limit;
        P.fpart = B[k].fpart;
        P.epart = B[k].errpart + V;
        P.pi = outs[k]->pi;
        P.pi_ld = outs[k]->pi_ld > 0 ? outs[k]->pi_ld : J;
        P.f_nat = outs[k]->f;
        P.eps_ln2 = eps[k] * LN2;
        P.F_in = nullptr;
        P.G_in = nullptr;
    }
    if (e != cudaSuccess) return cuda_error(ctx, e, "multi-solve memset");
    ctx->last_timings.valid = 0;
    timing_mark(ctx, 0, s);
    timing_mark(ctx, 1, s);
    {
        void* args[] = {&M, &S};
        e = cudaLaunchCooperativeKernel(kk.solve, dim3(grid), dim3(kk.nthreads), args, smem, s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "multi-solve launch");
    }
    timing_mark(ctx, 2, s);
    sk_multi_status<<<1, 32, 0, s>>>(M.grp, B[0].ls, n > 1 ? B[1].ls : nullptr, n > 2 ? B[2].ls : nullptr);
    const int nb_cols = (int)std::max<int64_t>(1, std::min<int64_t>((J + 15) / 16, 1024));
    for (int k = 0; k < n; ++k) {
        sk_finalize_cols<<<nb_cols, 512, 0, s>>>(B[k].fpart, V, Jp, J, a.q, B[k].sc, B[k].ls, B[k].G, 1,
                                                 eps[k] * LN2, outs[k]->g, outs[k]->rrh_load, B[k].cols);
        sk_summary<<<1, 256, 0, s>>>(B[k].errpart + V, V, B[k].cols, J, B[k].sc, B[k].ls, B[k].summ);
    }
    timing_mark(ctx, 3, s);
    ctx->launches += 2 + 2 * n;
    e = cudaGetLastError();
    for (int k = 0; k < n && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(hsum + k, B[k].summ, sizeof(SolveSummary), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "multi-solve");
    int mx = 0;
    for (int k = 0; k < n; ++k) {
        sum_host[k] = hsum[k];
        mx = std::max(mx, hsum[k].iters);
    }
    // the launch reads C once per fused sweep (max iters of the solves) and twice per solve
    // (its first iteration and its finalize sweep): sweeps + 2 = max iters + 2 n
    timing_collect(ctx, mx + 2 * n - 2);
    return OT_OK;
}

// Iteration 1 of the FP32 log-domain solver (the exact first sweep and the b-update):
// F'^1 (pairs) into F_out, G^1 (log2 units) into G_out.  Synchronises; *status gets the
// device status (invalid input is reported here).
ot_status f32_first_iteration(ot_assoc_ctx* ctx, const SolveArgs& a, float2* F_out, double* G_out, int* status) {
    ot_status st = OT_OK;
    const int J = a.J;
    const int Jp = (int)round_up(J, 4);
    Kernels kk;
    if (!pick_kernels(J, &kk)) return set_error(ctx, OT_EUNSUPPORTED, "J=%d above 8192", J);
    LoopLaunch LL;
    st = plan_solve(kk, a.I, Jp, a.ld, ctx->num_sms, 1 << 30, &LL);
    if (st) return set_error(ctx, st, "solver does not fit the shared memory (I=%lld J=%d)", (long long)a.I, J);
    SolveBufs B;
    st = solve_bufs(ctx, LL, Jp, &B);
    if (st) return st;
    SolveMode m;
    m.init = 1;
    m.F_out = F_out;
    cudaStream_t s = a.stream;
    cudaError_t e = enqueue_solve(a, kk, LL, B, ctx->spin_limit, s, nullptr, m);
    if (e == cudaSuccess) e = cudaMemcpyAsync(G_out, B.G + Jp, sizeof(double) * Jp, cudaMemcpyDeviceToDevice, s);
    LoopState* h = (LoopState*)host_staging(ctx, sizeof(LoopState), &st);
    if (st) return st;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, B.ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "first iteration");
    ctx->launches += 1;
    *status = h->status;
    return OT_OK;
}

// Finalize on given potentials (F' pairs, G log2 units): plan, f, g, loads and FP64 summary
// as the full solve gives them; iters / err / converged are reported as passed.
ot_status f32_finalize_on(ot_assoc_ctx* ctx, const SolveArgs& a, const float2* F_in, const double* G_in, int iters,
                          double err, int converged, SolveSummary* sum_host) {
    ot_status st = OT_OK;
    const int J = a.J;
    const int Jp = (int)round_up(J, 4);
    Kernels kk;
    if (!pick_kernels(J, &kk)) return set_error(ctx, OT_EUNSUPPORTED, "J=%d above 8192", J);
    LoopLaunch LL;
    st = plan_solve(kk, a.I, Jp, a.ld, ctx->num_sms, 1 << 30, &LL);
    if (st) return set_error(ctx, st, "solver does not fit the shared memory (I=%lld J=%d)", (long long)a.I, J);
    SolveBufs B;
    st = solve_bufs(ctx, LL, Jp, &B);
    if (st) return st;
    SolveSummary* hsum = (SolveSummary*)host_staging(ctx, sizeof(SolveSummary), &st);
    if (st) return st;
    SolveMode m;
    m.F_in = F_in;
    m.G_in = G_in;
    m.iters = iters;
    m.err = err;
    m.converged = converged;
    cudaStream_t s = a.stream;
    cudaError_t e = enqueue_solve(a, kk, LL, B, ctx->spin_limit, s, nullptr, m);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hsum, B.summ, sizeof(SolveSummary), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "finalize");
    ctx->launches += 4;
    *sum_host = *hsum;
    return OT_OK;
}

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
static constexpr size_t NOALLOC_BYTES = size_t(8) << 20;  // 8 MiB
static constexpr int64_t NOALLOC_MAX_I = 131072;
static constexpr int NOALLOC_MAX_J = 1024;
static constexpr int NOALLOC_MAX_CTAS = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Byte offsets inside g_noalloc_scratch (all multiples of 256).
static constexpr size_t NA_STATE = 0;                                     // DevScalars/LoopState/summary
static constexpr size_t NA_COLS = 4096;                                   // Jp double2
static constexpr size_t NA_G = NA_COLS + 16 * NOALLOC_MAX_J;              // gstate_words(Jp) doubles
static constexpr size_t NA_ERRPART = NA_G + (gstate_bytes(NOALLOC_MAX_J) + 255) / 256 * 256;  // 2 * CTAs doubles
static constexpr size_t NA_COLPART = NA_ERRPART + 16 * NOALLOC_MAX_CTAS;  // CTAs * Jp float2
static constexpr size_t NA_FPART = NA_COLPART + 8 * (size_t)NOALLOC_MAX_CTAS * NOALLOC_MAX_J;  // CTAs * Jp double2
static constexpr size_t NA_END = NA_FPART + 16 * (size_t)NOALLOC_MAX_CTAS * NOALLOC_MAX_J;
static_assert(NA_END <= NOALLOC_BYTES, "no-allocation scratch layout does not fit");
static_assert(NA_COLPART % 256 == 0 && NA_FPART % 256 == 0, "alignment");

// Device address of g_noalloc_scratch in the current device's context, looked up on every
// call.  The lookup allocates nothing and is cheap; caching it would keep a dead address once
// the context that loaded the module is destroyed and re-created (cudaDeviceReset).
static ot_status noalloc_base(unsigned char** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return OT_ECUDA;
    }
    *out = (unsigned char*)p;
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
    ot_status st = noalloc_base(&base);
    if (st) return st;
    Kernels kk;
    if (!pick_kernels(J, &kk)) return OT_EUNSUPPORTED;
    LoopLaunch LL;
    st = plan_solve(kk, I, Jp, a.ld, nsm, NOALLOC_MAX_CTAS, &LL);
    if (st) return st;
    SolveBufs B;
    char* state = (char*)(base + NA_STATE);
    B.sc = (DevScalars*)state;
    B.ls = (LoopState*)(state + 256);
    B.summ = (SolveSummary*)(state + 512);
    B.cols = (double2*)(base + NA_COLS);
    B.G = (double*)(base + NA_G);
    B.errpart = (double*)(base + NA_ERRPART);
    B.colpart = (void*)(base + NA_COLPART);
    B.fpart = (double2*)(base + NA_FPART);
    // The state words are cleared at the start of every call (the array keeps the last
    // call's data); enqueue_solve does that first.
    cudaError_t e = enqueue_solve(a, kk, LL, B, 1LL << 24, a.stream, nullptr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sum_host, B.summ, sizeof(SolveSummary), cudaMemcpyDeviceToHost, a.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(a.stream);
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
