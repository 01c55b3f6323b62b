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

#include "k_batch.cuh"

namespace ota {

// Instances planned for one group size, taken largest first from one queue.
struct BPhase {
    int gsize, first, count;
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
    const BGroup* groups;
    const int* cta_map;    // [nrounds][grid]: the group of each CTA in each round, or -1
    int nrounds;
    BCtl* ctl;
    unsigned* gbar;        // per group (all phases): barrier counter
    int* gcur;             // per group: the instance index the leader fetched
    long long spin;
};

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
    for (int rd = 0; rd < B.nrounds; ++rd) {
        const int gi = B.cta_map[rd * gridDim.x + blockIdx.x];
        if (gi >= 0) {
            const BGroup grp = B.groups[gi];
            const int ph = grp.phase;
            const BPhase PH = B.phases[ph];
            const int rank = blockIdx.x - grp.first_cta;
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
                const bool go = bt_run(B.inst[ii], B.res + ii, &B.ctl->abort, B.spin, grp, rank, PH.gsize, gbar,
                                       &s_gen, &s_nbar, &sh, dyn);
                if (!go) return;
            }
        }
        if (rd + 1 == B.nrounds) break;
        unsigned target = 0;
        if (threadIdx.x == 0) target = gridDim.x * ++s_ggen;
        if (!grid_barrier(&B.ctl->grid_bar, target, &B.ctl->abort, B.spin)) return;
    }
}

// ------------------------------------------------------------------------------------------
// Host side: size buckets, stage planning, schedule, autotuner, captured graph.
// ------------------------------------------------------------------------------------------
namespace {

std::vector<int> divisors(int n) {
    std::vector<int> d;
    for (int k = 1; k <= n; ++k)
        if (n % k == 0) d.push_back(k);
    return d;
}

// Schedule model (used before tuning and to pick the candidates the tuner times): one sweep
// of instance i on d CTAs takes the longer of streaming its cells at a CTA's share of HBM
// bandwidth and walking its rows at the consumer warps' row rate, plus the group barrier and
// the column update, plus the end of each of the CTA's row partitions (team partials merged
// through shared memory, fixed-point column totals): an instance keeps up to VMAX partitions
// whatever its group size, so small groups pay many partition ends a sweep.
constexpr double BW_CTA = 40e9;       // bytes/s one CTA streams with all SMs busy
constexpr double ROW_TIME = 0.5e-6;   // s per row per warp (latency of a row's chain)
constexpr double PART_END = 2e-6;     // s per partition end
double sweep_time(int64_t I, int J, int d) {
    const double stream = 4.0 * (double)I * J / (d * BW_CTA);
    const double rows = std::ceil((double)I / d) * ROW_TIME / BT_NCW;
    const double bar = d > 1 ? 3e-6 + 0.02e-6 * d : 0.5e-6;
    const int64_t rs = BT_NCW;  // rows per stage of one-warp teams at one row a team
    const int64_t V = std::max<int64_t>(1, std::min<int64_t>({(int64_t)VMAX, (I + rs - 1) / rs, I / 64}));
    const double ends = std::ceil((double)V / d) * PART_END;
    return std::max(stream, rows) + bar + ends;
}

// Group size of a batch: the divisor of the SM count that minimises the estimated makespan
// of a largest-first queue over nsm / d groups (every instance taken at the same number of
// sweeps), the larger group where estimates are within 2% (measured on the 256 ragged
// instances: groups of 2, 4, 8, 19, 38, 76 of 152 CTAs took 108, 108, 106, 92, 99, 115 ms,
// the autotuned plan 92 ms; the model misses costs that grow as groups shrink).  Results do
// not depend on it: every reduction runs over the instances' own row partitions.
int model_gsize(const std::vector<ot_assoc_instance>& v, int num_sms) {
    int best = 1;
    double best_t = 1e300;
    std::vector<int> ds = divisors(num_sms);
    std::reverse(ds.begin(), ds.end());
    for (int d : ds) {
        const int ng = num_sms / d;
        std::vector<double> t;
        t.reserve(v.size());
        for (const auto& a : v) t.push_back(sweep_time(a.I, a.J, d));
        std::sort(t.begin(), t.end(), std::greater<double>());
        std::vector<double> load(ng, 0.0);  // greedy list schedule, largest first
        for (double x : t) *std::min_element(load.begin(), load.end()) += x;
        const double m = *std::max_element(load.begin(), load.end());
        if (m < best_t * 0.98) {  // a smaller group only when clearly faster
            best_t = m;
            best = d;
        }
    }
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

// Stage target and group size of an instance: the tuned entry of its size bucket, else 24 KB
// and the batch's modelled group size.  The stage size fixes the instance's arithmetic (its
// rows per stage and row partitions); the group size only which CTAs do the work.
static void choose(const ot_assoc_ctx* ctx, int64_t I, int J, int g_batch, int* gsize, int* stage) {
    const TuneEntry& t = ctx->tune[batch_bucket(I, J)];
    *stage = t.stage > 0 ? t.stage : 24576;
    *gsize = t.gsize > 0 ? t.gsize : g_batch;
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
    const int g_batch = model_gsize(b->inst, nsm);
    for (int k = 0; k < n; ++k) {
        const ot_assoc_instance& a = b->inst[k];
        int g, st;
        choose(ctx, a.I, a.J, g_batch, &g, &st);
        if (forced_gsize > 0) g = forced_gsize;
        if (forced_stage > 0) st = forced_stage;
        std::memset(&d[k], 0, sizeof(BInst));
        fill_values(&d[k], a);
        d[k].vpt = vpt_for(a.J);
        size_t sm = 0;
        // grow the group until the CTA's share of the rows fits next to two stages
        bool ok = false;
        for (;;) {
            if (plan_stream(a.I, d[k].P.Jp, d[k].P.ld, g, st, &d[k].S, &sm, &d[k].P.V)) {
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
    std::vector<size_t> phase_jp, phase_v;
    std::vector<double> phase_work;  // estimated CTA-seconds per sweep
    for (int g : sizes) {
        BPhase ph;
        ph.gsize = g;
        ph.first = (int)b->h_order.size();
        std::vector<int> idx;
        int jpmax = 4, vmax = 1;
        double w = 0.0;
        for (int k = 0; k < n; ++k)
            if (gs[k] == g) {
                idx.push_back(k);
                jpmax = std::max(jpmax, d[k].P.Jp);
                vmax = std::max(vmax, d[k].P.V);
                w += sweep_time(b->inst[k].I, b->inst[k].J, g) * g;
            }
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
            return (double)b->inst[x].I * b->inst[x].J > (double)b->inst[y].I * b->inst[y].J;
        });
        ph.count = (int)idx.size();
        b->h_order.insert(b->h_order.end(), idx.begin(), idx.end());
        b->h_phases.push_back(ph);
        phase_jp.push_back((size_t)jpmax);
        phase_v.push_back((size_t)vmax);
        phase_work.push_back(w);
    }
    // rounds: phases that fit side by side (one group each) run at the same time; within a
    // round the remaining CTAs go, one group at a time, to the phase with the most work per
    // CTA (never more groups than the phase has instances)
    struct GroupPlan {
        int phase, first_cta;
    };
    std::vector<GroupPlan> gplan;
    std::vector<int> cta_map;
    int nrounds = 0;
    for (size_t p0 = 0; p0 < b->h_phases.size();) {
        size_t p1 = p0;
        int used = 0;
        while (p1 < b->h_phases.size() && used + b->h_phases[p1].gsize <= nsm) used += b->h_phases[p1++].gsize;
        std::vector<int> ngrp(p1 - p0, 1);
        for (;;) {
            int best = -1;
            double best_load = 0.0;
            for (size_t q = p0; q < p1; ++q) {
                const BPhase& ph = b->h_phases[q];
                if (used + ph.gsize > nsm || ngrp[q - p0] >= ph.count) continue;
                const double load = phase_work[q] / (ngrp[q - p0] * ph.gsize);
                if (load > best_load) {
                    best_load = load;
                    best = (int)q;
                }
            }
            if (best < 0) break;
            ++ngrp[best - p0];
            used += b->h_phases[best].gsize;
        }
        std::vector<int> map(nsm, -1);
        int cta = 0;
        for (size_t q = p0; q < p1; ++q)
            for (int r = 0; r < ngrp[q - p0]; ++r) {
                const int gi = (int)gplan.size();
                gplan.push_back({(int)q, cta});
                for (int c = 0; c < b->h_phases[q].gsize; ++c) map[cta + c] = gi;
                cta += b->h_phases[q].gsize;
            }
        cta_map.insert(cta_map.end(), map.begin(), map.end());
        ++nrounds;
        p0 = p1;
    }
    const int ngroups_total = (int)gplan.size();
    // device layout: [inst][res][ctl][gbar][gcur][order][phases][cta_map][groups][group scratch...]
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
    const size_t o_map = off;
    off = al(off + sizeof(int) * cta_map.size());
    const size_t o_groups = off;
    off = al(off + sizeof(BGroup) * ngroups_total);
    std::vector<size_t> g_off(ngroups_total);
    for (int gi = 0; gi < ngroups_total; ++gi) {
        const size_t Jp = phase_jp[gplan[gi].phase], nb = (size_t)b->h_phases[gplan[gi].phase].gsize;
        const size_t nv = phase_v[gplan[gi].phase];
        const size_t bytes = 1024 + al(gstate_bytes((int)Jp)) + al(nv * 2 * Jp * 4) + al(nv * 16) + al(nv * Jp * 16) +
                             al(nb * BT_NW * 16 + nv * 8);
        g_off[gi] = off;
        off = al(off + bytes);
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
    for (int gi = 0; gi < ngroups_total; ++gi) {
        const size_t Jp = phase_jp[gplan[gi].phase], nv = phase_v[gplan[gi].phase];
        char* g = base + g_off[gi];
        BGroup& G = b->h_groups[gi];
        G.sc = (DevScalars*)g;
        G.ls = (LoopState*)(g + 512);
        size_t o = 1024;
        G.G = (double*)(g + o);
        o += al(gstate_bytes((int)Jp));
        G.colpart = (float*)(g + o);
        o += al(nv * 2 * Jp * 4);
        G.errpart = (double*)(g + o);
        o += al(nv * 16);
        G.fpart = (double2*)(g + o);
        o += al(nv * Jp * 16);
        G.fred = (double*)(g + o);
        G.phase = gplan[gi].phase;
        G.first_cta = gplan[gi].first_cta;
    }
    std::memcpy(b->h_inst, d.data(), sizeof(BInst) * n);
    e = cudaMemcpy(base + o_order, b->h_order.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + o_phases, b->h_phases.data(), sizeof(BPhase) * b->h_phases.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + o_map, cta_map.data(), sizeof(int) * cta_map.size(), cudaMemcpyHostToDevice);
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
    BP.groups = (const BGroup*)(base + o_groups);
    BP.cta_map = (const int*)(base + o_map);
    BP.nrounds = nrounds;
    BP.ctl = b->d_ctl;
    BP.gbar = b->d_gbar;
    BP.gcur = b->d_gcur;
    BP.spin = ctx->spin_limit;
    b->smem = smem;
    b->grid = nsm;
    if (allow_max_dynamic_smem((const void*)sk_batch, smem) !=
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
// Autotuner.  Times the batch itself (a fixed number of iterations, tol = 0, outputs sent to
// scratch so the callers' buffers are untouched).  Size bucket by bucket (largest total
// work first), the bucket's instances try the group sizes around the current choice and
// the stage sizes, the others keeping theirs; the fastest pair becomes the bucket's entry.
// ------------------------------------------------------------------------------------------
static ot_status time_batch(ot_assoc_ctx* ctx, const std::vector<ot_assoc_instance>& tb,
                            const std::vector<TuneEntry>& trial, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                            float* ms_out) {
    TuneEntry saved[TUNE_BUCKETS];
    std::copy(ctx->tune, ctx->tune + TUNE_BUCKETS, saved);
    std::copy(trial.begin(), trial.end(), ctx->tune);
    ot_assoc_batch* b = nullptr;
    ot_status st = batch_create(ctx, tb.data(), (int)tb.size(), OT_BATCH_NO_GRAPH, &b);
    std::copy(saved, saved + TUNE_BUCKETS, ctx->tune);
    if (st) return st;
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
            st = set_error(ctx, OT_ECUDA, "autotune timing");
        }
    }
    batch_destroy(b);
    *ms_out = ms;
    return st;
}

ot_status batch_autotune(ot_assoc_ctx* ctx, const ot_assoc_instance* inst, int n, int iters, cudaStream_t s) {
    if (iters < 3) iters = 3;
    std::vector<ot_assoc_instance> tb(inst, inst + n);
    int64_t Isum = 0, Jsum = 0;
    for (int k = 0; k < n; ++k) {
        ot_status st = batch_check(ctx, inst[k], k);
        if (st) return st;
        Isum += round_up(inst[k].I, 32);
        Jsum += round_up(inst[k].J, 32);
    }
    ot_status st = OT_OK;
    double* outbuf = (double*)scratch(ctx, SLOT_TUNE, sizeof(double) * (size_t)(Isum + Jsum), &st);
    if (st) return st;
    {
        int64_t o = 0;
        for (int k = 0; k < n; ++k) {
            tb[k].f = outbuf + o;
            o += round_up(inst[k].I, 32);
            tb[k].g = outbuf + o;
            o += round_up(inst[k].J, 32);
            tb[k].rrh_load = nullptr;
            tb[k].pi = nullptr;
            tb[k].warm_start = 0;
            tb[k].tol = 0.0;
            tb[k].max_iter = iters;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return set_error(ctx, OT_ECUDA, "autotune events");
    }
    // current choice of every bucket present (tuned entry, else the model at the bucket's
    // largest instance and 24 KB stages), and the buckets' total work
    std::vector<TuneEntry> cur(ctx->tune, ctx->tune + TUNE_BUCKETS);
    std::vector<double> work(TUNE_BUCKETS, 0.0);
    const int g_batch = model_gsize(tb, ctx->num_sms);
    for (const auto& a : tb) {
        const int bk = batch_bucket(a.I, a.J);
        work[bk] += (double)a.I * a.J;
        if (cur[bk].gsize <= 0) cur[bk].gsize = g_batch;
        if (cur[bk].stage <= 0) cur[bk].stage = 24576;
    }
    std::vector<int> order;
    for (int bk = 0; bk < TUNE_BUCKETS; ++bk)
        if (work[bk] > 0) order.push_back(bk);
    std::sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    double cells_iter = 0.0;
    for (const auto& a : tb) cells_iter += (double)a.I * a.J * (iters + 1);
    const std::vector<int> divs = divisors(ctx->num_sms);
    const int stages[3] = {12288, 24576, 49152};
    for (int bk : order) {
        if (st) break;
        const int pos = (int)(std::find(divs.begin(), divs.end(), cur[bk].gsize) - divs.begin());
        TuneEntry best = cur[bk];
        float best_ms = 1e30f;
        for (int q = std::max(0, pos - 2); q <= std::min((int)divs.size() - 1, pos + 2) && !st; ++q)
            for (int stg : stages) {
                std::vector<TuneEntry> trial = cur;
                trial[bk].gsize = divs[q];
                trial[bk].stage = stg;
                float ms = 0.f;
                st = time_batch(ctx, tb, trial, s, e0, e1, &ms);
                if (st == OT_EUNSUPPORTED) {
                    ctx->err.clear();
                    st = OT_OK;
                    continue;
                }
                if (st) break;
                if (ms > 0.f && ms < best_ms) {
                    best_ms = ms;
                    best = trial[bk];
                }
            }
        if (!st && best_ms < 1e30f) {
            best.rate = cells_iter / (best_ms * 1e-3);
            cur[bk] = best;
            ctx->tune[bk] = best;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace ota
