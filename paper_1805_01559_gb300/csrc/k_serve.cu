// Serving: association solves of many cells' time instances, continuously batched onto one
// persistent launch (Algorithm 1 of the paper, Sec. III-B, per request).
//
// Every cell keeps its cost matrix C, traffic p, RRH marginal q and potentials f, g
// resident on the device; a request is one new time instance of a cell: new gains (given
// by the caller, or the cell's devices moved by dt on the device), from which the cost is
// rebuilt in place (rates of Sec. II-A, C = 1 / (mu R)), and a solve warm-started from the
// cell's previous g.  Requests of one cell run one after the other (each starts from its
// predecessor's result); requests of different cells run side by side.
//
// The server kernel is persistent: its CTAs form fixed groups, and each group takes the next
// published request from a queue in host-mapped memory (the host appends while the kernel
// runs), solves and finalizes it (the batched solver's group code), writes the result to
// host-mapped memory and takes the next.  A group that finds no work for `idle` polls
// leaves; when all have left the launch ends and the host starts a new one when work comes.
// A request's result depends only on its cell's data (row partitions fix every reduction
// order), so it is the same alone and in any mix.  Every wait is bounded.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <vector>

#include "k_batch.cuh"

namespace ota {

static constexpr int SV_CAP = 1024;  // descriptors in the queue ring

// Host-mapped queue (pinned host memory the kernel reads and writes).
struct SvQueue {
    unsigned tail;   // descriptors published (host writes, release)
    unsigned stop;   // host asks idle groups to leave at once
    unsigned pad[30];
    BInst desc[SV_CAP];
    BRes res[SV_CAP];
    unsigned done[SV_CAP];  // sequence number + 1 of the request whose result is in res[]
};

struct SvCtl {  // device memory, zeroed once
    unsigned head;  // descriptors claimed
    int abort;
};

struct ServeParams {
    SvQueue* q;          // device view of the mapped queue
    SvCtl* ctl;
    BRes* dres;          // [SV_CAP] device result slots (status words while solving)
    const BGroup* groups;
    unsigned* gbar;      // [ngroups]
    int* gcur;           // [ngroups]
    int gsize;
    long long idle_polls;
    long long spin;
};

__device__ __forceinline__ unsigned ld_acquire_sys_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void __launch_bounds__(BT_NT, 1) sk_serve(ServeParams S) {
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ SkShared sh;
    __shared__ __align__(16) BInst s_inst;
    __shared__ unsigned s_gen;
    __shared__ int s_idx, s_nbar;
    const int gi = blockIdx.x / S.gsize, rank = blockIdx.x % S.gsize;
    const BGroup grp = S.groups[gi];
    unsigned* gbar = S.gbar + gi;
    if (threadIdx.x == 0) {
        s_gen = 0;
        s_nbar = 0;
    }
    __syncthreads();
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            // claim the next published request, or give up after the idle limit
            int idx = -1;
            long long n = 0;
            for (;;) {
                if (ld_acquire_sys_u32(&S.q->stop)) break;
                const unsigned t = ld_acquire_sys_u32(&S.q->tail);
                const unsigned h = *(volatile unsigned*)&S.ctl->head;
                if (h < t) {
                    if (atomicCAS(&S.ctl->head, h, h + 1) == h) {
                        idx = (int)h;
                        break;
                    }
                    continue;
                }
                if (++n > S.idle_polls) break;
                __nanosleep(256);
            }
            if (idx >= 0) {
                BRes* r = S.dres + (idx % SV_CAP);
                r->status = DEV_OK;
                r->done = 0;
            }
            S.gcur[gi] = idx;
        }
        if (!group_sync(gbar, S.gsize, &s_gen, &S.ctl->abort, S.spin)) return;
        if (threadIdx.x == 0) s_idx = ld_volatile_i32(S.gcur + gi);
        __syncthreads();
        const int idx = s_idx;
        if (idx < 0) return;
        const int slot = idx % SV_CAP;
        {  // the descriptor into shared memory (read once from host memory)
            const unsigned* src = reinterpret_cast<const unsigned*>(&S.q->desc[slot]);
            unsigned* dst = reinterpret_cast<unsigned*>(&s_inst);
            for (int k = threadIdx.x; k < (int)(sizeof(BInst) / 4); k += blockDim.x) dst[k] = src[k];
        }
        __syncthreads();
        BRes* out = S.dres + slot;
        if (!bt_run(s_inst, out, &S.ctl->abort, S.spin, grp, rank, S.gsize, gbar, &s_gen, &s_nbar, &sh, dyn))
            return;
        if (rank == 0 && threadIdx.x == 0) {
            S.q->res[slot] = *out;
            __threadfence_system();
            st_release_sys_u32(&S.q->done[slot], (unsigned)idx + 1u);
        }
    }
}

// Cost of a drifting cell's new time instance: devices move by v dt (reflecting at the
// square's walls), gains from the path-loss model with the cell's fixed shadowing, rates
// with every other RRH interfering (Sec. II-A), C = 1 / (mu R).  One warp per device.
__global__ void __launch_bounds__(256) serve_channel(double* dev_xy, double* dev_v, const float* __restrict__ rrh_xy,
                                                     const float* __restrict__ shadow_db, int64_t I, int J,
                                                     double side, double dt, const float* __restrict__ P,
                                                     float N0, float W, float mu, float pl0_db, float pl_exp,
                                                     float d_min, float* C, int64_t ldc) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float inv_ln2 = 1.4426950408889634f;
    for (int64_t i = w0; i < I; i += nw) {
        double xy[2];
        if (lane == 0) {
            for (int ax = 0; ax < 2; ++ax) {
                const double x0 = dev_xy[2 * i + ax], v = dev_v[2 * i + ax];
                const double x1 = x0 + v * dt;
                double pm = fmod(x1, 2.0 * side);
                if (pm < 0.0) pm += 2.0 * side;
                if (pm > side) pm = 2.0 * side - pm;
                const long long k = (long long)floor(x1 / side);
                if (k & 1LL) dev_v[2 * i + ax] = -v;
                dev_xy[2 * i + ax] = pm;
                xy[ax] = pm;
            }
        }
        const float x = (float)__shfl_sync(0xffffffffu, xy[0], 0), y = (float)__shfl_sync(0xffffffffu, xy[1], 0);
        const float* sh = shadow_db + i * (int64_t)J;
        // received powers P_j G_ij: the row total first (pairs of FP32), then the rates
        float tot_hi = 0.f, tot_lo = 0.f;
        for (int j = lane; j < J; j += 32) {
            const float dx = x - rrh_xy[2 * j], dy = y - rrh_xy[2 * j + 1];
            const float d = fmaxf(sqrtf(dx * dx + dy * dy), d_min);
            const float pl = pl0_db + 10.f * pl_exp * log10f(d) - sh[j];
            const float pg = P[j] * exp10f(-0.1f * pl);
            float s, e;
            two_sum(tot_hi, pg, s, e);
            tot_hi = s;
            tot_lo += e;
        }
        float tot = tot_hi + tot_lo;
        tot = warp_sum(tot);
        float* row = C + i * ldc;
        for (int j = lane; j < J; j += 32) {
            const float dx = x - rrh_xy[2 * j], dy = y - rrh_xy[2 * j + 1];
            const float d = fmaxf(sqrtf(dx * dx + dy * dy), d_min);
            const float pl = pl0_db + 10.f * pl_exp * log10f(d) - sh[j];
            const float pg = P[j] * exp10f(-0.1f * pl);
            const float sinr = pg / ((tot - pg) + N0);
            const float R = W * log1pf(sinr) * inv_ln2;
            row[j] = 1.0f / (mu * R);
        }
    }
}

}  // namespace ota

// ------------------------------------------------------------------------------------------
// The server object (host).
// ------------------------------------------------------------------------------------------
namespace {

using Clock = std::chrono::steady_clock;

double now_us() {
    return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

struct Cell {
    int64_t I = 0;
    int J = 0;
    int64_t ldc = 0;
    double eps = 0, tol = 1e-6, mu = 0, N0 = 0, W = 0, side = 0;
    int max_iter = 2000;
    int warm = 1;
    bool drift = false;
    // device
    float* C = nullptr;
    float* p = nullptr;
    float* q = nullptr;
    float* P = nullptr;
    double* f = nullptr;
    double* g = nullptr;
    double* rho = nullptr;
    double* dev_xy = nullptr;
    double* dev_v = nullptr;
    float* rrh_xy = nullptr;
    float* shadow = nullptr;
    float* R = nullptr;  // rates scratch when the caller gives gains
    unsigned long long* bad = nullptr;  // invalid rates of the last cost rebuild
    std::vector<void*> allocs;
    size_t bytes = 0;
    // scheduling
    bool busy = false;
    int solved = 0;
};

struct Request {
    uint64_t ticket;
    int cell;
    const float* G;
    int64_t ld_g;
    double dt;
    double t_submit, t_start;
    unsigned seq;
    cudaEvent_t prep_done = nullptr;
};

}  // namespace

struct ot_assoc_server {
    ot_assoc_ctx* ctx = nullptr;
    ot_assoc_server_config cfg{};
    int gsize = 8, ngroups = 19;
    ota::SvQueue* q_host = nullptr;
    ota::SvQueue* q_dev = nullptr;
    void* dmem = nullptr;
    size_t dbytes = 0;
    ota::ServeParams params{};
    cudaStream_t prep_stream = nullptr, run_stream = nullptr;
    cudaEvent_t run_done = nullptr;
    bool running = false;
    size_t smem = 0;
    std::vector<Cell> cells;
    std::deque<Request> waiting;     // submitted, cell busy or not yet started
    std::vector<Request> prepping;   // cost rebuild enqueued
    std::vector<Request> inflight;   // published to the kernel
    std::vector<cudaEvent_t> free_events;
    uint64_t next_ticket = 1;
    unsigned published = 0;
    size_t resident = 0;
    std::vector<ot_assoc_server_result> ready;
    uint64_t launches = 0;
};

namespace ota {

static ot_status sv_alloc(ot_assoc_server* s, Cell& c, size_t bytes, void** out) {
    ot_assoc_ctx* ctx = s->ctx;
    if (s->cfg.hbm_budget && s->resident + bytes > s->cfg.hbm_budget)
        return set_error(ctx, OT_EBUSY, "cell needs %zu more bytes: over the server's HBM budget (%zu of %zu held)",
                         bytes, s->resident, (size_t)s->cfg.hbm_budget);
    cudaError_t e = cudaMalloc(out, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) return cuda_error(ctx, e, "cudaMalloc (cell)");
    c.allocs.push_back(*out);
    c.bytes += bytes;
    s->resident += bytes;
    return OT_OK;
}

static void sv_free_cell(ot_assoc_server* s, Cell& c) {
    for (void* p : c.allocs) cudaFree(p);
    c.allocs.clear();
    s->resident -= c.bytes;
    c.bytes = 0;
}

static ot_status sv_launch(ot_assoc_server* s) {
    ot_assoc_ctx* ctx = s->ctx;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(s->gsize * s->ngroups);
    cfg.blockDim = dim3(BT_NT);
    cfg.dynamicSmemBytes = s->smem;
    cfg.stream = s->run_stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // group barrier counters restart with every launch
    cudaError_t e = cudaMemsetAsync(s->params.gbar, 0, sizeof(unsigned) * s->ngroups, s->run_stream);
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, sk_serve, s->params);
    if (e == cudaSuccess) e = cudaEventRecord(s->run_done, s->run_stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "server launch");
    s->running = true;
    ++s->launches;
    ctx->launches += 1;
    return OT_OK;
}

// Enqueue the cost rebuild of a request's time instance on the prep stream.
static ot_status sv_prep(ot_assoc_server* s, Request& r) {
    ot_assoc_ctx* ctx = s->ctx;
    Cell& c = s->cells[r.cell];
    ot_status st = OT_OK;
    cudaError_t e0 = cudaMemsetAsync(c.bad, 0, sizeof(unsigned long long), s->prep_stream);
    if (e0 != cudaSuccess) return cuda_error(ctx, e0, "memset");
    if (r.G) {
        st = launch_rates(ctx, r.G, r.ld_g, c.P, c.I, c.J, c.N0, c.W, c.R, c.ldc, s->prep_stream);
        if (st) return st;
        st = launch_cost(ctx, c.R, c.ldc, c.I, c.J, c.mu, c.C, c.ldc, true, c.bad, s->prep_stream);
        if (st) return st;
    } else {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((c.I + 7) / 8, 8LL * ctx->num_sms));
        serve_channel<<<grid, 256, 0, s->prep_stream>>>(c.dev_xy, c.dev_v, c.rrh_xy, c.shadow, c.I, c.J, c.side, r.dt,
                                                       c.P, (float)c.N0, (float)c.W, (float)c.mu, 30.0f, 3.5f, 10.0f,
                                                       c.C, c.ldc);
        ctx->launches += 1;
    }
    if (s->free_events.empty()) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_error(ctx, e, "event");
        s->free_events.push_back(ev);
    }
    r.prep_done = s->free_events.back();
    s->free_events.pop_back();
    cudaError_t e = cudaEventRecord(r.prep_done, s->prep_stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "event record");
    return OT_OK;
}

// Publish a prepared request to the kernel's queue.
static ot_status sv_publish(ot_assoc_server* s, Request& r) {
    Cell& c = s->cells[r.cell];
    const unsigned seq = s->published;
    const int slot = (int)(seq % SV_CAP);
    BInst d;
    std::memset(&d, 0, sizeof(d));
    ot_assoc_instance a = {};
    a.C = c.C;
    a.ld = c.ldc;
    a.I = c.I;
    a.J = c.J;
    a.warm_start = (c.warm && c.solved > 0) ? 1 : 0;
    a.p = c.p;
    a.q = c.q;
    a.eps = c.eps;
    a.tol = c.tol;
    a.max_iter = c.max_iter;
    a.f = c.f;
    a.g = c.g;
    a.rrh_load = c.rho;
    fill_values(&d, a);
    d.P.input_bad = c.bad;  // invalid rates in the cost rebuild fail the request
    d.vpt = vpt_for(c.J);
    size_t sm = 0;
    if (!plan_stream(c.I, d.P.Jp, c.ldc, s->gsize, 24576, &d.S, &sm, &d.P.V))
        return set_error(s->ctx, OT_EUNSUPPORTED, "cell does not fit the server's groups");
    s->q_host->desc[slot] = d;
    s->q_host->done[slot] = 0;
    std::atomic_thread_fence(std::memory_order_release);
    __atomic_store_n(&s->q_host->tail, seq + 1u, __ATOMIC_RELEASE);
    r.seq = seq;
    r.t_start = now_us();
    s->published = seq + 1;
    return OT_OK;
}

static ot_status sv_progress(ot_assoc_server* s) {
    ot_assoc_ctx* ctx = s->ctx;
    // 1. start the cost rebuild of waiting requests whose cell is idle (in submit order)
    for (auto it = s->waiting.begin(); it != s->waiting.end();) {
        Cell& c = s->cells[it->cell];
        if (c.busy || (int)(s->prepping.size() + s->inflight.size()) >= SV_CAP / 2) {
            ++it;
            continue;
        }
        c.busy = true;
        Request r = *it;
        it = s->waiting.erase(it);
        ot_status st = sv_prep(s, r);
        if (st) return st;
        s->prepping.push_back(r);
    }
    // 2. publish the requests whose cost is ready
    for (size_t k = 0; k < s->prepping.size();) {
        cudaError_t e = cudaEventQuery(s->prepping[k].prep_done);
        if (e == cudaErrorNotReady) {
            ++k;
            continue;
        }
        if (e != cudaSuccess) return cuda_error(ctx, e, "cost rebuild");
        Request r = s->prepping[k];
        s->free_events.push_back(r.prep_done);
        r.prep_done = nullptr;
        s->prepping.erase(s->prepping.begin() + k);
        ot_status st = sv_publish(s, r);
        if (st) return st;
        s->inflight.push_back(r);
    }
    // 3. keep a launch running while published work is not done
    if (s->running) {
        cudaError_t e = cudaEventQuery(s->run_done);
        if (e == cudaSuccess) {
            s->running = false;
        } else if (e != cudaErrorNotReady) {
            return cuda_error(ctx, e, "server kernel");
        }
    }
    // 4. collect finished requests
    for (size_t k = 0; k < s->inflight.size();) {
        Request& r = s->inflight[k];
        const int slot = (int)(r.seq % SV_CAP);
        const unsigned d = __atomic_load_n(&s->q_host->done[slot], __ATOMIC_ACQUIRE);
        if (d != r.seq + 1u) {
            ++k;
            continue;
        }
        const BRes res = s->q_host->res[slot];
        ot_assoc_server_result o = {};
        o.ticket = r.ticket;
        o.cell = r.cell;
        o.iters = res.iters;
        o.transport_cost = res.cost;
        o.marg_err_row = res.err_row;
        o.marg_err_col = res.err_col;
        o.t_submit_us = r.t_submit;
        o.t_start_us = r.t_start;
        o.t_done_us = now_us();
        if (res.status == DEV_EINVAL || res.status == DEV_ENUMERIC) o.status = OT_EINVAL;
        else if (res.status == DEV_ETIMEOUT) o.status = OT_ETIMEOUT;
        else if (res.status != DEV_OK) o.status = OT_ECUDA;
        else o.status = res.converged ? OT_OK : OT_NOT_CONVERGED;
        Cell& c = s->cells[r.cell];
        c.busy = false;
        if (o.status == OT_OK || o.status == OT_NOT_CONVERGED) ++c.solved;
        s->ready.push_back(o);
        s->inflight.erase(s->inflight.begin() + k);
    }
    bool unclaimed = !s->inflight.empty();
    if (!s->running && unclaimed) {
        // an abort in the last launch leaves requests claimed but never done: report them
        int ab = 0;
        cudaError_t e = cudaMemcpy(&ab, &((SvCtl*)s->params.ctl)->abort, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_error(ctx, e, "server state");
        if (ab) return set_error(ctx, OT_ETIMEOUT, "a device-side wait of the server kernel exceeded its spin limit");
        ot_status st = sv_launch(s);
        if (st) return st;
    }
    return OT_OK;
}

}  // namespace ota

using namespace ota;

extern "C" {

ot_status ot_assoc_server_create(ot_assoc_ctx* ctx, const ot_assoc_server_config* cfg, ot_assoc_server** out) {
    if (!ctx) return OT_EINVAL;
    if (!out) return set_error(ctx, OT_EINVAL, "null output pointer");
    *out = nullptr;
    DeviceGuardLite guard(ctx->device);
    ot_assoc_server* s = new ot_assoc_server;
    s->ctx = ctx;
    if (cfg) s->cfg = *cfg;
    const int nsm = ctx->num_sms;
    s->gsize = s->cfg.group_ctas > 0 ? s->cfg.group_ctas : 8;
    if (nsm % s->gsize != 0) {
        delete s;
        return set_error(ctx, OT_EINVAL, "group_ctas must divide the SM count (%d)", nsm);
    }
    s->ngroups = nsm / s->gsize;
    const int maxJ = s->cfg.max_J > 0 ? s->cfg.max_J : 1024;
    if (maxJ > MAX_J_BATCH) {
        delete s;
        return set_error(ctx, OT_EUNSUPPORTED, "max_J above 1024");
    }
    const double idle = s->cfg.idle_us > 0 ? s->cfg.idle_us : 200.0;
    // device memory: control, result slots, group state
    auto al = [](size_t x) { return (size_t)round_up((int64_t)x, 256); };
    const size_t Jp = (size_t)round_up(maxJ, 4), nv = VMAX;
    const size_t gbytes = 1024 + al(3 * Jp * 8) + al(nv * 2 * Jp * 4) + al(nv * 16) + al(nv * Jp * 16) +
                          al((size_t)s->gsize * BT_NW * 16 + nv * 8);
    const size_t o_ctl = 0, o_res = al(sizeof(SvCtl)), o_gbar = o_res + al(sizeof(BRes) * SV_CAP);
    const size_t o_gcur = o_gbar + al(sizeof(unsigned) * s->ngroups), o_groups = o_gcur + al(sizeof(int) * s->ngroups);
    const size_t o_scr = o_groups + al(sizeof(BGroup) * s->ngroups), total = o_scr + gbytes * s->ngroups;
    cudaError_t e = cudaMalloc(&s->dmem, total);
    if (e == cudaSuccess) e = cudaMemset(s->dmem, 0, o_scr);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->q_host, sizeof(SvQueue), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&s->q_dev, s->q_host, 0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->prep_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->run_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->run_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        ot_status st = cuda_error(ctx, e, "server setup");
        ot_assoc_server_destroy(s);
        return st;
    }
    std::memset(s->q_host, 0, sizeof(SvQueue));
    s->dbytes = total;
    char* base = (char*)s->dmem;
    std::vector<BGroup> groups(s->ngroups);
    for (int g = 0; g < s->ngroups; ++g) {
        char* p = base + o_scr + gbytes * g;
        BGroup& G = groups[g];
        G.sc = (DevScalars*)p;
        G.ls = (LoopState*)(p + 512);
        size_t o = 1024;
        G.G = (double*)(p + o);
        o += al(3 * Jp * 8);
        G.colpart = (float*)(p + o);
        o += al(nv * 2 * Jp * 4);
        G.errpart = (double*)(p + o);
        o += al(nv * 16);
        G.fpart = (double2*)(p + o);
        o += al(nv * Jp * 16);
        G.fred = (double*)(p + o);
        G.phase = 0;
        G.first_cta = g * s->gsize;
    }
    e = cudaMemcpy(base + o_groups, groups.data(), sizeof(BGroup) * s->ngroups, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        ot_status st = cuda_error(ctx, e, "server setup");
        ot_assoc_server_destroy(s);
        return st;
    }
    ServeParams& P = s->params;
    P.q = s->q_dev;
    P.ctl = (SvCtl*)(base + o_ctl);
    P.dres = (BRes*)(base + o_res);
    P.groups = (const BGroup*)(base + o_groups);
    P.gbar = (unsigned*)(base + o_gbar);
    P.gcur = (int*)(base + o_gcur);
    P.gsize = s->gsize;
    P.idle_polls = (long long)(idle / 0.3);  // a poll sleeps about 0.3 us
    P.spin = ctx->spin_limit;
    s->smem = SMEM_BUDGET;
    if (cudaFuncSetAttribute((const void*)sk_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem) !=
        cudaSuccess) {
        cudaGetLastError();
        ot_assoc_server_destroy(s);
        return set_error(ctx, OT_ECUDA, "server kernel: shared memory");
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)sk_serve, BT_NT, s->smem) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        ot_assoc_server_destroy(s);
        return set_error(ctx, OT_EUNSUPPORTED, "server kernel cannot be resident");
    }
    *out = s;
    return OT_OK;
}

void ot_assoc_server_destroy(ot_assoc_server* s) {
    if (!s) return;
    DeviceGuardLite guard(s->ctx->device);
    if (s->q_host) __atomic_store_n(&s->q_host->stop, 1u, __ATOMIC_RELEASE);
    if (s->run_stream) cudaStreamSynchronize(s->run_stream);
    if (s->prep_stream) cudaStreamSynchronize(s->prep_stream);
    for (auto& c : s->cells) sv_free_cell(s, c);
    for (auto& r : s->prepping)
        if (r.prep_done) cudaEventDestroy(r.prep_done);
    for (cudaEvent_t ev : s->free_events) cudaEventDestroy(ev);
    if (s->run_done) cudaEventDestroy(s->run_done);
    if (s->run_stream) cudaStreamDestroy(s->run_stream);
    if (s->prep_stream) cudaStreamDestroy(s->prep_stream);
    if (s->q_host) cudaFreeHost(s->q_host);
    if (s->dmem) cudaFree(s->dmem);
    delete s;
}

ot_status ot_assoc_server_add_cell(ot_assoc_server* s, const ot_assoc_cell_desc* d, int32_t* cell_id) {
    if (!s) return OT_EINVAL;
    ot_assoc_ctx* ctx = s->ctx;
    if (!d || !cell_id) return set_error(ctx, OT_EINVAL, "null pointer");
    if (d->I <= 0 || d->J <= 0) return set_error(ctx, OT_EINVAL, "I and J must be positive");
    const int maxJ = s->cfg.max_J > 0 ? s->cfg.max_J : 1024;
    if (d->J > maxJ) return set_error(ctx, OT_EUNSUPPORTED, "J=%d above the server's max_J=%d", d->J, maxJ);
    if (!(d->eps > 0.0) || !(d->mu > 0.0) || !(d->W_hz > 0.0) || !(d->N0 > 0.0))
        return set_error(ctx, OT_EINVAL, "eps, mu, W and N0 must be > 0");
    if (!d->P || !d->p || !d->q) return set_error(ctx, OT_EINVAL, "P, p and q are required");
    const bool drift = d->dev_xy != nullptr;
    if (drift && (!d->dev_v || !d->rrh_xy || !d->shadow_db || !(d->side_m > 0.0)))
        return set_error(ctx, OT_EINVAL, "a drifting cell needs positions, velocities, RRH positions, shadowing, side");
    DeviceGuardLite guard(ctx->device);
    Cell c;
    c.I = d->I;
    c.J = d->J;
    c.ldc = round_up(d->J, 4);
    c.eps = d->eps;
    c.tol = d->tol >= 0 ? d->tol : 1e-6;
    c.max_iter = d->max_iter > 0 ? d->max_iter : 2000;
    c.warm = d->warm_start;
    c.mu = d->mu;
    c.N0 = d->N0;
    c.W = d->W_hz;
    c.side = d->side_m;
    c.drift = drift;
    // the cell must fit the server's groups
    {
        StreamCfg S;
        size_t sm = 0;
        int V = 0;
        if (!plan_stream(c.I, (int)round_up(c.J, 4), c.ldc, s->gsize, 24576, &S, &sm, &V))
            return set_error(ctx, OT_EUNSUPPORTED, "I=%lld rows do not fit groups of %d CTAs", (long long)c.I, s->gsize);
    }
    const size_t I = (size_t)c.I, J = (size_t)c.J, ldc = (size_t)c.ldc;
    ot_status st = OT_OK;
    void* p;
#define SV_ALLOC(field, type, n)                               \
    do {                                                       \
        st = sv_alloc(s, c, sizeof(type) * (n), &p);           \
        if (st) {                                              \
            sv_free_cell(s, c);                                \
            return st;                                         \
        }                                                      \
        c.field = (type*)p;                                    \
    } while (0)
    SV_ALLOC(C, float, I * ldc);
    SV_ALLOC(p, float, I);
    SV_ALLOC(q, float, J);
    SV_ALLOC(P, float, J);
    SV_ALLOC(f, double, I);
    SV_ALLOC(g, double, ldc);
    SV_ALLOC(rho, double, ldc);
    SV_ALLOC(bad, unsigned long long, 1);
    if (drift) {
        SV_ALLOC(dev_xy, double, 2 * I);
        SV_ALLOC(dev_v, double, 2 * I);
        SV_ALLOC(rrh_xy, float, 2 * J);
        SV_ALLOC(shadow, float, I * J);
    } else {
        SV_ALLOC(R, float, I * ldc);
    }
#undef SV_ALLOC
    cudaError_t e = cudaMemcpy(c.p, d->p, sizeof(float) * I, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.q, d->q, sizeof(float) * J, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.P, d->P, sizeof(float) * J, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c.g, 0, sizeof(double) * ldc);
    if (e == cudaSuccess) e = cudaMemset(c.bad, 0, sizeof(unsigned long long));
    if (drift) {
        if (e == cudaSuccess) e = cudaMemcpy(c.dev_xy, d->dev_xy, sizeof(double) * 2 * I, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c.dev_v, d->dev_v, sizeof(double) * 2 * I, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c.rrh_xy, d->rrh_xy, sizeof(float) * 2 * J, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c.shadow, d->shadow_db, sizeof(float) * I * J, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        sv_free_cell(s, c);
        return cuda_error(ctx, e, "cell upload");
    }
    *cell_id = (int32_t)s->cells.size();
    s->cells.push_back(c);
    return OT_OK;
}

ot_status ot_assoc_server_submit(ot_assoc_server* s, int32_t cell, const float* G, int64_t ld_g, double dt,
                                 uint64_t* ticket) {
    if (!s) return OT_EINVAL;
    ot_assoc_ctx* ctx = s->ctx;
    if (cell < 0 || cell >= (int32_t)s->cells.size()) return set_error(ctx, OT_EINVAL, "unknown cell %d", cell);
    const Cell& c = s->cells[cell];
    if (G) {
        if (c.drift) return set_error(ctx, OT_EINVAL, "cell %d moves its own devices: submit with G = NULL", cell);
        if (ld_g == 0) ld_g = c.J;
        if (ld_g < c.J) return set_error(ctx, OT_EINVAL, "ld_g < J");
    } else if (!c.drift) {
        return set_error(ctx, OT_EINVAL, "cell %d needs gains with every request", cell);
    }
    Request r;
    r.ticket = s->next_ticket++;
    r.cell = cell;
    r.G = G;
    r.ld_g = ld_g;
    r.dt = dt;
    r.t_submit = now_us();
    r.t_start = 0;
    r.seq = 0;
    s->waiting.push_back(r);
    if (ticket) *ticket = r.ticket;
    DeviceGuardLite guard(ctx->device);
    return sv_progress(s);
}

ot_status ot_assoc_server_poll(ot_assoc_server* s, ot_assoc_server_result* out, int32_t max, int32_t* n) {
    if (!s) return OT_EINVAL;
    DeviceGuardLite guard(s->ctx->device);
    ot_status st = sv_progress(s);
    int k = 0;
    if (out && n) {
        const int m = std::min<int>(max, (int)s->ready.size());
        for (; k < m; ++k) out[k] = s->ready[k];
        s->ready.erase(s->ready.begin(), s->ready.begin() + m);
        *n = k;
    }
    return st;
}

ot_status ot_assoc_server_drain(ot_assoc_server* s, double timeout_s) {
    if (!s) return OT_EINVAL;
    DeviceGuardLite guard(s->ctx->device);
    const double t_end = now_us() + 1e6 * (timeout_s > 0 ? timeout_s : 60.0);
    while (!s->waiting.empty() || !s->prepping.empty() || !s->inflight.empty()) {
        ot_status st = sv_progress(s);
        if (st) return st;
        if (now_us() > t_end) return set_error(s->ctx, OT_ETIMEOUT, "drain: requests still pending");
    }
    return OT_OK;
}

ot_status ot_assoc_server_cell_state(const ot_assoc_server* s, int32_t cell, const float** C, double** f, double** g,
                                     double** rrh_load) {
    if (!s || cell < 0 || cell >= (int32_t)s->cells.size()) return OT_EINVAL;
    const Cell& c = s->cells[cell];
    if (C) *C = c.C;
    if (f) *f = c.f;
    if (g) *g = c.g;
    if (rrh_load) *rrh_load = c.rho;
    return OT_OK;
}

ot_status ot_assoc_server_stats(const ot_assoc_server* s, ot_assoc_server_stats_t* out) {
    if (!s || !out) return OT_EINVAL;
    out->resident_bytes = s->resident;
    out->cells = (int32_t)s->cells.size();
    out->groups = s->ngroups;
    out->group_ctas = s->gsize;
    out->waiting = (int32_t)s->waiting.size();
    out->inflight = (int32_t)(s->prepping.size() + s->inflight.size());
    out->launches = s->launches;
    return OT_OK;
}

}  // extern "C"
