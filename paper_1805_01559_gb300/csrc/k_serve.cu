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
// counts itself idle; when every group is counted, the launch closes (one compare-and-swap
// marks the count) and all groups leave together; the host starts a new launch when work
// comes.  A counted group leaves the count before it claims work, which a closing launch
// refuses: a launch never goes on with only some of its groups.
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
// How a request's cost is rebuilt, by the CTAs that solve it, from their own rows.
struct SvPrep {
    const float* G;      // gains [I][ld_g] (caller mode), or nullptr: drifting cell
    int64_t ld_g;
    double* dev_xy;      // [I][2] (drift mode)
    double* dev_v;       // [I][2]
    const float* rrh_xy; // [J][2]
    const float* shadow; // [I][J] dB
    const float* P;      // [J]
    double dt, side;
    float N0, W, mu, pad;
};

struct SvQueue {
    unsigned tail;   // descriptors published (host writes, release)
    unsigned stop;   // host asks idle groups to leave at once
    unsigned pad[30];
    BInst desc[SV_CAP];
    SvPrep prep[SV_CAP];
    BRes res[SV_CAP];
    unsigned done[SV_CAP];  // sequence number + 1 of the request whose result is in res[]
};

struct SvCtl {  // device memory, zeroed once
    unsigned head;  // descriptors claimed
    int abort;
    unsigned idle;  // groups of the current launch that found no work, | SV_CLOSING once every
                    // group was counted and the launch is ending (zeroed per launch)
};
constexpr unsigned SV_CLOSING = 1u << 31;

struct ServeParams {
    SvQueue* q;          // device view of the mapped queue
    SvCtl* ctl;
    BRes* dres;          // [SV_CAP] device result slots (status words while solving)
    const BGroup* groups;
    unsigned* gbar;      // [ngroups]
    int* gcur;           // [ngroups]
    int gsize, ngroups;
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

// Received power P G of one link from the path-loss model with the link's fixed shadowing X
// (dB), which adds to the path loss: G = 10^(-(PL0 + 10 n log10 d + X) / 10), evaluated as
// 2^(a0 - X/10 log2(10) - (n/2) log2 d^2) on the SFU (a simulation input).
__device__ __forceinline__ float sv_pl(float x, float y, float rx, float ry, float sh, float P) {
    const float l2_10 = 3.3219280948873622f;  // log2(10)
    const float a0 = -30.0f * 0.1f * l2_10;   // -PL0/10 log2(10), PL0 = 30 dB
    const float half_n = 0.5f * 3.5f;         // n/2 with the path-loss exponent n = 3.5
    const float dx = x - rx, dy = y - ry;
    const float d2 = fmaxf(fmaf(dx, dx, dy * dy), 100.0f);  // d >= 10 m
    const float e = fmaf(sh, -0.1f * l2_10, a0) - half_n * __log2f(d2);
    return P * ex2(e);
}

// Received power P_j G_ij of one cell: the caller's gains, or the path-loss model.
__device__ __forceinline__ float sv_power(const SvPrep& Q, int64_t i, int J, int j, float x, float y) {
    if (Q.G) return Q.P[j] * __ldg(Q.G + i * Q.ld_g + j);
    return sv_pl(x, y, Q.rrh_xy[2 * j], Q.rrh_xy[2 * j + 1], __ldg(Q.shadow + i * (int64_t)J + j), Q.P[j]);
}

// Rate (Sec. II-A, every other RRH interfering; the row total of received powers as the FP32
// pair (hi, lo)) and cost C = 1 / (mu R) of a cell with received power pg; +inf (and bad set)
// when the rate is not finite and > 0.
__device__ __forceinline__ float sv_cost(const SvPrep& Q, float pg, float hi, float lo, int& bad) {
    const float inv_ln2 = 1.4426950408889634f;
    const float interf = ((hi - pg) + lo) + Q.N0;
    const float R = Q.W * log1pf(__fdividef(pg, interf)) * inv_ln2;
    const bool ok = R > 0.f && isfinite(R);
    bad |= !ok;
    return ok ? __frcp_rn(Q.mu * R) : INFINITY;
}

// One row in chunks of four columns (J a multiple of 4 and every row 16-byte aligned): a lane
// owns chunks col = 4 (lane + 32 v), loads gains or shadowing, RRH coordinates and powers as
// 16-byte vectors and keeps its received powers in registers between the pass that forms the
// row total and the pass that writes the costs.
template <int VPT>
__device__ __forceinline__ void sv_row_vec(const SvPrep& Q, float* row, int J, int64_t i, float x, float y, int lane,
                                           int& bad) {
    float4 pw[VPT];
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int col = 4 * (lane + 32 * v);
        float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (col < J) {
            const float4 P4 = __ldg(reinterpret_cast<const float4*>(Q.P + col));
            if (Q.G) {
                const float4 g = __ldg(reinterpret_cast<const float4*>(Q.G + i * Q.ld_g + col));
                p4 = make_float4(P4.x * g.x, P4.y * g.y, P4.z * g.z, P4.w * g.w);
            } else {
                const float4 s4 = __ldg(reinterpret_cast<const float4*>(Q.shadow + i * (int64_t)J + col));
                const float4 ra = __ldg(reinterpret_cast<const float4*>(Q.rrh_xy + 2 * col));
                const float4 rb = __ldg(reinterpret_cast<const float4*>(Q.rrh_xy + 2 * col + 4));
                p4 = make_float4(sv_pl(x, y, ra.x, ra.y, s4.x, P4.x), sv_pl(x, y, ra.z, ra.w, s4.y, P4.y),
                                 sv_pl(x, y, rb.x, rb.y, s4.z, P4.z), sv_pl(x, y, rb.z, rb.w, s4.w, P4.w));
            }
        }
        pw[v] = p4;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float t, e2;
            two_sum(hi, comp(p4, c), t, e2);
            hi = t;
            lo += e2;
        }
    }
    warp_sum_pair(hi, lo);
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int col = 4 * (lane + 32 * v);
        if (col < J) {
            float4 o;
#pragma unroll
            for (int c = 0; c < 4; ++c) comp(o, c) = sv_cost(Q, comp(pw[v], c), hi, lo, bad);
            *reinterpret_cast<float4*>(row + col) = o;
        }
    }
}

// Rebuild the cost of rows [r0, r1) of a request's instance (all threads of the CTA, one warp
// per row): positions moved by dt (drift mode; FP32 arithmetic, lanes 0 and 1 one axis each)
// and received powers from the path-loss model with the cell's fixed shadowing, or the
// caller's gains; then the rates with every other RRH interfering (Sec. II-A) and
// C = 1 / (mu R).  Rows of up to 1024 columns whose arrays are 16-byte aligned go in float4
// chunks (sv_row_vec); others column by column, the second pass recomputing each power.
// Invalid rates fail the request.
__device__ __forceinline__ void sv_rebuild_rows(const SvPrep& Q, float* C, int64_t ldc, int J, int64_t r0, int64_t r1,
                                                int* status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float side = (float)Q.side, dt = (float)Q.dt;
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
    const bool vec = J <= 1024 && J % 4 == 0 && ldc % 4 == 0 && a16(C) && a16(Q.P) &&
                     (Q.G ? (Q.ld_g % 4 == 0 && a16(Q.G)) : (a16(Q.shadow) && a16(Q.rrh_xy)));
    int bad = 0;
    for (int64_t i = r0 + warp; i < r1; i += nw) {
        float pos = 0.f;
        if (!Q.G && lane < 2) {  // lane 0: x, lane 1: y
            const float x0 = (float)Q.dev_xy[2 * i + lane], v = (float)Q.dev_v[2 * i + lane];
            const float x1 = fmaf(v, dt, x0);
            const float per = 2.f * side;
            float pm = x1 - per * floorf(x1 / per);
            if (pm > side) pm = per - pm;
            if (((int)floorf(x1 / side)) & 1) Q.dev_v[2 * i + lane] = -(double)v;
            Q.dev_xy[2 * i + lane] = (double)pm;
            pos = pm;
        }
        const float x = __shfl_sync(0xffffffffu, pos, 0), y = __shfl_sync(0xffffffffu, pos, 1);
        float* row = C + i * ldc;
        if (vec && J <= 128) {
            sv_row_vec<1>(Q, row, J, i, x, y, lane, bad);
        } else if (vec && J <= 256) {
            sv_row_vec<2>(Q, row, J, i, x, y, lane, bad);
        } else if (vec && J <= 512) {
            sv_row_vec<4>(Q, row, J, i, x, y, lane, bad);
        } else if (vec) {
            sv_row_vec<8>(Q, row, J, i, x, y, lane, bad);
        } else {
            float hi = 0.f, lo = 0.f;
            for (int j = lane; j < J; j += 32) {
                float t, e2;
                two_sum(hi, sv_power(Q, i, J, j, x, y), t, e2);
                hi = t;
                lo += e2;
            }
            warp_sum_pair(hi, lo);
            for (int j = lane; j < J; j += 32) row[j] = sv_cost(Q, sv_power(Q, i, J, j, x, y), hi, lo, bad);
        }
    }
    if (bad) atomicCAS(status, DEV_OK, DEV_EINVAL);
}

// The same rebuild as a standalone launch over all rows (a cell's first instance, dt = 0).
__global__ void __launch_bounds__(256) sv_rebuild_all(SvPrep Q, float* C, int64_t ldc, int64_t I, int J, int* status) {
    const int64_t rows_per_block = 8 * ((I + 8LL * gridDim.x - 1) / (8LL * gridDim.x));
    const int64_t r0 = min(I, (int64_t)blockIdx.x * rows_per_block), r1 = min(I, r0 + rows_per_block);
    sv_rebuild_rows(Q, C, ldc, J, r0, r1, status);
}

__global__ void __launch_bounds__(BT_NT, 1) sk_serve(ServeParams S) {
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ SkShared sh;
    __shared__ __align__(16) BInst s_inst;
    __shared__ __align__(16) SvPrep s_prep;
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
            // claim the next published request.  A group that found nothing for idle_polls
            // polls counts itself idle and keeps polling.  The group that finds every group
            // counted closes the launch (CAS: all counted -> all counted | CLOSING) and every
            // group leaves; a counted group that sees work first leaves the count, by a CAS
            // that fails once the launch is closing.  So either all groups stay or all leave
            // (the host relaunches on new work).  At most `spin` polls.
            int idx = -1;
            long long n = 0;
            bool counted = false;
            const unsigned all = (unsigned)S.ngroups;
            for (;;) {
                if (ld_acquire_sys_u32(&S.q->stop)) break;
                const unsigned iv = *(volatile unsigned*)&S.ctl->idle;
                if (iv & SV_CLOSING) break;
                const unsigned t = ld_acquire_sys_u32(&S.q->tail);
                const unsigned h = *(volatile unsigned*)&S.ctl->head;
                if (h < t) {
                    if (counted) {
                        if (atomicCAS(&S.ctl->idle, iv, iv - 1u) != iv) continue;  // changed: look again
                        counted = false;
                        n = 0;
                    }
                    if (atomicCAS(&S.ctl->head, h, h + 1) == h) {
                        idx = (int)h;
                        break;
                    }
                    continue;
                }
                ++n;
                if (!counted && n > S.idle_polls) {
                    atomicAdd(&S.ctl->idle, 1u);
                    counted = true;
                    continue;
                }
                if (counted && iv == all && atomicCAS(&S.ctl->idle, all, all | SV_CLOSING) == all) break;
                if (n > S.spin) break;
                __nanosleep(n < 4096 ? 256 : 2048);
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
        {  // the descriptors into shared memory (read once from host memory)
            const unsigned* src = reinterpret_cast<const unsigned*>(&S.q->desc[slot]);
            unsigned* dst = reinterpret_cast<unsigned*>(&s_inst);
            for (int k = threadIdx.x; k < (int)(sizeof(BInst) / 4); k += blockDim.x) dst[k] = src[k];
            const unsigned* src2 = reinterpret_cast<const unsigned*>(&S.q->prep[slot]);
            unsigned* dst2 = reinterpret_cast<unsigned*>(&s_prep);
            for (int k = threadIdx.x; k < (int)(sizeof(SvPrep) / 4); k += blockDim.x) dst2[k] = src2[k];
        }
        __syncthreads();
        BRes* out = S.dres + slot;
        {  // this CTA's rows of the new cost, before its bulk copies read them
            int64_t r0, r1;
            cta_rows(s_inst.P.I, s_inst.S.rows_per_stage, s_inst.P.V, rank, S.gsize, &r0, &r1);
            sv_rebuild_rows(s_prep, const_cast<float*>(s_inst.P.C), s_inst.P.ld, s_inst.P.J, r0, r1, &out->status);
            asm volatile("fence.proxy.async.global;" ::: "memory");
            __syncthreads();
        }
        if (!bt_run(s_inst, out, &S.ctl->abort, S.spin, grp, rank, S.gsize, gbar, &s_gen, &s_nbar, &sh, dyn))
            return;
        if (rank == 0 && threadIdx.x == 0) {
            S.q->res[slot] = *out;
            __threadfence_system();
            st_release_sys_u32(&S.q->done[slot], (unsigned)idx + 1u);
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
    cudaStream_t run_stream = nullptr;
    cudaEvent_t run_done = nullptr;
    bool running = false;
    size_t smem = 0;
    std::vector<Cell> cells;
    std::deque<Request> waiting;     // submitted, cell busy or not yet started
    std::vector<Request> inflight;   // published to the kernel
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
    // group barrier counters and the idle count restart with every launch
    cudaError_t e = cudaMemsetAsync(s->params.gbar, 0, sizeof(unsigned) * s->ngroups, s->run_stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&s->params.ctl->idle, 0, sizeof(unsigned), s->run_stream);
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, sk_serve, s->params);
    if (e == cudaSuccess) e = cudaEventRecord(s->run_done, s->run_stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "server launch");
    s->running = true;
    ++s->launches;
    ctx->launches += 1;
    return OT_OK;
}

// Publish a request to the kernel's queue (its cell is idle).
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
    d.vpt = vpt_for(c.J);
    size_t sm = 0;
    if (!plan_stream(c.I, d.P.Jp, c.ldc, s->gsize, 24576, &d.S, &sm, &d.P.V))
        return set_error(s->ctx, OT_EUNSUPPORTED, "cell does not fit the server's groups");
    SvPrep pr;
    std::memset(&pr, 0, sizeof(pr));
    pr.G = r.G;
    pr.ld_g = r.ld_g;
    pr.dev_xy = c.dev_xy;
    pr.dev_v = c.dev_v;
    pr.rrh_xy = c.rrh_xy;
    pr.shadow = c.shadow;
    pr.P = c.P;
    pr.dt = r.dt;
    pr.side = c.side;
    pr.N0 = (float)c.N0;
    pr.W = (float)c.W;
    pr.mu = (float)c.mu;
    s->q_host->desc[slot] = d;
    s->q_host->prep[slot] = pr;
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
    // 1. publish waiting requests whose cell is idle (in submission order)
    for (auto it = s->waiting.begin(); it != s->waiting.end();) {
        Cell& c = s->cells[it->cell];
        if (c.busy || (int)s->inflight.size() >= SV_CAP / 2) {
            ++it;
            continue;
        }
        c.busy = true;
        Request r = *it;
        it = s->waiting.erase(it);
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

ot_status ot_assoc_build_cost_mobile(ot_assoc_ctx* ctx, double* dev_xy, double* dev_v, const float* rrh_xy,
                                     const float* shadow_db, const float* P, int64_t I, int64_t J, double dt,
                                     double side_m, double N0, double W_hz, double mu, float* C_out, int64_t ld_c,
                                     double eps_rel, double* eps_out, void* stream) {
    using namespace ota;
    if (!ctx) return OT_EINVAL;
    if (!dev_xy || !dev_v || !rrh_xy || !shadow_db || !P || !C_out) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0) return set_error(ctx, OT_EINVAL, "I and J must be positive");
    if (J > (1 << 20)) return set_error(ctx, OT_EUNSUPPORTED, "J too large");
    if (ld_c == 0) ld_c = J;
    if (ld_c < J) return set_error(ctx, OT_EINVAL, "leading dimension < J");
    if (!(dt >= 0.0) || !std::isfinite(dt) || !(side_m > 0.0) || !std::isfinite(side_m))
        return set_error(ctx, OT_EINVAL, "need dt >= 0 and side_m > 0");
    if (!(N0 >= 0.0) || !(W_hz > 0.0)) return set_error(ctx, OT_EINVAL, "need N0 >= 0 and W_hz > 0");
    if (!(mu > 0.0) || !std::isfinite(mu)) return set_error(ctx, OT_EINVAL, "mu must be finite and > 0");
    if (eps_out && !(eps_rel > 0.0)) return set_error(ctx, OT_EINVAL, "eps_rel must be > 0");
    DeviceGuardLite g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    SvPrep pr;
    std::memset(&pr, 0, sizeof(pr));
    pr.dev_xy = dev_xy;
    pr.dev_v = dev_v;
    pr.rrh_xy = rrh_xy;
    pr.shadow = shadow_db;
    pr.P = P;
    pr.dt = dt;
    pr.side = side_m;
    pr.N0 = (float)N0;
    pr.W = (float)W_hz;
    pr.mu = (float)mu;
    ot_status st = OT_OK;
    char* state = (char*)scratch(ctx, SLOT_MISC, 256, &st);
    if (st) return st;
    int* dstat = (int*)state;
    double* dmed = (double*)(state + 64);
    cudaError_t e = cudaMemsetAsync(dstat, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "memset");
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((I + 63) / 64, 4LL * ctx->num_sms));
    sv_rebuild_all<<<grid, 256, 0, s>>>(pr, C_out, ld_c, I, (int)J, dstat);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "mobile cost");
    ctx->launches += 1;
    if (!eps_out) return OT_OK;
    st = launch_median(ctx, C_out, I, J, ld_c, dmed, s);
    if (st) return st;
    struct {
        int bad;
        int pad;
        double med;
    }* h = (decltype(h))host_staging(ctx, 64, &st);
    if (st) return st;
    e = cudaMemcpyAsync(&h->bad, dstat, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h->med, dmed, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "mobile cost");
    if (h->bad != DEV_OK) return set_error(ctx, OT_EINVAL, "some rate is not finite and > 0");
    *eps_out = eps_rel * h->med;
    return OT_OK;
}

ot_status ot_assoc_server_create(ot_assoc_ctx* ctx, const ot_assoc_server_config* cfg, ot_assoc_server** out) {
    if (!ctx) return OT_EINVAL;
    if (!out) return set_error(ctx, OT_EINVAL, "null output pointer");
    *out = nullptr;
    DeviceGuardLite guard(ctx->device);
    ot_assoc_server* s = new ot_assoc_server;
    s->ctx = ctx;
    if (cfg) s->cfg = *cfg;
    const int nsm = ctx->num_sms;
    // default: four groups (a quarter of the SMs each), the best measured on the mixed-size
    // serving cells (groups of 152 / 76 / 38 / 19 CTAs served 1298 / 1658 / 2838 / 2821
    // solves/s on 152 SMs); an SM count that is not a multiple of 4 takes one group
    s->gsize = s->cfg.group_ctas > 0 ? s->cfg.group_ctas : (nsm % 4 == 0 ? nsm / 4 : nsm);
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
    const size_t gbytes = 1024 + al(gstate_bytes((int)Jp)) + al(nv * 2 * Jp * 4) + al(nv * 16) + al(nv * Jp * 16) +
                          al((size_t)s->gsize * BT_NW * 16 + nv * 8);
    const size_t o_ctl = 0, o_res = al(sizeof(SvCtl)), o_gbar = o_res + al(sizeof(BRes) * SV_CAP);
    const size_t o_gcur = o_gbar + al(sizeof(unsigned) * s->ngroups), o_groups = o_gcur + al(sizeof(int) * s->ngroups);
    const size_t o_scr = o_groups + al(sizeof(BGroup) * s->ngroups), total = o_scr + gbytes * s->ngroups;
    cudaError_t e = cudaMalloc(&s->dmem, total);
    if (e == cudaSuccess) e = cudaMemset(s->dmem, 0, o_scr);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->q_host, sizeof(SvQueue), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&s->q_dev, s->q_host, 0);
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
        o += al(gstate_bytes((int)Jp));
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
    P.ngroups = s->ngroups;
    P.idle_polls = (long long)(idle / 0.3);  // a poll sleeps about 0.3 us
    P.spin = ctx->spin_limit;
    s->smem = SMEM_BUDGET;
    if (allow_max_dynamic_smem((const void*)sk_serve, s->smem) !=
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
    for (auto& c : s->cells) sv_free_cell(s, c);
    if (s->run_done) cudaEventDestroy(s->run_done);
    if (s->run_stream) cudaStreamDestroy(s->run_stream);
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
    if (!(d->mu > 0.0) || !(d->W_hz > 0.0) || !(d->N0 > 0.0))
        return set_error(ctx, OT_EINVAL, "mu, W and N0 must be > 0");
    if (!(d->eps > 0.0) && !(d->eps_rel > 0.0 && d->dev_xy))
        return set_error(ctx, OT_EINVAL, "eps must be > 0 (or eps_rel > 0 for a drifting cell)");
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
    if (drift) {
        SV_ALLOC(dev_xy, double, 2 * I);
        SV_ALLOC(dev_v, double, 2 * I);
        SV_ALLOC(rrh_xy, float, 2 * J);
        SV_ALLOC(shadow, float, I * J);
    }
#undef SV_ALLOC
    cudaError_t e = cudaMemcpy(c.p, d->p, sizeof(float) * I, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.q, d->q, sizeof(float) * J, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.P, d->P, sizeof(float) * J, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c.g, 0, sizeof(double) * ldc);
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
    if (!(c.eps > 0.0)) {  // eps = eps_rel * median(C) of the first instance (built here, dt = 0)
        SvPrep pr;
        std::memset(&pr, 0, sizeof(pr));
        pr.dev_xy = c.dev_xy;
        pr.dev_v = c.dev_v;
        pr.rrh_xy = c.rrh_xy;
        pr.shadow = c.shadow;
        pr.P = c.P;
        pr.side = c.side;
        pr.N0 = (float)c.N0;
        pr.W = (float)c.W;
        pr.mu = (float)c.mu;
        int* dstat = nullptr;
        double* dmed = nullptr;
        st = OT_OK;
        char* tmp = (char*)scratch(ctx, SLOT_MISC, 256, &st);
        if (st) {
            sv_free_cell(s, c);
            return st;
        }
        dstat = (int*)tmp;
        dmed = (double*)(tmp + 64);
        e = cudaMemset(dstat, 0, sizeof(int));
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((c.I + 63) / 64, 4LL * ctx->num_sms));
        if (e == cudaSuccess) {
            sv_rebuild_all<<<grid, 256, 0, s->run_stream>>>(pr, c.C, c.ldc, c.I, c.J, dstat);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            st = launch_median(ctx, c.C, c.I, c.J, c.ldc, dmed, s->run_stream);
            if (st) {
                sv_free_cell(s, c);
                return st;
            }
        }
        double med = 0.0;
        int hs = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&med, dmed, sizeof(double), cudaMemcpyDeviceToHost, s->run_stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, dstat, sizeof(int), cudaMemcpyDeviceToHost, s->run_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->run_stream);
        if (e != cudaSuccess) {
            sv_free_cell(s, c);
            return cuda_error(ctx, e, "first instance");
        }
        if (hs != DEV_OK || !(med > 0.0) || !std::isfinite(med)) {
            sv_free_cell(s, c);
            return set_error(ctx, OT_EINVAL, "the cell's first instance has invalid rates");
        }
        c.eps = d->eps_rel * med;
        ctx->launches += 1;
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
    while (!s->waiting.empty() || !s->inflight.empty()) {
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

ot_status ot_assoc_server_cell_eps(const ot_assoc_server* s, int32_t cell, double* eps) {
    if (!s || !eps || cell < 0 || cell >= (int32_t)s->cells.size()) return OT_EINVAL;
    *eps = s->cells[cell].eps;
    return OT_OK;
}

ot_status ot_assoc_server_stats(const ot_assoc_server* s, ot_assoc_server_stats_t* out) {
    if (!s || !out) return OT_EINVAL;
    out->resident_bytes = s->resident;
    out->cells = (int32_t)s->cells.size();
    out->groups = s->ngroups;
    out->group_ctas = s->gsize;
    out->waiting = (int32_t)s->waiting.size();
    out->inflight = (int32_t)s->inflight.size();
    out->launches = s->launches;
    return OT_OK;
}

}  // extern "C"
