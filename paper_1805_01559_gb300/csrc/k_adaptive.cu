// Adaptive Sinkhorn association (Algorithm 2 of the paper, Sec. V) in one persistent launch.
//
// The RRH targets start from the equal split q_j = sum_i lambda_i / J.  Each outer step solves
// Algorithm 1 with the current q (the whole grid as one group, the same consumer code and
// in-launch finalize as the batched kernel), takes the per-RRH loads rho_j of that plan
// (Sec. II-B, with x = pi the mass plan), picks the most loaded RRH j* (lowest index on
// ties) and moves delta of its target to the other J - 1 RRHs in equal parts.  The paper
// gives no stopping rule for the outer loop: it runs a fixed number of steps and returns the
// last solve's plan with the q that solve used.  A target that delta would drive to zero or
// below moves half of itself instead, so every marginal stays positive.  Each solve after the
// first starts from the previous step's g (warm start).
//
// The targets are kept in FP64 (the algorithm's state, updated with the same operations in
// the same order on every step) and copied to FP32 for the solver.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "k_batch.cuh"

namespace ota {

struct AdStep {  // device-written per outer step
    double max_load, cost, err_row, err_col, err_loop;
    int jstar, iters, converged, status, done, pad;
};

struct AdParams {
    BInst inst;      // the instance; inst.P.q points at q32, inst.rrh_load at the loads
    BGroup grp;      // scratch of the grid-wide group
    double* q64;     // [J] targets (FP64 state); the caller's q_out
    float* q32;      // [J] FP32 copy the solver reads
    BRes* res;       // [outer] per-step solve results (zeroed before the launch)
    AdStep* steps;   // [outer]
    unsigned* gbar;  // group barrier counter (zeroed)
    int* abort;      // launch-wide abort word (zeroed)
    float* pi_last;  // plan of the last step, or null
    double delta;
    int outer;
    int warm;        // 1: steps after the first start from the previous step's g
    long long spin;
};

static constexpr int AD_NW = BT_NT / 32;
// the kernel's static shared memory must stay inside what the stage planner leaves free
static_assert(sizeof(SkShared) + sizeof(BInst) + 64 * AD_NW + 256 <= 4096, "static shared memory");

// Largest value, lowest index on ties, over the CTA (all threads call; result in thread 0).
__device__ __forceinline__ void block_argmax(double v, int i, double* sv, int* si, double* out_v, int* out_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
    if (lane == 0) {
        sv[warp] = v;
        si[warp] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = sv[0];
        int bi = si[0];
        for (int w = 1; w < AD_NW; ++w)
            if (sv[w] > bv || (sv[w] == bv && si[w] < bi)) {
                bv = sv[w];
                bi = si[w];
            }
        *out_v = bv;
        *out_i = bi;
    }
}

__global__ void __launch_bounds__(BT_NT, 1) sk_adaptive(AdParams A) {
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ SkShared sh;
    __shared__ BInst s_inst;
    __shared__ unsigned s_gen;
    __shared__ int s_nbar, s_status, s_js;
    __shared__ double s_v[AD_NW], s_d, s_max;
    __shared__ int s_i[AD_NW];
    const int rank = blockIdx.x, gsize = gridDim.x, tid = threadIdx.x;
    const int J = A.inst.P.J;
    if (tid == 0) {
        s_gen = 0;
        s_nbar = 0;
    }
    // Algorithm 2, initialisation: equal split of the total traffic
    if (rank == 0) {
        double t = 0.0;
        for (int64_t i = tid; i < A.inst.P.I; i += BT_NT) t += (double)A.inst.P.p[i];
        t = warp_sum(t);
        if ((tid & 31) == 0) s_v[tid >> 5] = t;
        __syncthreads();
        double tot = 0.0;
        for (int w = 0; w < AD_NW; ++w) tot += s_v[w];
        const double q0 = tot / (double)J;
        for (int j = tid; j < J; j += BT_NT) {
            A.q64[j] = q0;
            A.q32[j] = (float)q0;
        }
    }
    __syncthreads();
    // the first solve's setup reads q only after its first group barrier: no barrier here
    for (int s = 0; s < A.outer; ++s) {
        if (tid == 0) {
            s_inst = A.inst;
            s_inst.P.g_warm = (s > 0 && A.warm) ? A.inst.g_out : nullptr;
            s_inst.pi = (s + 1 == A.outer) ? A.pi_last : nullptr;
        }
        __syncthreads();
        if (!bt_run(s_inst, A.res + s, A.abort, A.spin, A.grp, rank, gsize, A.gbar, &s_gen, &s_nbar, &sh, dyn))
            return;  // a wait gave up (abort raised)
        // after this barrier every write of the step (status, loads, potentials) is visible
        // and final, so every CTA takes the same decision below
        if (!group_sync(A.gbar, gsize, &s_gen, A.abort, A.spin)) return;
        if (tid == 0) s_status = ld_volatile_i32(&A.res[s].status);
        __syncthreads();
        if (rank == 0) {
            // step 5: the most loaded RRH of this plan
            const double* rho = A.inst.rrh_load;
            double bv = -INFINITY;
            int bi = INT_MAX;
            if (s_status == DEV_OK)
                for (int j = tid; j < J; j += BT_NT) {
                    const double v = rho[j];
                    if (v > bv) {  // j increases within a thread: the first maximum stays
                        bv = v;
                        bi = j;
                    }
                }
            block_argmax(bv, bi, s_v, s_i, &s_max, &s_js);
            if (tid == 0) {
                const BRes& r = A.res[s];
                AdStep o;
                o.max_load = s_status == DEV_OK ? s_max : 0.0;
                o.jstar = s_status == DEV_OK ? s_js : -1;
                o.cost = r.cost;
                o.err_row = r.err_row;
                o.err_col = r.err_col;
                o.err_loop = r.err_loop;
                o.iters = r.iters;
                o.converged = r.converged;
                o.status = s_status;
                o.done = r.done;
                o.pad = 0;
                A.steps[s] = o;
                // step 6 amount: delta, or half the target when delta would exhaust it
                const double qs = A.q64[s_js < J ? s_js : 0];
                s_d = A.delta < qs ? A.delta : 0.5 * qs;
            }
            __syncthreads();
            if (s_status == DEV_OK && s + 1 < A.outer) {
                // step 6: q_j* -= d, every other q_j += d / (J - 1); the next solve's setup
                // reads q after its first group barrier, which orders these writes before it
                const int js = s_js;
                const double d = s_d;
                for (int j = tid; j < J; j += BT_NT) {
                    const double qn = (j == js) ? A.q64[j] - d : A.q64[j] + d / (double)(J - 1);
                    A.q64[j] = qn;
                    A.q32[j] = (float)qn;
                }
            }
        }
        if (s_status != DEV_OK) return;  // the same decision in every CTA
    }
}

}  // namespace ota

using namespace ota;

extern "C" {

ot_status ot_assoc_adaptive(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* traffic, int64_t I,
                            int64_t J, const ot_assoc_adaptive_params* prm, double* f, double* g, double* q_out,
                            double* rrh_load, float* pi, int64_t pi_ld, ot_assoc_adaptive_step* steps,
                            void* stream) {
    if (!ctx) return OT_EINVAL;
    DeviceGuardLite guard(ctx->device);
    if (!C || !traffic || !prm || !f || !g || !q_out || !steps) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J < 2) return set_error(ctx, OT_EINVAL, "need I >= 1 and J >= 2");
    if (J > MAX_J_BATCH) return set_error(ctx, OT_EUNSUPPORTED, "J=%lld above 1024 (adaptive)", (long long)J);
    const int64_t ld = ld_c ? ld_c : J;
    if (ld < J || ld % 4 != 0 || ((uintptr_t)C & 15u))
        return set_error(ctx, OT_EINVAL, "C must be 16-byte aligned with ld %% 4 == 0 and ld >= J");
    if (!(prm->eps > 0.0) || !std::isfinite(prm->eps)) return set_error(ctx, OT_EINVAL, "eps");
    if (!(prm->tol >= 0.0)) return set_error(ctx, OT_EINVAL, "tol");
    if (prm->max_iter < 1) return set_error(ctx, OT_EINVAL, "max_iter");
    if (prm->outer < 1) return set_error(ctx, OT_EINVAL, "outer steps must be >= 1");
    if (!(prm->delta >= 0.0) || !std::isfinite(prm->delta)) return set_error(ctx, OT_EINVAL, "delta");
    if (pi && pi_ld != 0 && pi_ld < J) return set_error(ctx, OT_EINVAL, "pi_ld < J");
    const int nsm = ctx->num_sms;
    const int Jp = (int)round_up(J, 4);
    // partitions first (they depend on I and the stage rows only), then one CTA per partition
    StreamCfg S;
    size_t smem = 0;
    int V = 1;
    if (!plan_stage(BT_NCW, I, Jp, ld, 1, 24576, (size_t)1 << 40, &S, &smem, &V))
        return set_error(ctx, OT_EUNSUPPORTED, "adaptive: no stage plan");
    const int grid = std::max(1, std::min(V, nsm));
    if (!plan_stream(I, Jp, ld, grid, 24576, &S, &smem, &V))
        return set_error(ctx, OT_EUNSUPPORTED, "adaptive: rows do not fit the shared memory (I=%lld)", (long long)I);
    // scratch: [res][steps][gbar][abort] (zeroed) [q32][rho][group scratch]
    auto al = [](size_t x) { return (size_t)round_up((int64_t)x, 256); };
    const int outer = prm->outer;
    size_t off = 0;
    const size_t o_res = off;
    off = al(off + sizeof(BRes) * outer);
    const size_t o_steps = off;
    off = al(off + sizeof(AdStep) * outer);
    const size_t o_bar = off;
    off = al(off + 2 * sizeof(int));
    const size_t zero_end = off;
    const size_t o_q32 = off;
    off = al(off + sizeof(float) * Jp);
    const size_t o_rho = off;
    off = al(off + sizeof(double) * Jp);
    const size_t o_grp = off;
    const size_t gbytes = 1024 + al(gstate_bytes(Jp)) + al((size_t)V * 2 * Jp * 4) + al((size_t)V * 16) +
                          al((size_t)V * Jp * 16) + al((size_t)grid * BT_NW * 16 + (size_t)V * 8);
    off = al(off + gbytes);
    ot_status st = OT_OK;
    char* base = (char*)scratch(ctx, SLOT_MISC, off, &st);
    if (st) return st;
    AdStep* hsteps = (AdStep*)host_staging(ctx, sizeof(AdStep) * outer, &st);
    if (st) return st;
    AdParams A;
    std::memset(&A, 0, sizeof(A));
    ot_assoc_instance a;
    std::memset(&a, 0, sizeof(a));
    a.C = C;
    a.ld = ld;
    a.I = I;
    a.J = (int32_t)J;
    a.p = traffic;
    a.q = (const float*)(base + o_q32);
    a.eps = prm->eps;
    a.tol = prm->tol;
    a.max_iter = prm->max_iter;
    a.f = f;
    a.g = g;
    a.rrh_load = rrh_load ? rrh_load : (double*)(base + o_rho);
    a.pi = pi;
    a.pi_ld = pi_ld;
    fill_values(&A.inst, a);
    A.inst.vpt = vpt_for((int)J);
    A.inst.S = S;
    A.inst.P.V = V;
    A.inst.pi = nullptr;  // only the last step writes the plan
    A.pi_last = pi;
    char* gb = base + o_grp;
    A.grp.sc = (DevScalars*)gb;
    A.grp.ls = (LoopState*)(gb + 512);
    size_t o = 1024;
    A.grp.G = (double*)(gb + o);
    o += al(gstate_bytes(Jp));
    A.grp.colpart = (float*)(gb + o);
    o += al((size_t)V * 2 * Jp * 4);
    A.grp.errpart = (double*)(gb + o);
    o += al((size_t)V * 16);
    A.grp.fpart = (double2*)(gb + o);
    o += al((size_t)V * Jp * 16);
    A.grp.fred = (double*)(gb + o);
    A.grp.phase = 0;
    A.grp.first_cta = 0;
    A.q64 = q_out;
    A.q32 = (float*)(base + o_q32);
    A.res = (BRes*)(base + o_res);
    A.steps = (AdStep*)(base + o_steps);
    A.gbar = (unsigned*)(base + o_bar);
    A.abort = (int*)(base + o_bar + sizeof(int));
    A.delta = prm->delta;
    A.outer = outer;
    A.warm = prm->cold_start ? 0 : 1;
    A.spin = ctx->spin_limit;
    if (allow_max_dynamic_smem((const void*)sk_adaptive, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, OT_ECUDA, "adaptive kernel: %zu bytes of shared memory refused", smem);
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)sk_adaptive, BT_NT, smem) != cudaSuccess ||
        occ < 1 || grid > occ * nsm) {
        cudaGetLastError();
        return set_error(ctx, OT_EUNSUPPORTED, "adaptive kernel cannot be resident");
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(base, 0, zero_end, s);
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(BT_NT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, sk_adaptive, A);
    }
    if (e != cudaSuccess) return cuda_error(ctx, e, "adaptive launch");
    ctx->launches += 1;
    e = cudaMemcpyAsync(hsteps, A.steps, sizeof(AdStep) * outer, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "adaptive");
    // steps after a failed one did not run: they carry the failure's status
    ot_status out = OT_OK;
    for (int k = 0; k < outer; ++k) {
        const AdStep& h = hsteps[k];
        ot_assoc_adaptive_step& d = steps[k];
        std::memset(&d, 0, sizeof(d));
        d.jstar = -1;
        if (out < 0) {
            d.status = out;
            continue;
        }
        int sk;
        if (!h.done) sk = OT_ETIMEOUT;  // the launch gave up before the step ended
        else if (h.status == DEV_EINVAL || h.status == DEV_ENUMERIC) sk = OT_EINVAL;
        else if (h.status == DEV_ETIMEOUT) sk = OT_ETIMEOUT;
        else if (h.status != DEV_OK) sk = OT_ECUDA;
        else sk = h.converged ? OT_OK : OT_NOT_CONVERGED;
        d.status = sk;
        if (sk < 0) {
            out = (ot_status)sk;
            continue;
        }
        d.max_load = h.max_load;
        d.transport_cost = h.cost;
        d.marg_err_row = h.err_row;
        d.marg_err_col = h.err_col;
        d.err_loop = h.err_loop;
        d.jstar = h.jstar;
        d.iters = h.iters;
        d.converged = h.converged;
        if (sk == OT_NOT_CONVERGED) out = OT_NOT_CONVERGED;
    }
    if (out < 0) return set_error(ctx, out, "adaptive: an outer step failed (see the step statuses)");
    return out;
}

}  // extern "C"
