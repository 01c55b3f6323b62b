// eps-scaling (annealing) for Algorithm 1 in one persistent launch.
//
// Small eps makes Sinkhorn slow to converge from b = 1: the plan starts far from the
// minimiser of Eq. (5).  Solving first at a larger eps, where the iteration converges fast,
// and starting each smaller eps from the previous stage's potentials g keeps every stage
// close to its answer: the dual potentials move continuously with eps (they tend to the LP
// duals as eps -> 0).  The stages are eps_s = max(eps, eps0 * factor^s), s = 0, 1, ...;
// intermediate stages stop at tol_stage, the last one at tol.  The answer is the last
// stage's, i.e. the solution of Eq. (5) at the requested eps; the stages only choose the
// starting point of its iteration.  Every stage runs the solver core with the whole grid as
// one group and finalizes in the same launch (the batched kernel's code).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "k_batch.cuh"

namespace ota {

struct EsStage {  // host-written per stage
    double k;     // log2(e) / eps_s
    double eps_ln2;
    double tol;
    float k_hi, k_lo;
    int max_iter;
    int pad;
};

struct EsParams {
    BInst inst;          // the instance (eps fields overwritten per stage)
    BGroup grp;
    const EsStage* stages;
    BRes* res;           // [nstages] (zeroed)
    unsigned* gbar;      // (zeroed)
    int* abort;          // (zeroed)
    float* pi_last;
    int nstages;
    int warm0;           // the first stage starts from the caller's g
    long long spin;
};

static_assert(sizeof(SkShared) + sizeof(BInst) + 256 <= 4096, "static shared memory");

__global__ void __launch_bounds__(BT_NT, 1) sk_eps_scaling(EsParams A) {
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ SkShared sh;
    __shared__ BInst s_inst;
    __shared__ unsigned s_gen;
    __shared__ int s_nbar, s_status;
    const int rank = blockIdx.x, gsize = gridDim.x, tid = threadIdx.x;
    if (tid == 0) {
        s_gen = 0;
        s_nbar = 0;
    }
    for (int s = 0; s < A.nstages; ++s) {
        if (tid == 0) {
            const EsStage st = A.stages[s];
            s_inst = A.inst;
            s_inst.P.k = st.k;
            s_inst.P.k_hi = st.k_hi;
            s_inst.P.k_lo = st.k_lo;
            s_inst.P.tol = st.tol;
            s_inst.P.max_iter = st.max_iter;
            s_inst.eps_ln2 = st.eps_ln2;
            s_inst.P.g_warm = (s > 0 || A.warm0) ? A.inst.g_out : nullptr;
            s_inst.pi = (s + 1 == A.nstages) ? A.pi_last : nullptr;
        }
        __syncthreads();
        if (!bt_run(s_inst, A.res + s, A.abort, A.spin, A.grp, rank, gsize, A.gbar, &s_gen, &s_nbar, &sh, dyn))
            return;  // a wait gave up (abort raised)
        // the stage's g (written before the finalize's last barrier) seeds the next stage;
        // every CTA reads the stage's final status after one more barrier
        if (s + 1 == A.nstages) return;
        if (!group_sync(A.gbar, gsize, &s_gen, A.abort, A.spin)) return;
        if (tid == 0) s_status = ld_volatile_i32(&A.res[s].status);
        __syncthreads();
        if (s_status != DEV_OK) return;  // the same decision in every CTA
    }
}

}  // namespace ota

using namespace ota;

extern "C" {

ot_status ot_assoc_solve_eps_scaling(ot_assoc_ctx* ctx, const float* C, int64_t ld_c, const float* p,
                                     const float* q, int64_t I, int64_t J, double eps, double eps0,
                                     double factor, double tol_stage, double tol, int32_t max_iter,
                                     int32_t warm_start, ot_assoc_result* out, int32_t* stage_iters,
                                     int32_t* nstages_out, void* stream) {
    if (!ctx) return OT_EINVAL;
    DeviceGuardLite guard(ctx->device);
    if (!C || !p || !q || !out || !out->f || !out->g) return set_error(ctx, OT_EINVAL, "null pointer");
    if (I <= 0 || J <= 0) return set_error(ctx, OT_EINVAL, "I and J must be positive");
    if (J > MAX_J_BATCH) return set_error(ctx, OT_EUNSUPPORTED, "J=%lld above 1024 (eps-scaling)", (long long)J);
    const int64_t ld = ld_c ? ld_c : J;
    if (ld < J || ld % 4 != 0 || ((uintptr_t)C & 15u))
        return set_error(ctx, OT_EINVAL, "C must be 16-byte aligned with ld %% 4 == 0 and ld >= J");
    if (!(eps > 0.0) || !std::isfinite(eps)) return set_error(ctx, OT_EINVAL, "eps");
    if (!(eps0 >= eps) || !std::isfinite(eps0)) return set_error(ctx, OT_EINVAL, "eps0 must be >= eps");
    if (!(factor > 0.0 && factor < 1.0)) return set_error(ctx, OT_EINVAL, "factor must be in (0, 1)");
    if (!(tol >= 0.0) || !(tol_stage >= 0.0)) return set_error(ctx, OT_EINVAL, "tol");
    if (max_iter < 1) return set_error(ctx, OT_EINVAL, "max_iter");
    if (out->pi && out->pi_ld != 0 && out->pi_ld < J) return set_error(ctx, OT_EINVAL, "pi_ld < J");
    // stages eps0 * factor^s until eps is reached (the last stage is exactly eps)
    std::vector<EsStage> hs;
    for (double e = eps0;; e *= factor) {
        const bool last = e <= eps * (1.0 + 1e-12);
        const double es = last ? eps : e;
        EsStage st;
        std::memset(&st, 0, sizeof(st));
        st.k = LOG2E / es;
        split_k(st.k, &st.k_hi, &st.k_lo);
        st.eps_ln2 = es * LN2;
        st.tol = last ? tol : tol_stage;
        st.max_iter = max_iter;
        hs.push_back(st);
        if (last) break;
        if (hs.size() >= 64) return set_error(ctx, OT_EINVAL, "more than 64 stages (eps0 / eps too large)");
    }
    const int ns = (int)hs.size();
    const int nsm = ctx->num_sms;
    const int Jp = (int)round_up(J, 4);
    StreamCfg S;
    size_t smem = 0;
    int V = 1;
    if (!plan_stage(BT_NCW, I, Jp, ld, 1, 24576, (size_t)1 << 40, &S, &smem, &V))
        return set_error(ctx, OT_EUNSUPPORTED, "eps-scaling: no stage plan");
    const int grid = std::max(1, std::min(V, nsm));
    if (!plan_stream(I, Jp, ld, grid, 24576, &S, &smem, &V))
        return set_error(ctx, OT_EUNSUPPORTED, "eps-scaling: rows do not fit the shared memory (I=%lld)",
                         (long long)I);
    auto al = [](size_t x) { return (size_t)round_up((int64_t)x, 256); };
    size_t off = 0;
    const size_t o_res = off;
    off = al(off + sizeof(BRes) * ns);
    const size_t o_bar = off;
    off = al(off + 2 * sizeof(int));
    const size_t zero_end = off;
    const size_t o_st = off;
    off = al(off + sizeof(EsStage) * ns);
    const size_t o_grp = off;
    const size_t gbytes = 1024 + al(gstate_bytes(Jp)) + al((size_t)V * 2 * Jp * 4) + al((size_t)V * 16) +
                          al((size_t)V * Jp * 16) + al((size_t)grid * BT_NW * 16 + (size_t)V * 8);
    off = al(off + gbytes);
    ot_status st = OT_OK;
    char* base = (char*)scratch(ctx, SLOT_MISC, off, &st);
    if (st) return st;
    BRes* hres = (BRes*)host_staging(ctx, sizeof(BRes) * ns, &st);
    if (st) return st;
    EsParams A;
    std::memset(&A, 0, sizeof(A));
    ot_assoc_instance a;
    std::memset(&a, 0, sizeof(a));
    a.C = C;
    a.ld = ld;
    a.I = I;
    a.J = (int32_t)J;
    a.p = p;
    a.q = q;
    a.eps = eps;
    a.tol = tol;
    a.max_iter = max_iter;
    a.f = out->f;
    a.g = out->g;
    a.rrh_load = out->rrh_load;
    a.pi = out->pi;
    a.pi_ld = out->pi_ld;
    fill_values(&A.inst, a);
    A.inst.vpt = vpt_for((int)J);
    A.inst.S = S;
    A.inst.P.V = V;
    A.inst.pi = nullptr;
    A.pi_last = out->pi;
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
    A.stages = (const EsStage*)(base + o_st);
    A.res = (BRes*)(base + o_res);
    A.gbar = (unsigned*)(base + o_bar);
    A.abort = (int*)(base + o_bar + sizeof(int));
    A.nstages = ns;
    A.warm0 = warm_start ? 1 : 0;
    A.spin = ctx->spin_limit;
    if (allow_max_dynamic_smem((const void*)sk_eps_scaling, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, OT_ECUDA, "eps-scaling kernel: %zu bytes of shared memory refused", smem);
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)sk_eps_scaling, BT_NT, smem) !=
            cudaSuccess ||
        occ < 1 || grid > occ * nsm) {
        cudaGetLastError();
        return set_error(ctx, OT_EUNSUPPORTED, "eps-scaling kernel cannot be resident");
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(base, 0, zero_end, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_st, hs.data(), sizeof(EsStage) * ns, cudaMemcpyHostToDevice, s);
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
        e = cudaLaunchKernelEx(&cfg, sk_eps_scaling, A);
    }
    if (e != cudaSuccess) return cuda_error(ctx, e, "eps-scaling launch");
    ctx->launches += 1;
    e = cudaMemcpyAsync(hres, A.res, sizeof(BRes) * ns, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "eps-scaling");
    if (nstages_out) *nstages_out = ns;
    int total = 0;
    for (int k = 0; k < ns; ++k) {
        if (stage_iters) stage_iters[k] = hres[k].done ? hres[k].iters : 0;
        total += hres[k].done ? hres[k].iters : 0;
    }
    // the answer is the last stage's; an earlier failure ends the launch before it
    int fail = 0;
    for (int k = 0; k < ns && !fail; ++k)
        if (!hres[k].done) fail = OT_ETIMEOUT;
        else if (hres[k].status == DEV_EINVAL || hres[k].status == DEV_ENUMERIC) fail = OT_EINVAL;
        else if (hres[k].status == DEV_ETIMEOUT) fail = OT_ETIMEOUT;
        else if (hres[k].status != DEV_OK) fail = OT_ECUDA;
    const BRes& L = hres[ns - 1];
    out->transport_cost = L.cost;
    out->marg_err_row = L.err_row;
    out->marg_err_col = L.err_col;
    out->iters = total;
    out->absorptions = 0;
    if (fail) {
        out->status = fail;
        return set_error(ctx, (ot_status)fail, "eps-scaling: a stage failed");
    }
    out->status = L.converged ? OT_OK : OT_NOT_CONVERGED;
    return (ot_status)out->status;
}

}  // extern "C"
