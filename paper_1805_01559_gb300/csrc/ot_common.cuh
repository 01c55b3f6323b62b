// Device helpers shared by the library's kernels (not by the oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ota {

// Device status word values (the host maps them to ot_status).
enum : int {
    DEV_OK = 0,
    DEV_EINVAL = -1,
    DEV_ETIMEOUT = -4,
};

// 2^x on the SFU (MUFU.EX2), flushing subnormal results to zero.  2^-inf = 0.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// log2(r) with full relative accuracy near r = 1, where Sinkhorn's row and column
// corrections live (r - 1 is exact there by Sterbenz' lemma).
__device__ __forceinline__ float log2_rel(float r) {
    if (r > 0.5f && r < 2.0f) return log1pf(r - 1.0f) * 1.4426950408889634f;
    return log2f(r);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Merge two (max, sum of 2^(x - max)) pairs.
__device__ __forceinline__ void lse2_merge(float& m, float& s, float m2, float s2) {
    float mx = fmaxf(m, m2);
    if (mx == -INFINITY) return;  // both empty
    s = s * ex2(m - mx) + s2 * ex2(m2 - mx);
    m = mx;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    return *(volatile const int*)p;
}

// Grid-wide barrier for a cooperative (co-resident) launch, with a bounded spin.
// `count` is monotonic within a launch (zeroed by the host before it); the
// caller passes target = gridDim.x * generation.  Returns false when the wait gave
// up (status set to DEV_ETIMEOUT) or another CTA already reported an error; the
// caller must then leave the kernel.  Every thread of the CTA must call it.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned target, int* status,
                                             long long spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(count, 1u);
        long long n = 0;
        while (ld_acquire_u32(count) < target) {
            if (ld_volatile_i32(status) != DEV_OK) { ok = 0; break; }
            if (++n > spin_limit) {
                atomicCAS(status, DEV_OK, DEV_ETIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void bar_named(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ float& comp(float4& v, int c) {
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }

template <int TW>
struct Team {
    static constexpr int TT = 32 * TW;
    int team, wit, lane, tl;
    __device__ __forceinline__ Team() {
        const int warp = threadIdx.x >> 5;
        lane = threadIdx.x & 31;
        team = warp / TW;
        wit = warp % TW;
        tl = wit * 32 + lane;
    }
};

// Team-wide sum/max in a fixed order.  `red` has room for 2 * nteams * TW values of T;
// the two halves alternate so one named barrier per call suffices.
template <int TW, typename T, bool MAX>
__device__ __forceinline__ T team_reduce(T v, T* red, int nteams, const Team<TW>& tm, int& par) {
    if (MAX) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = vmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    if constexpr (TW == 1) {
        return v;
    } else {
        T* r = red + (par * nteams + tm.team) * TW;
        if (tm.lane == 0) r[tm.wit] = v;
        bar_named(1 + tm.team, 32 * TW);
        T s = r[0];
#pragma unroll
        for (int w = 1; w < TW; ++w) s = MAX ? vmax(s, r[w]) : s + r[w];
        par ^= 1;
        return s;
    }
}

// Row load: thread chunk v covers columns 4*(tl + TT*v) .. +3.  Columns >= J read as
// `fill` (+inf for a cost: zero mass).  Rows are 16-byte aligned (ld % 4 == 0), so a chunk
// that starts below J never leaves the padded row.
template <int TW, int VPT>
__device__ __forceinline__ void load_row(const float* __restrict__ row, int J, int tl,
                                         float4 (&x)[VPT], float fill = INFINITY) {
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int col = 4 * (tl + 32 * TW * v);
        if (col < J) {
            float4 t = __ldg(reinterpret_cast<const float4*>(row + col));
            if (col + 4 > J) {
                if (col + 1 >= J) t.y = fill;
                if (col + 2 >= J) t.z = fill;
                if (col + 3 >= J) t.w = fill;
            }
            x[v] = t;
        } else {
            x[v] = make_float4(fill, fill, fill, fill);
        }
    }
}


// ---- mbarrier + bulk-copy (TMA) helpers, CTA scope ---------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_try_wait, but a thread whose phase is not complete is suspended in hardware for
// up to `ns` nanoseconds (woken as soon as the phase completes) instead of returning at
// once, so waiting warps do not take issue slots from working ones.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with the given parity, at most `limit` polls.  On expiry the
// device status becomes DEV_ETIMEOUT; a status already set by another CTA also ends the wait.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit, int* status) {
    long long n = 0;
    while (!mbar_try_wait_sleep(bar, parity, 1000)) {
        if ((++n & 1023) == 0 && ld_volatile_i32(status) != DEV_OK) return false;
        if (n > limit) {
            atomicCAS(status, DEV_OK, DEV_ETIMEOUT);
            return false;
        }
    }
    return true;
}

// One bulk copy global -> shared completing on `bar` (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Grid barrier for kernels whose CTAs hold a warp that does not take part (a copy producer):
// the CTA-level synchronisation is the named barrier `bar_id` over `nthreads` threads.  One
// thread publishes the CTA's arrival with a release add (ordered after the CTA's writes by
// the named barrier) and polls with acquire loads; the second named barrier passes what it
// acquired on to the rest of the CTA.  Polls sleep only after the first few hundred.
__device__ __forceinline__ bool grid_barrier_named(unsigned* count, unsigned target, int* status,
                                                   long long spin_limit, int bar_id, int nthreads,
                                                   int* s_ok) {
    bar_named(bar_id, nthreads);
    if (threadIdx.x == 0) {
        int ok = 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        long long n = 0;
        while (ld_acquire_u32(count) < target) {
            ++n;
            if ((n & 63) == 0 && ld_volatile_i32(status) != DEV_OK) { ok = 0; break; }
            if (n > spin_limit) {
                atomicCAS(status, DEV_OK, DEV_ETIMEOUT);
                ok = 0;
                break;
            }
            if (n > 256) __nanosleep(32);
        }
        *s_ok = ok;
    }
    bar_named(bar_id, nthreads);
    return *(volatile int*)s_ok != 0;
}

// ---- FP32 pair ("double-float") arithmetic: GB300 issues FP64 at a small fraction of the
// FP32 rate, so sums that need more than 24 bits are carried as unevaluated pairs. -------
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) + b, renormalised.
__device__ __forceinline__ float2 df_add(float2 a, float b) {
    float s, e;
    two_sum_f(a.x, b, s, e);
    e += a.y;
    float h, l;
    two_sum_f(s, e, h, l);
    return make_float2(h, l);
}

__device__ __forceinline__ float2 df_add2(float2 a, float2 b) {
    float s, e;
    two_sum_f(a.x, b.x, s, e);
    e += a.y + b.y;
    float h, l;
    two_sum_f(s, e, h, l);
    return make_float2(h, l);
}

__device__ __forceinline__ float2 warp_sum_df(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float2 w;
        w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
        w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
        v = df_add2(v, w);
    }
    return v;
}

// log2 of a positive pair value: exact exponent plus the FP32 log2 of the mantissa, so the
// absolute error is that of log2f on [1, 2) (a few 2^-24), whatever the magnitude.
__device__ __forceinline__ float2 df_log2(float2 a) {
    int e;
    const float m = frexpf(a.x, &e);  // a.x = m 2^e, m in [0.5, 1)
    const float lm = log2f(m) + a.y / (a.x * 0.69314718f);
    return make_float2((float)e, lm);  // value = e + lm (both exact in the pair)
}

}  // namespace ota
