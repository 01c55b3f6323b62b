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

}  // namespace ota
