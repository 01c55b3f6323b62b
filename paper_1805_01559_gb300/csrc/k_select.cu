// Exact median of FP32 values.
// eps = eps_rel * median(C) is how the benchmark configurations fix the regularization
// strength of Eq. (5); the median of an even count is the mean of the two middle values.
//
// Method (all on the device, no host round trip):
//   1. take s = 65536 entries at a fixed stride and select, exactly, the sample ranks
//      s/2 -+ 6 sd (sd = sqrt(s)/2, the rank spread of a sample median): a bracket [lo, hi];
//   2. one pass over all n entries counts those below lo and compacts those in [lo, hi]
//      into a candidate buffer (a few percent of n);
//   3. if both middle ranks fall inside the bracket and the candidates fit, select them
//      among the candidates; otherwise select over all n entries.
// Selection is a radix select (8 bits per pass) on order-preserving keys that tracks both
// middle ranks at once; among the candidates it starts below the leading bits that lo and
// hi share, which spreads the first pass over many bins.  Each histogram pass ends with
// its last block to finish (a counter, no waiting) picking the digits for the next pass.
// The result is exact either way and does not depend on the order in which candidates were
// compacted or blocks finished.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "ot_common.cuh"
#include "ot_internal.h"

namespace ota {

static constexpr int RS_BITS = 8;
static constexpr int RS_BINS = 1 << RS_BITS;
static constexpr int RS_PASSES = 32 / RS_BITS;
static constexpr int64_t SAMPLE = 65536;

// Order-preserving map float bits -> unsigned key (negative values reversed).
__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

struct SelectState {
    unsigned long long hist[2][RS_BINS];
    long long rank[2];          // rank still to find inside the current prefix
    uint32_t prefix[2];         // key bits fixed so far (in the low bits)
    int two;                    // 1 when two targets are tracked
    int bits_done;              // leading key bits fixed so far (32: done)
    int use_cand;               // histogram the candidate buffer (1) or all entries (0)
    unsigned int arrived;       // blocks of the current launch that have finished
    unsigned long long n_cand;  // entries found in [lo, hi]
    unsigned long long c_lo;    // entries found below lo
    long long k1, k2;           // target ranks in the full data
};

// The data a pass reads: a strided row-major view (rows x cols, leading dimension ld), or
// the candidate buffer.  flat: the view is one contiguous run of rows * cols entries.
struct SelSrc {
    const float* x;
    int64_t rows, cols, ld;
    const float* cand;
    int vec;   // 16-byte aligned rows (or run): float4 loads
    int flat;
};

// Number of 4-entry chunks of the view.
__host__ __device__ __forceinline__ int64_t n_chunks(const SelSrc& src) {
    return src.flat ? (src.rows * src.cols + 3) / 4 : src.rows * ((src.cols + 3) / 4);
}

// Up to four consecutive entries of the view: chunk t of n chunks.
__device__ __forceinline__ void load_chunk(const SelSrc& src, int64_t t, int64_t n, float v[4], bool ok[4]) {
    v[0] = v[1] = v[2] = v[3] = 0.f;
    ok[0] = ok[1] = ok[2] = ok[3] = false;
    if (t >= n) return;
    const float* p;
    int64_t left;  // entries of this row (or run) from p on
    if (src.flat) {
        p = src.x + 4 * t;
        left = src.rows * src.cols - 4 * t;
    } else {
        const int64_t cch = (src.cols + 3) / 4;
        const int64_t r = t / cch;
        const int64_t c = (t - r * cch) * 4;
        p = src.x + r * src.ld + c;
        left = src.cols - c;
    }
    if (src.vec && left >= 4) {
        const float4 w = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
        ok[0] = ok[1] = ok[2] = ok[3] = true;
    } else {
        for (int e = 0; e < 4; ++e)
            if (e < left) { v[e] = __ldg(p + e); ok[e] = true; }
    }
}

// Block-wide digit pick (every thread of the block calls it; threads 0..RS_BINS-1 carry the
// counts).  Thread d holds cnt = count[d]; the digit d with excl(d) <= rank < excl(d) +
// count[d] lands in *s_digit and rank - excl(d) in *s_rank.  s_warp holds 8 words.
__device__ __forceinline__ void block_pick(unsigned long long cnt, long long rank, unsigned long long* s_warp,
                                           int* s_digit, long long* s_rank) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    unsigned long long incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (tid < RS_BINS && lane == 31) s_warp[w] = incl;
    if (tid == 0) {
        *s_digit = RS_BINS - 1;  // kept only for an out-of-range rank, which cannot occur
        *s_rank = rank;
    }
    __syncthreads();
    if (tid < RS_BINS) {
        unsigned long long base = 0;
        for (int k = 0; k < w; ++k) base += s_warp[k];
        const long long excl = (long long)(base + incl - cnt);
        if (cnt && rank >= excl && rank < excl + (long long)cnt) {
            *s_digit = tid;
            *s_rank = rank - excl;
        }
    }
    __syncthreads();
}

// True in every thread of the last block of the launch to reach this point (the block's
// global writes and atomics made before the call are then visible to it).
__device__ __forceinline__ bool last_block(unsigned int* arrived) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(arrived, 1u) == gridDim.x - 1);
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

__device__ __forceinline__ void state_init(SelectState* st, long long k1, long long k2) {
    for (int t = threadIdx.x; t < 2 * RS_BINS; t += blockDim.x) (&st->hist[0][0])[t] = 0ull;
    if (threadIdx.x == 0) {
        st->rank[0] = k1;
        st->rank[1] = k2;
        st->prefix[0] = st->prefix[1] = 0u;
        st->two = (k1 != k2);
        st->bits_done = 0;
        st->use_cand = 0;
        st->arrived = 0u;
        st->n_cand = 0ull;
        st->c_lo = 0ull;
        st->k1 = k1;
        st->k2 = k2;
    }
}

// Initialise the full-data state (ranks k1, k2) and, if given, the sample state.
__global__ void rs_init(SelectState* st, long long k1, long long k2, SelectState* sst, long long s1, long long s2) {
    state_init(st, k1, k2);
    if (sst) state_init(sst, s1, s2);
}

// Fixed-stride sample: entry (n / s) * k of the row-major order, k < s.
__global__ void rs_sample(SelSrc src, int64_t n, float* out) {
    const int64_t step = n / SAMPLE;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < SAMPLE; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = step * k;
        const int64_t r = t / src.cols, c = t - r * src.cols;
        out[k] = __ldg(src.x + r * src.ld + c);
    }
}

// Histogram of the next digit (the up to 8 key bits below the bits_done fixed ones) of the
// keys whose fixed bits match; the last block picks the digits.  Reads the candidate buffer
// when the state says so; does nothing once all 32 bits are fixed.  256 threads per block.
__global__ void __launch_bounds__(256) rs_hist(SelSrc src, SelectState* st) {
    const int hs = st->bits_done;
    if (hs >= 32) return;
    __shared__ unsigned int h[2][RS_BINS];
    __shared__ unsigned long long s_warp[8];
    __shared__ int s_digit;
    __shared__ long long s_rank;
    for (int t = threadIdx.x; t < 2 * RS_BINS; t += blockDim.x) (&h[0][0])[t] = 0u;
    __syncthreads();
    const int width = min(RS_BITS, 32 - hs);
    const int shift = 32 - hs - width;
    const uint32_t dmask = (1u << width) - 1u;
    const uint32_t p0 = st->prefix[0], p1 = st->prefix[1];
    const int two = st->two;
    auto add = [&](float f, bool valid) {
        const uint32_t k = fkey(f);
        const uint32_t hi = hs ? (k >> (32 - hs)) : 0u;
        const uint32_t d = (k >> shift) & dmask;
        if (valid && hi == p0) atomicAdd(&h[0][d], 1u);
        if (two && valid && hi == p1) atomicAdd(&h[1][d], 1u);
    };
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the candidate buffer is one aligned contiguous run of n_cand entries
    const SelSrc in = st->use_cand ? SelSrc{src.cand, 1, (int64_t)st->n_cand, (int64_t)st->n_cand, nullptr, 1, 1} : src;
    const int64_t n = n_chunks(in);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += stride) {
        float v[4];
        bool ok[4];
        load_chunk(in, t, n, v, ok);
#pragma unroll
        for (int e = 0; e < 4; ++e) add(v[e], ok[e]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < RS_BINS; t += blockDim.x) {
        if (h[0][t]) atomicAdd(&st->hist[0][t], (unsigned long long)h[0][t]);
        if (two && h[1][t]) atomicAdd(&st->hist[1][t], (unsigned long long)h[1][t]);
    }
    if (!last_block(&st->arrived)) return;
    // last block: pick the digit of each target, clear the histograms for the next pass
    for (int t = 0; t < 1 + two; ++t) {
        const unsigned long long cnt = __ldcg(&st->hist[t][threadIdx.x]);
        block_pick(cnt, st->rank[t], s_warp, &s_digit, &s_rank);
        if (threadIdx.x == 0) {
            st->rank[t] = s_rank;
            st->prefix[t] = (st->prefix[t] << width) | (uint32_t)s_digit;
        }
        __syncthreads();
    }
    st->hist[0][threadIdx.x] = 0ull;
    st->hist[1][threadIdx.x] = 0ull;
    if (threadIdx.x == 0) {
        st->bits_done = hs + width;
        st->arrived = 0u;
    }
}

// One pass over all entries: count those below lo, compact those in [lo, hi] (the first
// `cap` of them are stored; the count keeps going so that an overflow is seen); lo and hi
// are the values the sample state selected.  Each warp loads RS_UNROLL chunk groups before
// testing them, stages its candidates in shared memory and reserves space in the buffer
// once per GROUP or more of them.  The last block decides: candidates when they hold both
// target ranks (then the leading bits that lo and hi share, which all candidates share too,
// are fixed at once), else all entries.
static constexpr int RS_UNROLL = 4;
__global__ void __launch_bounds__(256) rs_count_compact(SelSrc src, const SelectState* sample_st, SelectState* st,
                                                        float* cand, unsigned long long cap) {
    constexpr int GROUP = 32 * RS_UNROLL * 4;  // entries a warp tests per iteration
    constexpr int STAGE = 2 * GROUP;
    __shared__ float s_stage[8][STAGE];
    __shared__ unsigned long long s_below[8];
    const uint32_t kl = sample_st->prefix[0], kh = sample_st->prefix[1];
    const float lo = fkey_inv(kl), hi = fkey_inv(kh);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* wb = s_stage[warp];
    unsigned fill = 0;  // warp-uniform
    unsigned long long below = 0;
    auto flush = [&]() {
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&st->n_cand, (unsigned long long)fill);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (unsigned i = lane; i < fill; i += 32)
            if (base + i < cap) cand[base + i] = wb[i];
        __syncwarp();
        fill = 0;
    };
    const int64_t n = n_chunks(src);
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // whole warps walk the chunk space together (the compaction uses warp ballots)
    for (int64_t t0 = gwarp * 32 * RS_UNROLL; t0 < n; t0 += nwarps * 32 * RS_UNROLL) {
        float v[RS_UNROLL][4];
        bool ok[RS_UNROLL][4];
#pragma unroll
        for (int u = 0; u < RS_UNROLL; ++u) load_chunk(src, t0 + 32 * u + lane, n, v[u], ok[u]);
#pragma unroll
        for (int u = 0; u < RS_UNROLL; ++u) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                below += (ok[u][e] && v[u][e] < lo) ? 1ull : 0ull;
                const bool in = ok[u][e] && v[u][e] >= lo && v[u][e] <= hi;
                const unsigned m = __ballot_sync(0xffffffffu, in);
                if (in) wb[fill + __popc(m & ((1u << lane) - 1u))] = v[u][e];
                fill += __popc(m);
            }
        }
        if (fill >= STAGE - GROUP) flush();  // keep room for one more iteration
    }
    if (fill) flush();
    for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
    if (lane == 0) s_below[warp] = below;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_below[w];
        atomicAdd(&st->c_lo, b);
    }
    if (!last_block(&st->arrived)) return;
    if (threadIdx.x == 0) {
        const long long c_lo = (long long)__ldcg(&st->c_lo);
        const long long nc = (long long)__ldcg(&st->n_cand);
        const long long a = st->k1 - c_lo, b = st->k2 - c_lo;
        const int ok = nc <= (long long)cap && a >= 0 && a < nc && b >= 0 && b < nc;
        st->use_cand = ok;
        st->rank[0] = ok ? a : st->k1;
        st->rank[1] = ok ? b : st->k2;
        const int common = ok ? __clz((int)(kl ^ kh)) : 0;  // 32 when lo == hi
        st->prefix[0] = st->prefix[1] = common == 0 ? 0u : (common == 32 ? kl : (kl >> (32 - common)));
        st->bits_done = common;
        st->arrived = 0u;
    }
}

__global__ void rs_finish(const SelectState* st, double* out) {
    if (threadIdx.x == 0) {
        const double a = (double)fkey_inv(st->prefix[0]);
        const double b = st->two ? (double)fkey_inv(st->prefix[1]) : a;
        *out = 0.5 * (a + b);
    }
}

ot_status launch_median(ot_assoc_ctx* ctx, const float* x, int64_t rows, int64_t cols, int64_t ld, double* out_dev,
                        cudaStream_t s) {
    ot_status st = OT_OK;
    const int64_t n = rows * cols;
    const long long k1 = (n - 1) / 2, k2 = n / 2;  // equal for odd n
    const int flat = (rows == 1 || ld == cols);
    const int vec = !((uintptr_t)x & 15u) && (flat || ld % 4 == 0);
    const SelSrc src0{x, rows, cols, ld, nullptr, vec, flat};
    const int64_t nch = n_chunks(src0);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nch + 255) / 256, 8LL * ctx->num_sms));
    const bool bracket = n >= 16 * SAMPLE;  // below that, four passes over the data cost little
    // the bracket spans about 2.3% of the entries; more than n/16 means heavy ties
    const unsigned long long cap = bracket ? (unsigned long long)(n / 16) : 0ull;
    const size_t off_sst = (size_t)round_up(sizeof(SelectState), 256);
    const size_t off_sample = off_sst + (size_t)round_up(sizeof(SelectState), 256);
    const size_t off_cand = off_sample + sizeof(float) * (size_t)SAMPLE;
    const size_t bytes = bracket ? off_cand + sizeof(float) * (size_t)cap : sizeof(SelectState);
    char* ws = (char*)scratch(ctx, SLOT_SELECT, bytes, &st);
    if (st) return st;
    SelectState* ss = (SelectState*)ws;
    SelSrc src = src0;
    int launches = 0;
    int hist_grid = grid;
    if (bracket) {
        SelectState* sst = (SelectState*)(ws + off_sst);
        float* sample = (float*)(ws + off_sample);
        float* cand = (float*)(ws + off_cand);
        const double sd = 0.5 * std::sqrt((double)SAMPLE);
        const long long slo = (long long)(SAMPLE / 2 - 6.0 * sd);
        const long long shi = (long long)(SAMPLE / 2 + 6.0 * sd);
        rs_init<<<1, 256, 0, s>>>(ss, k1, k2, sst, slo, shi);
        rs_sample<<<(int)(SAMPLE / 256), 256, 0, s>>>(src, n, sample);
        const SelSrc ssrc{sample, 1, SAMPLE, SAMPLE, nullptr, 1, 1};
        for (int pass = 0; pass < RS_PASSES; ++pass) rs_hist<<<(int)(SAMPLE / 1024), 256, 0, s>>>(ssrc, sst);
        rs_count_compact<<<grid, 256, 0, s>>>(src, sst, ss, cand, cap);
        src.cand = cand;
        // candidates are at most n/16 entries; the rare full-data fallback runs on this grid too
        hist_grid = std::max(1, std::min(grid, 2 * ctx->num_sms));
        launches += 3 + RS_PASSES;
    } else {
        rs_init<<<1, 256, 0, s>>>(ss, k1, k2, nullptr, 0, 0);
        ++launches;
    }
    for (int pass = 0; pass < RS_PASSES; ++pass) rs_hist<<<hist_grid, 256, 0, s>>>(src, ss);
    rs_finish<<<1, 32, 0, s>>>(ss, out_dev);
    launches += 1 + RS_PASSES;
    ctx->launches += launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(ctx, e, "median launch");
    return OT_OK;
}

}  // namespace ota
