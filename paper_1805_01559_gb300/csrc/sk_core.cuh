// Sinkhorn solver core shared by the single-instance and the batched persistent kernels
// (Algorithm 1 of the paper, Sec. III-B, in the log2-unit form described in k_sinkhorn.cu):
// constants, FP32-pair helpers, the row-streaming producer and the consumer warps' loop.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "ot_common.cuh"

namespace ota {

static constexpr int NT_F = 256;  // threads per CTA of the finalize kernel (row blocks)
static constexpr double LN2 = 0.69314718055994530942;
static constexpr double LOG2E = 1.44269504088896340736;

enum : int { DEV_ENUMERIC = -7 };

struct DevScalars {
    double sp, sq;  // sums of the caller's p and q
    double inv_sp, inv_sq;
    float inv_sp_f;
    int status;
};

// The loop test compares the FP32 residual of the plan with tol (1 - 2^-5).  That residual is
// formed from FP32 cell values (approximate ex2, one rounding at about |G| per exponent) and
// sits within about 1e-8 of the exact FP64 residual of the same potentials at tol = 1e-6 (it
// can be on either side); the 3% margin keeps the returned plan's exact residual <= tol.
__host__ __device__ __forceinline__ double stop_tol(double tol) { return tol * (1.0 - 0.03125); }

struct LoopState {
    unsigned bar;
    int status;
    int iters;
    int converged;
    double err;
};

// Column state of one solve in global memory (Jp a multiple of 4), in doubles:
//   [0, 2 Jp)       G^k (log2 units, FP64) in buffer k & 1 (the returned potentials)
//   [2 Jp, 3 Jp)    log2 q^_j (FP64)
//   [3 Jp, 4 Jp)    log2 q^_j as FP32 pairs
//   [4 Jp, 4.5 Jp)  fixed-point shift S_j of column j (int)
//   then 3 rows of Jp + 4 64-bit words: per-column fixed-point totals of a sweep's column
//   partials and its row residual (word Jp); sweep s adds into row s mod 3.
// The totals are sums of integers, the same in any order, so every CTA reads the same column
// sums whatever the number of CTAs or the order in which partitions arrive.
static constexpr int FX_BITS = 40;   // a column total of q^_j is about 2^40 units
static constexpr int FX_ERR = 50;    // row residuals in units of 2^-50
__host__ __device__ constexpr size_t gstate_words(int Jp) { return (size_t)Jp * 15 / 2 + 12; }
__host__ __device__ constexpr size_t gstate_bytes(int Jp) { return 8 * gstate_words(Jp); }
__device__ __forceinline__ float2* gs_lq2(double* G, int Jp) { return reinterpret_cast<float2*>(G + 3 * (size_t)Jp); }
__device__ __forceinline__ int* gs_sx(double* G, int Jp) { return reinterpret_cast<int*>(G + 4 * (size_t)Jp); }
__device__ __forceinline__ unsigned long long* gs_acc(double* G, int Jp) {
    return reinterpret_cast<unsigned long long*>(G + 4 * (size_t)Jp + Jp / 2);
}

template <int TW, int VPT>
__device__ __forceinline__ void load_G(const double* __restrict__ G, int J, int tl, float4 (&g)[VPT]) {
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int col = 4 * (tl + 32 * TW * v);
#pragma unroll
        for (int c = 0; c < 4; ++c) comp(g[v], c) = (col + c < J) ? (float)G[col + c] : 0.0f;
    }
}

// Cell exponent x = F + G - k C in log2 units, with F = F_hi + F_lo (FP32 pair) and
// k = k_hi + k_lo.  The exact FMA product cancels the large parts F_hi - C k_hi first, so
// the only roundings happen at the magnitude of |G| and |x|, however large k C and F are on
// the support.  k_lo > 0 always (see split_k): a +inf cost (masked column, forbidden link)
// gives -inf and never inf - inf.
__device__ __forceinline__ float expo(float F_hi, float F_lo_plus_G, float c, float k_hi, float k_lo) {
    return fmaf(-c, k_hi, F_hi) + fmaf(-c, k_lo, F_lo_plus_G);
}

// The same with the column potential as an FP32 pair G = G_hi + G_lo: F_hi - C k_hi (one
// rounding at about |G|) meets G_hi first, where the two nearly cancel on the cells that
// carry mass, and the low parts join at the magnitude of |x|.  No rounding of G itself enters
// the plan, so the plan the sweep measures is the plan of the FP64 potentials it returns.
__device__ __forceinline__ float expo2(float F_hi, float F_lo_plus_G_lo, float G_hi, float c, float k_hi,
                                       float k_lo) {
    return (fmaf(-c, k_hi, F_hi) + G_hi) + fmaf(-c, k_lo, F_lo_plus_G_lo);
}

// Error-free sum a + b = s + e (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) - d as a renormalised FP32 pair.
__device__ __forceinline__ float2 df_sub(float2 f, float d) {
    float s, e;
    two_sum(f.x, -d, s, e);
    e += f.y;
    float h, l;
    two_sum(s, e, h, l);
    return make_float2(h, l);
}

// k = k_hi + k_lo with k_hi rounded down and 0 < k_lo <= ulp(k_hi): the low part is never
// zero or negative, so -inf * k_lo = -inf and no inf - inf can occur for C = +inf.
static inline void split_k(double k, float* hi, float* lo) {
    float h = (float)k;
    if ((double)h >= k) h = nextafterf(h, 0.0f);
    float l = (float)(k - (double)h);
    if (!(l > 0.0f)) l = 1.4e-45f;  // smallest subnormal; adds nothing measurable
    *hi = h;
    *lo = l;
}

// ------------------------------------------------------------------------------------------
// Row streaming: one producer warp copies contiguous blocks of rows of C into a ring of
// shared-memory stages with bulk copies; the consumer warps work on them.
// ------------------------------------------------------------------------------------------
// Consumer warps per CTA.  A sub-partition of the SM holds 16K registers, so a block whose
// busiest sub-partition runs 4 warps gets 128 registers a thread, whether the block has 13
// warps or 16.  One-warp teams take the full 16 (15 consumers + the producer): the sweep is
// latency-bound, and 15 warps instead of 12 at the same 128 registers made the 50,000 x 800
// solves 10% faster.  Other team widths take the largest multiple of the width that still
// fits: 14 for teams of 2 (5% faster than 12 at 200,000 x 1,536), 12 for teams of 4, and 8
// when a row needs a team of 8 warps.
template <int TW>
struct Cons {
    static constexpr int NCW = (TW == 8) ? 8 : (TW == 1 ? 15 : (TW == 2 ? 14 : 12));
    static constexpr int NT = 32 * (NCW + 1);  // + one producer warp
};
static constexpr int MAX_STAGES = 8;
static constexpr int CONS_BAR = 15;          // named barrier of the consumer warps
static constexpr int SMEM_HDR = 256;         // mbarriers at the start of dynamic smem

struct StreamCfg {
    int rows_per_stage;  // NTEAMS * rpt
    int rpt;             // rows per team per stage
    int stages;
    int stage_floats;    // rows_per_stage * ld (elements of the streamed matrix)
    int rmax;            // most rows any CTA owns
    int off_G;           // byte offsets inside dynamic smem
    int off_F;
    int off_P;
    int off_ring;
};

// Column potentials as FP32 pairs in shared memory: high parts Gs[0, Jp), low parts
// Gs[Jp, 2 Jp) with G_j = hi + lo to about 2^-48 relative (padding columns 0).
__device__ __forceinline__ void load_G_smem(const double* __restrict__ G, int J, int Jp, float* Gs, int tid,
                                            int nthreads) {
    for (int j = tid; j < Jp; j += nthreads) {
        const double x = (j < J) ? G[j] : 0.0;
        const float hi = (float)x;
        Gs[j] = hi;
        Gs[Jp + j] = (float)(x - (double)hi);
    }
}

// log2(r) for the row and column corrections: a short series when r is within 2^-7 of 1
// (|u|^5/5 < 2^-37 relative to the result), the SFU logarithm otherwise.
__device__ __forceinline__ float log2_corr(float r) {
    const float u = r - 1.0f;  // exact for r in [0.5, 2]
    const float series = u * (1.0f + u * (-0.5f + u * (0.33333334f + u * -0.25f))) * 1.44269504f;
    const float sfu = __log2f(r);
    return fabsf(u) < 0.0078125f ? series : sfu;
}

// A lane's chunk v is certainly inside the row when the dispatch chose VPT = ceil(J4 / 32)
// for a one-warp team (pick_kernels does exactly that for TW = 1): then every chunk but the
// lane's last ends at or before column J.  Wider teams check every chunk.
template <int TW, int VPT>
__device__ __forceinline__ constexpr bool chunk_inside(int v) {
    return TW == 1 && v < VPT - 1;
}

// Row load from a shared-memory stage; chunks that can leave the row are checked.
template <int TW, int VPT>
__device__ __forceinline__ void load_row_smem(const float* row, int J, int tl, float4 (&x)[VPT]) {
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int col = 4 * (tl + 32 * TW * v);
        if (chunk_inside<TW, VPT>(v)) {
            x[v] = *reinterpret_cast<const float4*>(row + col);
        } else if (col < J) {
            float4 t = *reinterpret_cast<const float4*>(row + col);
            if (col + 4 > J) {
                if (col + 1 >= J) t.y = INFINITY;
                if (col + 2 >= J) t.z = INFINITY;
                if (col + 3 >= J) t.w = INFINITY;
            }
            x[v] = t;
        } else {
            x[v] = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
        }
    }
}

// Euclidean cost of four columns from coordinates: sqrt(dx^2 + dy^2) in FP32 with explicit
// roundings (no contraction), so any IEEE single-precision evaluation of the same formula
// gives the same values; columns at or past J give +inf (no mass).
__device__ __forceinline__ float4 euclid_chunk(float2 d, const float* rx, const float* ry, int col, int J) {
    float4 a = *reinterpret_cast<const float4*>(rx + col);
    float4 b = *reinterpret_cast<const float4*>(ry + col);
    float4 o;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float dx = __fsub_rn(d.x, comp(a, c));
        const float dy = __fsub_rn(d.y, comp(b, c));
        comp(o, c) = col + c < J ? __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy))) : INFINITY;
    }
    return o;
}
template <int TW, int VPT>
__device__ __forceinline__ void euclid_row(float2 d, const float* rx, const float* ry, int J, int tl, float4 (&x)[VPT]) {
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int col = 4 * (tl + 32 * TW * v);
        x[v] = col < J ? euclid_chunk(d, rx, ry, col, J) : make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
    }
}

// Producer: stream the CTA's row blocks sweep after sweep until the consumers raise s_stop,
// then wait for every copy still in flight before leaving.
template <typename T>
__device__ __forceinline__ void stream_rows_producer(const T* C, int64_t ld, int64_t r0, int64_t r1,
                                                     const StreamCfg& S, T* ring, uint64_t* full,
                                                     uint64_t* empty, volatile int* s_stop, int* status,
                                                     long long spin) {
    const int nblk = (int)((r1 - r0 + S.rows_per_stage - 1) / S.rows_per_stage);
    uint32_t seq = 0;
    bool stop = (nblk <= 0);
    while (!stop) {
        for (int k = 0; k < nblk && !stop; ++k) {
            const int st = (int)(seq % (uint32_t)S.stages);
            const uint32_t use = seq / (uint32_t)S.stages;
            if (use > 0) {  // wait for the consumers to release this stage's previous copy
                long long n = 0;
                while (!mbar_try_wait_sleep(&empty[st], (use - 1) & 1u, 500)) {
                    if (*s_stop) { stop = true; break; }
                    if ((++n & 1023) == 0 && ld_volatile_i32(status) != DEV_OK) { stop = true; break; }
                    if (n > spin) {
                        atomicCAS(status, DEV_OK, DEV_ETIMEOUT);
                        stop = true;
                        break;
                    }
                }
                if (stop) break;
            }
            if (*s_stop) { stop = true; break; }
            const int64_t row0 = r0 + (int64_t)k * S.rows_per_stage;
            const int rows = (int)min((int64_t)S.rows_per_stage, r1 - row0);
            const uint32_t bytes = (uint32_t)(rows * ld * (int64_t)sizeof(T));
            mbar_arrive_expect_tx(&full[st], bytes);
            bulk_g2s(ring + (size_t)st * S.stage_floats, C + row0 * ld, bytes, &full[st]);
            ++seq;
        }
    }
    // Leave no copy in flight: wait for the last use of every stage to land.  This wait has
    // its own limit (about a second), independent of the caller's spin limit: a copy that was
    // issued completes on its own, and the CTA must not leave while one can still land.
    const long long drain_limit = spin > (1LL << 20) ? spin : (1LL << 20);
    for (int st = 0; st < S.stages; ++st) {
        if (seq <= (uint32_t)st) continue;
        const uint32_t uses = (seq - (uint32_t)st + S.stages - 1) / (uint32_t)S.stages;
        long long n = 0;
        while (!mbar_try_wait_sleep(&full[st], (uses - 1) & 1u, 1000) && ++n <= drain_limit) {
        }
    }
}

struct SolveParams {
    const float* C;
    int64_t ld;
    int64_t I;
    int J;
    int Jp;
    int V;            // row partitions (see part_row): the unit of every cross-row reduction
    const float* p;
    const float* q;
    const double* g_warm;                 // warm-start g (natural units) or nullptr
    const unsigned long long* input_bad;  // nonzero => invalid rates upstream, or nullptr
    DevScalars* sc;
    LoopState* st;
    double* G;        // gstate_words(Jp): column potentials G^k (log2 units, FP64) in buffer
                      // k & 1, log2 q^_j, the fixed-point column totals (see gstate_words)
    float2* F_out;    // [I] row potentials of the returned plan (hi, lo), or nullptr
    float* colpart;   // [V][2 * Jp]
    double* errpart;  // [V] during setup (sums of p); reused as float2 [V] residual pairs
    double k;
    float k_hi, k_lo;
    double tol;
    int max_iter;
    long long spin;
    // Finalize sweep after the stop (skipped when fpart is null): column partials
    // (sum_i p^_i t_ij, sum_i p^_i C_ij t_ij) per partition in FP64, row residual per
    // partition, and optionally the plan pi_ij = p_i t_ij and the natural-unit row potentials.
    double2* fpart;   // [V][Jp]
    double* epart;    // [V]
    float* pi;        // [I][pi_ld] or nullptr
    int64_t pi_ld;
    double* f_nat;    // [I] f_i = eps ln2 (F'_i + log2 p_i), or nullptr
    double eps_ln2;
    // Finalize only (F_in not null): no iteration; the finalize sweep runs on the caller's
    // potentials F' (pairs) and G (log2 units).
    const float2* F_in;  // [I]
    const double* G_in;  // [Jp]
    // Euclidean cost formed on the fly (Sec. IV cost choice (i)) instead of read from C:
    // device and RRH coordinates; the RRH coordinates are staged in shared memory at the
    // ring's offset (x then y, Jp floats each).
    const float2* dev_xy;  // [I]
    const float2* rrh_xy;  // [J]
    // Iteration 1 only (the stored-kernel form starts from its potentials): F'^1 to F_out and
    // G^1 in G + Jp, no test sweep and no finalize.
    int init_only = 0;
};

// Row partitions.  The I rows form B = ceil(I / rs) stage blocks of rs rows; partition v of V
// is the run of blocks [B v / V, B (v + 1) / V).  Every sum over rows (column partials, row
// residuals, sums of p) is formed per partition, in a fixed order inside it, and partitions
// are combined in partition order, so the result does not depend on how many CTAs share the
// work: a CTA owns a contiguous run of partitions and walks them one after the other.
__host__ __device__ __forceinline__ int64_t part_row(int64_t I, int rs, int V, int v) {
    const int64_t B = (I + rs - 1) / rs;
    const int64_t r = (B * v / V) * rs;
    return r < I ? r : I;
}
__host__ __device__ __forceinline__ void cta_parts(int V, int b, int nb, int* v0, int* v1) {
    *v0 = (int)((int64_t)V * b / nb);
    *v1 = (int)((int64_t)V * (b + 1) / nb);
}
// Rows [r0, r1) of CTA b of nb.
__host__ __device__ __forceinline__ void cta_rows(int64_t I, int rs, int V, int b, int nb, int64_t* r0,
                                                  int64_t* r1) {
    int v0, v1;
    cta_parts(V, b, nb, &v0, &v1);
    *r0 = part_row(I, rs, V, v0);
    *r1 = part_row(I, rs, V, v1);
}
// Partitions of an instance: at most VMAX, at least one stage block and 64 rows each.
static constexpr int VMAX = 152;
__host__ __device__ __forceinline__ int parts_for(int64_t I, int rs) {
    const int64_t B = (I + rs - 1) / rs;
    int64_t v = I / 64;
    if (v > B) v = B;
    if (v > VMAX) v = VMAX;
    return v < 1 ? 1 : (int)v;
}

// Stage geometry and shared-memory layout of an instance solved by nb CTAs with teams of
// `nteams` rows (g_words floats per column at off_G: 2 for the FP32 pairs of G; f_bytes per
// row in each of the two row-potential buffers: an FP32 pair, or one float for the stored
// kernel's scalings).  The rows per stage depend only on the stage target and the row length,
// and the partitions only on I and the rows per stage: the arithmetic of a solve is fixed
// by (I, J, ld, stage target) whatever nb is.  Returns false when a CTA's rows do not fit
// next to two stages.
inline bool plan_stage(int nteams, int64_t I, int Jp, int64_t ld, int nb, int stage_target, size_t budget,
                       StreamCfg* S, size_t* smem, int* Vout, int esize = 4, int g_words = 2,
                       int f_bytes = (int)sizeof(float2), int comb_bufs = 0) {
    // comb_bufs: rows of Jp floats for merging the teams' column partials (0: half the teams)
    const size_t comb = (size_t)(comb_bufs > 0 ? comb_bufs : (nteams + 1) / 2) * Jp * sizeof(float);
    const size_t row_bytes = (size_t)ld * esize;
    const int rpt = (int)(stage_target / ((size_t)nteams * row_bytes) > 1 ? stage_target / ((size_t)nteams * row_bytes)
                                                                           : 1);
    const int rs = nteams * rpt;
    const int V = parts_for(I, rs);
    int64_t rmax = 0;
    for (int b = 0; b < nb; ++b) {
        int64_t r0, r1;
        cta_rows(I, rs, V, b, nb, &r0, &r1);
        rmax = r1 - r0 > rmax ? r1 - r0 : rmax;
    }
    auto up = [](size_t x, size_t m) { return (x + m - 1) / m * m; };
    const size_t off_G = up(SMEM_HDR + comb, 16);
    const size_t off_F = up(off_G + (size_t)g_words * Jp * sizeof(float), 16);  // G pairs: hi, then lo
    const size_t off_P = up(off_F + (size_t)2 * rmax * f_bytes, 16);  // two row-potential buffers
    const size_t off_ring = up(off_P + (size_t)rmax * sizeof(float), 128);
    const size_t stage = (size_t)rs * row_bytes;
    const size_t room = off_ring < budget ? (budget - off_ring) / stage : 0;
    const int stages = (int)(room < (size_t)MAX_STAGES ? room : (size_t)MAX_STAGES);
    if (stages < 2) return false;
    S->rpt = rpt;
    S->rows_per_stage = rs;
    S->stages = stages;
    S->stage_floats = (int)(stage / esize);
    S->rmax = (int)(rmax > 0 ? rmax : 1);
    S->off_G = (int)off_G;
    S->off_F = (int)off_F;
    S->off_P = (int)off_P;
    S->off_ring = (int)off_ring;
    *smem = off_ring + (size_t)stages * stage;
    *Vout = V;
    return true;
}

// Sum of (s, e) pairs over a warp with error-free additions.
__device__ __forceinline__ void warp_sum_pair(float& s, float& e) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
        float t, u;
        two_sum(s, s2, t, u);
        s = t;
        e = e + e2 + u;
    }
}

// Shared-memory words of the consumer warps (and the producer's stop flag).
struct SkShared {
    float red[64];          // team reductions: 2 * NTEAMS * TW <= 24 values (float2 pairs: 48 floats)
    float errf[16];         // per-team row residuals
    double sh_sum[24][2];   // per-warp setup sums (up to 24 consumer warps)
    int s_dec, s_ok, s_bad;
    volatile int s_stop;    // consumers -> producer: stop streaming
    int pend[VMAX + 1];     // stage blocks (from the CTA's first row) at which its partitions end
};

// The CTAs that solve one instance together: nb CTAs, this one is number b.  `bar` counts
// arrivals at the group's barriers (monotonic; every CTA of the group passes the same
// barriers, `gen` of them so far).  A nonzero *abort ends every wait; *status is the
// instance's status word (the same word as *abort for a single-instance launch).
struct GroupCtx {
    int nb, b;
    unsigned* bar;
    unsigned gen;
    int* abort;
    int* status;
};

// Team sum of per-lane FP32 values as an error-free (hi, lo) pair; `red` holds 4 * NTEAMS * TW
// floats, the halves alternating by `par` as in team_reduce.
template <int TW>
__device__ __forceinline__ float2 team_sum_pair(float s, float* red, int nteams, const Team<TW>& tm, int& par) {
    float e = 0.f;
    warp_sum_pair(s, e);
    if constexpr (TW == 1) {
        return make_float2(s, e);
    } else {
        float2* r = reinterpret_cast<float2*>(red) + (par * nteams + tm.team) * TW;
        if (tm.lane == 0) r[tm.wit] = make_float2(s, e);
        bar_named(1 + tm.team, 32 * TW);
        float2 a = r[0];
#pragma unroll
        for (int w = 1; w < TW; ++w) a = df_add2(a, r[w]);
        par ^= 1;
        return a;
    }
}

// Sum of the teams' float4 column partials acc (in team order: the first half of the teams
// stores, the second half adds onto slot team - HALF, then the HALF slots are summed in
// order); f(j, sum) receives column j's total.  Named barriers over the consumer warps; the
// comb buffer (HALF rows of Jp floats) is free again when it returns.
template <int TW, int VPT, typename Fn>
__device__ __forceinline__ void cta_col_sum(float* comb, const float4 (&acc)[VPT], int J, int Jp, const Team<TW>& tm,
                                            Fn f) {
    constexpr int NCW = Cons<TW>::NCW;
    constexpr int TT = 32 * TW, NTEAMS = NCW / TW, NC = NCW * 32;
    constexpr int HALF = (NTEAMS + 1) / 2;
    if (tm.team < HALF) {
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int col = 4 * (tm.tl + TT * v);
            if (col < Jp) *reinterpret_cast<float4*>(comb + tm.team * Jp + col) = acc[v];
        }
    }
    bar_named(CONS_BAR, NC);
    if (tm.team >= HALF) {
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int col = 4 * (tm.tl + TT * v);
            if (col < Jp) {
                float4* d = reinterpret_cast<float4*>(comb + (tm.team - HALF) * Jp + col);
                float4 o = *d;
                o.x += acc[v].x;
                o.y += acc[v].y;
                o.z += acc[v].z;
                o.w += acc[v].w;
                *d = o;
            }
        }
    }
    bar_named(CONS_BAR, NC);
    for (int j = threadIdx.x; j < J; j += NC) {
        float sum = comb[j];
        for (int t = 1; t < HALF; ++t) sum += comb[t * Jp + j];
        f(j, sum);
    }
    bar_named(CONS_BAR, NC);
}

// Finalize sweep of the consumer warps, run right after the loop stops: the producer has
// already streamed the next pass over the CTA's rows into the ring, so this is one more
// sweep at streaming speed.  Plan of the returned potentials F' (Fold) and G (Gs, still the
// returned plan's column potentials): t_ij = 2^(F'_i + G_j - k C_ij).  Each team keeps FP32
// column sums of p^ t and p^ C t over at most FIN_ROWS rows, then the CTA adds the teams'
// sums (in team order) into the partition's FP64 partials P.fpart[v]; the row residual
// sum_i p^_i |sum_j t_ij - 1| uses error-free row sums.
static constexpr int FIN_ROWS = 16;
template <int TW, int VPT, bool EUC = false>
__device__ __forceinline__ void sk_finalize_sweep(const SolveParams& P, const StreamCfg& S, SkShared* sh,
                                                  unsigned char* dyn, int64_t r0, int nrow, int v0, int v1,
                                                  const float2* Fold, uint32_t& cseq, int* abort) {
    constexpr int NCW = Cons<TW>::NCW;
    constexpr int TT = 32 * TW, NTEAMS = NCW / TW, NC = NCW * 32;
    uint64_t* full = reinterpret_cast<uint64_t*>(dyn);
    uint64_t* empty = full + MAX_STAGES;
    float* comb = reinterpret_cast<float*>(dyn + SMEM_HDR);
    const float* Gs = reinterpret_cast<const float*>(dyn + S.off_G);
    const float* Ps = reinterpret_cast<const float*>(dyn + S.off_P);
    const float* ring = reinterpret_cast<const float*>(dyn + S.off_ring);
    const float* rx = ring;  // Euclidean cost: RRH x then y coordinates
    const int tid = threadIdx.x, lane = tid & 31;
    const int J = P.J, Jp = P.Jp, rs_ = S.rows_per_stage;
    const Team<TW> tm;
    int par = 0;
    for (int v = v0; v < v1; ++v)
        for (int j = tid; j < J; j += NC) P.fpart[(int64_t)v * Jp + j] = make_double2(0.0, 0.0);
    float4 cpi[VPT], crho[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) cpi[v] = crho[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    float errt = 0.f;
    const int nblk = (nrow + rs_ - 1) / rs_;
    const bool want_pi = P.pi != nullptr;
    const int every = max(1, FIN_ROWS / S.rpt);  // stages between flushes
    // Multi-warp teams: a row's sum is reduced within each warp (shuffles only) and the warps'
    // pairs wait in the merge buffer with p^_i; one thread per team combines them, row by row
    // in the same order and arithmetic as a per-row team sum, at the next flush (where the CTA
    // synchronises anyway) instead of a team barrier on every row.
    constexpr int HALF = (NTEAMS + 1) / 2;  // rows of Jp floats in the merge buffer
    const int wrows = every * S.rpt;        // rows a team sees between two flushes
    const bool defer = TW > 1 && (int64_t)wrows * NTEAMS * (2 * TW + 1) <= (int64_t)HALF * Jp;
    float2* wpair = reinterpret_cast<float2*>(comb);                       // [NTEAMS][wrows][TW]
    float* wph = comb + 2 * (size_t)NTEAMS * wrows * TW;                   // [NTEAMS][wrows]
    int wr = 0;
    const int* pend = sh->pend - v0;
    int vp = v0, vbeg = 0;
    int vend = v0 < v1 ? pend[v0] : 0;
    for (int kb = 0; kb < nblk; ++kb) {
        const int st = (int)(cseq % (uint32_t)S.stages);
        const uint32_t ph = (cseq / (uint32_t)S.stages) & 1u;
        const bool ok = EUC || mbar_try_wait(&full[st], ph) || mbar_wait_bounded(&full[st], ph, P.spin, abort);
        const int lr0 = kb * rs_;
        const int rows = min(rs_, nrow - lr0);
        const float* stage = ring + (size_t)st * S.stage_floats;
        for (int jr = 0; ok && jr < S.rpt; ++jr) {
            const int rr = tm.team + NTEAMS * jr;
            if (rr >= rows) break;
            const int lr = lr0 + rr;
            const float* row = stage + (size_t)rr * P.ld;
            const float2 dxy = EUC ? __ldg(P.dev_xy + r0 + lr) : make_float2(0.f, 0.f);
            const float2 F = Fold[lr];
            const float phat = Ps[lr];
            const int64_t i = r0 + lr;
            const float pf = want_pi ? __ldg(P.p + i) : 0.f;
            float rsum = 0.f;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int col = 4 * (tm.tl + TT * v);
                if (chunk_inside<TW, VPT>(v) || col < J) {
                    float4 x = EUC ? euclid_chunk(dxy, rx, rx + Jp, col, J) : *reinterpret_cast<const float4*>(row + col);
                    float4 gv = *reinterpret_cast<const float4*>(Gs + col);
                    float4 gl = *reinterpret_cast<const float4*>(Gs + Jp + col);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float cost = comp(x, c);
                        float t = ex2(expo2(F.x, F.y + comp(gl, c), comp(gv, c), cost, P.k_hi, P.k_lo));
                        if (!chunk_inside<TW, VPT>(v) && col + c >= J) t = 0.f;  // past the row
                        rsum += t;
                        comp(cpi[v], c) = fmaf(phat, t, comp(cpi[v], c));
                        comp(crho[v], c) = fmaf(phat, t > 0.f ? cost * t : 0.f, comp(crho[v], c));
                        comp(x, c) = t;
                    }
                    if (want_pi)  // one uniform branch per chunk, not per cell
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (col + c < J) P.pi[i * P.pi_ld + col + c] = pf * comp(x, c);
                }
            }
            if (defer) {
                float e = 0.f;
                warp_sum_pair(rsum, e);
                if (tm.lane == 0) wpair[((size_t)tm.team * wrows + wr) * TW + tm.wit] = make_float2(rsum, e);
                if (tm.tl == 0) wph[tm.team * wrows + wr] = phat;
                ++wr;
            } else {
                const float2 r = team_sum_pair<TW>(rsum, sh->red, NTEAMS, tm, par);
                errt = fmaf(phat, fabsf((r.x - 1.0f) + r.y), errt);
            }
        }
        __syncwarp();
        if (!EUC && lane == 0) mbar_arrive(&empty[st]);
        ++cseq;
        const bool at_end = (kb + 1 == vend);
        if ((kb + 1 - vbeg) % every == 0 || at_end) {
            if (defer) {
                bar_named(CONS_BAR, NC);  // every warp's parked row pairs are visible
                if (tm.tl == 0)
                    for (int k = 0; k < wr; ++k) {
                        const float2* r = wpair + ((size_t)tm.team * wrows + k) * TW;
                        float2 a = r[0];
#pragma unroll
                        for (int w = 1; w < TW; ++w) a = df_add2(a, r[w]);
                        errt = fmaf(wph[tm.team * wrows + k], fabsf((a.x - 1.0f) + a.y), errt);
                    }
                wr = 0;
                bar_named(CONS_BAR, NC);  // the merge buffer is free for the column sums
            }
            // Wide rows (multi-warp teams): reductions without a returned value.  The thread that
            // zeroed fp[j] is the one that adds to it, flush after flush, so the sums are the
            // serial ones, bit for bit, but no thread waits on L2 for the old value (at 4,096
            // columns a read-modify-write per column cost 0.2 ms of a 2.2 ms finalize).  One-warp
            // teams keep the read-modify-write: there the flushes are rare, and the reductions
            // changed the register allocation of the whole solver loop (1.5% slower at 800
            // columns).
            double2* fp = P.fpart + (int64_t)vp * Jp;
            if constexpr (TW > 1) {
                cta_col_sum<TW, VPT>(comb, cpi, J, Jp, tm, [&](int j, float sum) { atomicAdd(&fp[j].x, (double)sum); });
                cta_col_sum<TW, VPT>(comb, crho, J, Jp, tm, [&](int j, float sum) { atomicAdd(&fp[j].y, (double)sum); });
            } else {
                cta_col_sum<TW, VPT>(comb, cpi, J, Jp, tm, [&](int j, float sum) { fp[j].x += (double)sum; });
                cta_col_sum<TW, VPT>(comb, crho, J, Jp, tm, [&](int j, float sum) { fp[j].y += (double)sum; });
            }
#pragma unroll
            for (int v = 0; v < VPT; ++v) cpi[v] = crho[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (at_end) {
            if (tm.tl == 0) sh->errf[tm.team] = errt;
            bar_named(CONS_BAR, NC);
            if (tid == 0) {
                float2 e = make_float2(sh->errf[0], 0.f);
                for (int t = 1; t < NTEAMS; ++t) e = df_add(e, sh->errf[t]);
                P.epart[vp] = (double)e.x + (double)e.y;
            }
            bar_named(CONS_BAR, NC);
            errt = 0.f;
            ++vp;
            vbeg = kb + 1;
            if (vp < v1) vend = pend[vp];
        }
    }
    // natural-unit row potentials, one row per thread (an FP64 log2 each, off the sweep)
    if (P.f_nat)
        for (int r = tid; r < nrow; r += NC) {
            const float2 F = Fold[r];
            P.f_nat[r0 + r] = P.eps_ln2 * ((double)F.x + (double)F.y + log2((double)__ldg(P.p + r0 + r)));
        }
}

// The consumer warps' part of one solve (Algorithm 1 on the CTA's partitions, rows [r0, r1)):
// setup, the exact first sweep, then plan-scale sweeps until the loop test stops.  Returns
// true when the loop stopped normally (the returned plan's row potentials are then in row
// potential buffer *ret_par of shared memory, and in P.F_out when given), false when the
// instance failed or a wait gave up.  Either way s_stop is raised for the producer.
// Every decision that ends the loop is taken identically by every CTA of the group.
template <int TW, int VPT, bool EUC = false>
__device__ __forceinline__ bool sk_consumers(const SolveParams& P, const StreamCfg& S, GroupCtx& g, SkShared* sh,
                                             unsigned char* dyn, int64_t r0, int64_t r1, int* ret_par) {
    constexpr int NCW = Cons<TW>::NCW;
    constexpr int TT = 32 * TW, NTEAMS = NCW / TW, NC = NCW * 32;
    constexpr int HALF = (NTEAMS + 1) / 2;
    static_assert(4 * NTEAMS * TW <= 64 && NTEAMS <= 16 && NCW <= 16, "SkShared sizes");
    uint64_t* full = reinterpret_cast<uint64_t*>(dyn);
    uint64_t* empty = full + MAX_STAGES;
    float* comb = reinterpret_cast<float*>(dyn + SMEM_HDR);    // [ceil(NTEAMS / 2)][Jp]
    float* Gs = reinterpret_cast<float*>(dyn + S.off_G);       // [2][Jp]: G pairs (hi, lo)
    float2* Fs = reinterpret_cast<float2*>(dyn + S.off_F);     // [2][rmax]
    float* Ps = reinterpret_cast<float*>(dyn + S.off_P);       // [rmax]
    float* ring = reinterpret_cast<float*>(dyn + S.off_ring);  // [stages][stage_floats]
    const float* rxs = ring;  // Euclidean cost: RRH x then y coordinates [2][Jp]
    float* red = sh->red;
    float* errf = sh->errf;
    double(*sh_sum)[2] = sh->sh_sum;
    int& s_bad = sh->s_bad;
    volatile int& s_stop = sh->s_stop;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = g.nb, b = g.b;
    const int V = P.V, rs_ = S.rows_per_stage;
    int v0, v1;
    cta_parts(V, b, nb, &v0, &v1);
    const int nrow = (int)max((int64_t)0, r1 - r0);
    int* status = g.status;
    const int J = P.J, Jp = P.Jp;
    const int tid = threadIdx.x;
    // stage blocks (from the CTA's first row) at which each of the CTA's partitions ends
    for (int v = v0 + tid; v < v1; v += NC) sh->pend[v - v0] = (int)((part_row(P.I, rs_, V, v + 1) - r0 + rs_ - 1) / rs_);
    const int* pend = sh->pend - v0;
#define OTA_BARRIER()                                                                              \
    do {                                                                                           \
        if (!grid_barrier_named(g.bar, (unsigned)nb * ++g.gen, g.abort, P.spin, CONS_BAR, NC, &sh->s_ok)) { \
            if (tid == 0) s_stop = 1;                                                              \
            return false;                                                                          \
        }                                                                                          \
    } while (0)
// After a barrier that no status write can overtake (the next write comes after the next
// barrier): leave when the instance failed.  Only needed when a failed instance does not
// also end every wait (batched launches keep the abort word apart from instance status).
#define OTA_BARRIER_CHECK()                                                                        \
    do {                                                                                           \
        OTA_BARRIER();                                                                             \
        if (g.abort != status && ld_volatile_i32(status) != DEV_OK) {                              \
            if (tid == 0) s_stop = 1;                                                              \
            return false;                                                                          \
        }                                                                                          \
    } while (0)

    // ---- setup: sums of p (per partition) and q (every CTA), checks, starting G ----------
    {
        int bad = 0;
        for (int v = v0; v < v1; ++v) {
            const int a = (int)(part_row(P.I, rs_, V, v) - r0), e = (int)(part_row(P.I, rs_, V, v + 1) - r0);
            double sp = 0.0;
            for (int r = a + tid; r < e; r += NC) {
                const float x = __ldg(P.p + r0 + r);
                bad |= !(x > 0.0f) || !isfinite(x);
                sp += (double)x;
                Ps[r] = x;
            }
            sp = warp_sum(sp);
            if (lane == 0) sh_sum[warp][0] = sp;
            bar_named(CONS_BAR, NC);
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < NCW; ++w) t += sh_sum[w][0];
                P.errpart[v] = t;
            }
            bar_named(CONS_BAR, NC);
        }
        const int gw = b * NCW + warp, nw = nb * NCW;
        for (int j = gw * 32 + lane; j < J; j += nw * 32) {
            const double g0 = P.g_warm ? P.g_warm[j] * P.k : 0.0;
            bad |= !isfinite(g0);
            P.G[j] = g0;
        }
        if (b == 0 && tid == 0 && P.input_bad && *P.input_bad) bad = 1;
        if (bad) atomicOr(&s_bad, 1);
        bar_named(CONS_BAR, NC);
        if (tid == 0 && s_bad) atomicCAS(status, DEV_OK, DEV_EINVAL);
    }
    OTA_BARRIER_CHECK();
    double sp = 0.0, sq = 0.0;
    {
        // every CTA forms the same totals in the same order
        double a = 0.0, c = 0.0;
        int badq = 0;
        for (int bb = tid; bb < V; bb += NC) a += P.errpart[bb];
        for (int j = tid; j < J; j += NC) {
            const float x = __ldcg(P.q + j);
            badq |= !(x > 0.0f) || !isfinite(x);
            c += (double)x;
        }
        a = warp_sum(a);
        c = warp_sum(c);
        if (tid == 0) s_bad = 0;
        bar_named(CONS_BAR, NC);
        if (lane == 0) {
            sh_sum[warp][0] = a;
            sh_sum[warp][1] = c;
        }
        if (badq) atomicOr(&s_bad, 1);
        bar_named(CONS_BAR, NC);
        for (int w = 0; w < NCW; ++w) {
            sp += sh_sum[w][0];
            sq += sh_sum[w][1];
        }
        if (s_bad || !(fabs(sp - sq) <= 1e-5 * sp)) {
            if (b == 0 && tid == 0) atomicCAS(status, DEV_OK, DEV_EINVAL);
            if (tid == 0) s_stop = 1;
            return false;  // the same decision in every CTA
        }
        if (b == 0 && tid == 0) {
            P.sc->sp = sp;
            P.sc->sq = sq;
            P.sc->inv_sp = 1.0 / sp;
            P.sc->inv_sq = 1.0 / sq;
            P.sc->inv_sp_f = (float)(1.0 / sp);
            P.sc->status = DEV_OK;
        }
    }
    const double inv_sq = 1.0 / sq;
    double* LQ = P.G + 2 * Jp;  // log2 q^_j, formed once here (read after the next grid barrier)
    float2* LQ2 = gs_lq2(P.G, Jp);
    int* SX = gs_sx(P.G, Jp);
    unsigned long long* ACC = gs_acc(P.G, Jp);
    {
        const int gw = b * NCW + warp, nw = nb * NCW;
        for (int j = gw * 32 + lane; j < J; j += nw * 32) {
            const double lq = log2((double)__ldcg(P.q + j) * inv_sq);
            LQ[j] = lq;
            const float hi = (float)lq;
            LQ2[j] = make_float2(hi, (float)(lq - (double)hi));
            // the total of column j is about 2^FX_BITS when its sum is q^_j; shifts that the
            // FP32 scale cannot carry send the column to the exact path (shift 0 = "never")
            const int sx = FX_BITS - (int)floor(lq);
            SX[j] = sx <= 126 ? sx : 0;
        }
        for (int t = (b * NCW + warp) * 32 + lane; t < 3 * (Jp + 4); t += nw * 32) ACC[t] = 0ull;
        const float inv_sp_f = (float)(1.0 / sp);
        for (int r = tid; r < nrow; r += NC) Ps[r] *= inv_sp_f;  // p^_i
        bar_named(CONS_BAR, NC);
    }
    const Team<TW> tm;
    uint32_t cseq = 0;
    if (P.F_in) {  // finalize only
        for (int r = tid; r < nrow; r += NC) Fs[r] = P.F_in[r0 + r];
        load_G_smem(P.G_in, J, Jp, Gs, tid, NC);
        bar_named(CONS_BAR, NC);
        *ret_par = 0;
        sk_finalize_sweep<TW, VPT, EUC>(P, S, sh, dyn, r0, nrow, v0, v1, Fs, cseq, g.abort);
        if (tid == 0) s_stop = 1;
        return true;
    }
    load_G_smem(P.G, J, Jp, Gs, tid, NC);
    bar_named(CONS_BAR, NC);
    int par = 0;

    // ---- sweep 1: the log-domain iteration from G^0 with a fixed column scale --------------
    // Every row of the half-step plan is normalised (t_ij = pi_ij / p_i <= 1 after the row
    // shift), so the column sums of p^_i t_ij 2^64 cannot overflow: one ex2 a cell, like the
    // later sweeps.  A column whose scaled sum falls below 2^-60 (a true sum below 2^-124) is
    // marked, and then the whole first iteration is taken again in the exact form below (an
    // online (max, sum) pair per column) on the next pass of the stream.
    unsigned long long* flag1 = ACC + Jp + 1;  // zeroed with the totals in setup
    bool exact1 = false;
    {
        float4 acc[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        float2* F1 = Fs + S.rmax;  // F'^1 lives in buffer 1
        int kb = 0;
        for (int vp = v0; vp < v1; ++vp) {
            const int vend = pend[vp];
            for (; kb < vend; ++kb) {
                const int st = (int)(cseq % (uint32_t)S.stages);
                const uint32_t ph = (cseq / (uint32_t)S.stages) & 1u;
                const bool ok = EUC || mbar_try_wait(&full[st], ph) || mbar_wait_bounded(&full[st], ph, P.spin, g.abort);
                const int lr0 = kb * rs_;
                const int rows = min(rs_, nrow - lr0);
                const float* stage = ring + (size_t)st * S.stage_floats;
                for (int j = 0; ok && j < S.rpt; ++j) {
                    const int rr = tm.team + NTEAMS * j;
                    if (rr >= rows) break;
                    float4 x[VPT];
                    if constexpr (EUC)
                        euclid_row<TW, VPT>(__ldg(P.dev_xy + r0 + lr0 + rr), rxs, rxs + Jp, J, tm.tl, x);
                    else
                        load_row_smem<TW, VPT>(stage + (size_t)rr * P.ld, J, tm.tl, x);
                    float m = -INFINITY;  // row maximum of G^0 - k C (approximate: only a shift)
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        const int col = 4 * (tm.tl + TT * v);
                        float4 gv = col < Jp ? *reinterpret_cast<const float4*>(Gs + col) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int c = 0; c < 4; ++c) m = fmaxf(m, fmaf(-comp(x[v], c), P.k_hi, comp(gv, c)));
                    }
                    m = team_reduce<TW, float, true>(m, red, NTEAMS, tm, par);
                    float sum = 0.f;
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        const int col = 4 * (tm.tl + TT * v);
                        float4 gv = col < Jp ? *reinterpret_cast<const float4*>(Gs + col) : make_float4(0.f, 0.f, 0.f, 0.f);
                        float4 gl = col < Jp ? *reinterpret_cast<const float4*>(Gs + Jp + col) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float t = ex2(expo2(-m, comp(gl, c), comp(gv, c), comp(x[v], c), P.k_hi, P.k_lo));
                            comp(x[v], c) = t;
                            sum += t;
                        }
                    }
                    sum = team_reduce<TW, float, false>(sum, red, NTEAMS, tm, par);
                    const float ls = log2f(sum);
                    if (tm.tl == 0) {  // F'^1 = -LSE2_j(y) = -(m + log2 sum), exact as an FP32 pair
                        float hi, lo;
                        two_sum(m, ls, hi, lo);
                        F1[lr0 + rr] = make_float2(-hi, -lo);
                    }
                    const float w = __fdividef(Ps[lr0 + rr], sum) * 0x1p64f;  // p^_i 2^64 / sum
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        acc[v].x = fmaf(x[v].x, w, acc[v].x);
                        acc[v].y = fmaf(x[v].y, w, acc[v].y);
                        acc[v].z = fmaf(x[v].z, w, acc[v].z);
                        acc[v].w = fmaf(x[v].w, w, acc[v].w);
                    }
                }
                __syncwarp();
                if (!EUC && lane == 0) mbar_arrive(&empty[st]);
                ++cseq;
            }
            float* cp = P.colpart + (int64_t)vp * Jp;
            cta_col_sum<TW, VPT>(comb, acc, J, Jp, tm, [&](int j, float sum) { cp[j] = sum; });
#pragma unroll
            for (int v = 0; v < VPT; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        OTA_BARRIER();
        // G^1_j = G^0_j + log2 q^_j - log2(column sum of pi^(1/2)), one warp per column
        {
            const int gw = b * NCW + warp, nw = nb * NCW;
            for (int j = gw; j < J; j += nw) {
                float2 sum = make_float2(0.f, 0.f);
                for (int bb = lane; bb < V; bb += 32) sum = df_add(sum, P.colpart[(int64_t)bb * Jp + j]);
                sum = warp_sum_df(sum);
                if (lane == 0) {
                    if (!(sum.x >= 0x1p-60f) || !isfinite(sum.x)) {
                        atomicOr(flag1, 1ull);
                    } else {
                        const float2 ls = df_log2(sum);
                        P.G[Jp + j] = P.G[j] + LQ[j] - (((double)ls.x - 64.0) + (double)ls.y);
                    }
                }
            }
        }
        OTA_BARRIER_CHECK();
        exact1 = __ldcg(flag1) != 0ull;
        if (!exact1) {
            load_G_smem(P.G + Jp, J, Jp, Gs, tid, NC);
            bar_named(CONS_BAR, NC);
        }
    }
    // ---- sweep 1 again, exact log-domain form (a column sum below the fixed scale's range) --
    if (exact1) {
        float4 M[VPT], Sm[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            M[v] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
            Sm[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float2* F1 = Fs + S.rmax;  // F'^1 lives in buffer 1
        float2* part2 = reinterpret_cast<float2*>(P.colpart);
        int kb = 0;
        for (int vp = v0; vp < v1; ++vp) {
          const int vend = pend[vp];
          for (; kb < vend; ++kb) {
            const int st = (int)(cseq % (uint32_t)S.stages);
            const uint32_t ph = (cseq / (uint32_t)S.stages) & 1u;
            const bool ok = EUC || mbar_try_wait(&full[st], ph) || mbar_wait_bounded(&full[st], ph, P.spin, g.abort);
            const int lr0 = kb * rs_;
            const int rows = min(rs_, nrow - lr0);
            const float* stage = ring + (size_t)st * S.stage_floats;
            for (int j = 0; ok && j < S.rpt; ++j) {
                const int rr = tm.team + NTEAMS * j;
                if (rr >= rows) break;
                float4 x[VPT];
                if constexpr (EUC)
                    euclid_row<TW, VPT>(__ldg(P.dev_xy + r0 + lr0 + rr), rxs, rxs + Jp, J, tm.tl, x);
                else
                    load_row_smem<TW, VPT>(stage + (size_t)rr * P.ld, J, tm.tl, x);
                // row maximum of y = G0 - k C (approximate values suffice for the shift)
                float m = -INFINITY;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const int col = 4 * (tm.tl + TT * v);
                    float4 gv = col < Jp ? *reinterpret_cast<const float4*>(Gs + col) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < 4; ++c) m = fmaxf(m, fmaf(-comp(x[v], c), P.k_hi, comp(gv, c)));
                }
                m = team_reduce<TW, float, true>(m, red, NTEAMS, tm, par);
                // z = y - m with the large parts cancelled by the exact product
                float s = 0.f;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const int col = 4 * (tm.tl + TT * v);
                    float4 gv = col < Jp ? *reinterpret_cast<const float4*>(Gs + col) : make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 gl = col < Jp ? *reinterpret_cast<const float4*>(Gs + Jp + col) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float z = expo2(-m, comp(gl, c), comp(gv, c), comp(x[v], c), P.k_hi, P.k_lo);
                        comp(x[v], c) = z;
                        s += ex2(z);
                    }
                }
                s = team_reduce<TW, float, false>(s, red, NTEAMS, tm, par);
                const float ls = log2f(s);
                if (tm.tl == 0) {  // F'^1 = -LSE2_j(y) = -(m + log2 s), exact as an FP32 pair
                    float hi, lo;
                    two_sum(m, ls, hi, lo);
                    F1[lr0 + rr] = make_float2(-hi, -lo);
                }
                const float cst = log2f(Ps[lr0 + rr]) - ls;
#pragma unroll
                for (int v = 0; v < VPT; ++v)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        // online (max, sum) of log2 pi^(1/2)_ij, without a branch: a divergent
                        // branch per cell costs more than the second ex2.  The floor keeps
                        // -inf - -inf (a column no row reaches yet) out of the exponent.
                        const float u = comp(x[v], c) + cst;
                        float& Mc = comp(M[v], c);
                        float& Sc = comp(Sm[v], c);
                        const float mn = fmaxf(fmaxf(Mc, u), -1e30f);
                        Sc = fmaf(Sc, ex2(Mc - mn), ex2(u - mn));
                        Mc = mn;
                    }
            }
            __syncwarp();
            if (!EUC && lane == 0) mbar_arrive(&empty[st]);
            ++cseq;
          }
            // end of partition vp: merge the teams' (max, sum) pairs in two rounds through
            // the float buffer, the column maxima first (held in Gs meanwhile), then the sums
            // rescaled to them; teams in a fixed order.  Gs gets G^0 back afterwards.
            for (int round = 0; round < 2; ++round) {  // the first half stores, the second half merges
                if ((tm.team < HALF) == (round == 0)) {
                    const int slot = round == 0 ? tm.team : tm.team - HALF;
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        const int col = 4 * (tm.tl + TT * v);
                        if (col < Jp) {
                            float4* d = reinterpret_cast<float4*>(comb + slot * Jp + col);
                            if (round == 0) {
                                *d = M[v];
                            } else {
                                float4 o = *d;
                                o.x = fmaxf(o.x, M[v].x);
                                o.y = fmaxf(o.y, M[v].y);
                                o.z = fmaxf(o.z, M[v].z);
                                o.w = fmaxf(o.w, M[v].w);
                                *d = o;
                            }
                        }
                    }
                }
                bar_named(CONS_BAR, NC);
            }
            for (int j = tid; j < Jp; j += NC) {
                float mm = comb[j];
                for (int t = 1; t < HALF; ++t) mm = fmaxf(mm, comb[t * Jp + j]);
                Gs[j] = mm;
            }
            bar_named(CONS_BAR, NC);
            for (int round = 0; round < 2; ++round) {
                if ((tm.team < HALF) == (round == 0)) {
                    const int slot = round == 0 ? tm.team : tm.team - HALF;
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        const int col = 4 * (tm.tl + TT * v);
                        if (col < Jp) {
                            float4 sc;
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const float Mc = comp(M[v], c), mm = Gs[col + c];
                                comp(sc, c) = Mc > -INFINITY ? comp(Sm[v], c) * ex2(Mc - mm) : 0.f;
                            }
                            float4* d = reinterpret_cast<float4*>(comb + slot * Jp + col);
                            if (round == 0) {
                                *d = sc;
                            } else {
                                float4 o = *d;
                                o.x += sc.x;
                                o.y += sc.y;
                                o.z += sc.z;
                                o.w += sc.w;
                                *d = o;
                            }
                        }
                    }
                }
                bar_named(CONS_BAR, NC);
            }
            for (int j = tid; j < J; j += NC) {
                float ss = comb[j];
                for (int t = 1; t < HALF; ++t) ss += comb[t * Jp + j];
                part2[(int64_t)vp * Jp + j] = make_float2(Gs[j], ss);
            }
            bar_named(CONS_BAR, NC);
            load_G_smem(P.G, J, Jp, Gs, tid, NC);
            bar_named(CONS_BAR, NC);
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                M[v] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
                Sm[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        OTA_BARRIER();
        // G^1_j = G^0_j + log2 q^_j - log2(column sum of pi^(1/2)), one warp per column
        {
            const int gw = b * NCW + warp, nw = nb * NCW;
            for (int j = gw; j < J; j += nw) {
                float mm = -INFINITY;
                for (int bb = lane; bb < V; bb += 32) mm = fmaxf(mm, part2[(int64_t)bb * Jp + j].x);
                mm = warp_max(mm);
                double ss = 0.0;
                if (mm > -INFINITY)
                    for (int bb = lane; bb < V; bb += 32) {
                        const float2 o = part2[(int64_t)bb * Jp + j];
                        if (o.x > -INFINITY) ss += (double)o.y * (double)ex2(o.x - mm);
                    }
                ss = warp_sum(ss);
                if (lane == 0) {
                    if (!(ss > 0.0) || !isfinite(ss)) {
                        atomicCAS(status, DEV_OK, DEV_ENUMERIC);
                    } else {
                        P.G[Jp + j] = P.G[j] + LQ[j] - ((double)mm + log2(ss));
                    }
                }
            }
        }
        OTA_BARRIER_CHECK();
        load_G_smem(P.G + Jp, J, Jp, Gs, tid, NC);
        bar_named(CONS_BAR, NC);
    }

    if (P.init_only) {  // iteration 1 is all that was asked for: no sweep to test its plan
        if (P.F_out)
            for (int r = tid; r < nrow; r += NC) P.F_out[r0 + r] = Fs[S.rmax + r];
        if (b == 0 && tid == 0) {
            P.st->iters = 1;
            P.st->err = 0.0;
            P.st->converged = 0;
        }
        *ret_par = 1;
        if (tid == 0) s_stop = 1;
        return true;
    }

    // ---- sweeps 2, 3, ...: one read of C and one ex2 per cell -----------------------------
    // Each partition adds its column partials (and row residual) as fixed-point integers into
    // the row of totals of this sweep; after the one grid barrier of the iteration every CTA
    // reads the totals and forms all column updates itself in its shared-memory copy of G.
    for (int s = 2;; ++s) {
        unsigned long long* acc_s = ACC + (size_t)(s % 3) * (Jp + 4);
        const float2* Fold = Fs + ((s - 1) & 1) * S.rmax;  // F'^(s-1)
        float2* Fnew = Fs + (s & 1) * S.rmax;
        float4 acc[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        float errt = 0.f;  // every lane of a team holds the same value
        int kb = 0;
        for (int vp = v0; vp < v1; ++vp) {
          const int vend = pend[vp];
          for (; kb < vend; ++kb) {
            const int st = (int)(cseq % (uint32_t)S.stages);
            const uint32_t ph = (cseq / (uint32_t)S.stages) & 1u;
            const bool ok = EUC || mbar_try_wait(&full[st], ph) || mbar_wait_bounded(&full[st], ph, P.spin, g.abort);
            const int lr0 = kb * rs_;
            const int rows = min(rs_, nrow - lr0);
            const float* stage = ring + (size_t)st * S.stage_floats;
            for (int j = 0; ok && j < S.rpt; ++j) {
                const int rr = tm.team + NTEAMS * j;
                if (rr >= rows) break;
                const int lr = lr0 + rr;
                float4 x[VPT];
                if constexpr (EUC)
                    euclid_row<TW, VPT>(__ldg(P.dev_xy + r0 + lr), rxs, rxs + Jp, J, tm.tl, x);
                else
                    load_row_smem<TW, VPT>(stage + (size_t)rr * P.ld, J, tm.tl, x);
                const float2 F = Fold[lr];
                float rsum = 0.f;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const int col = 4 * (tm.tl + TT * v);
                    if (chunk_inside<TW, VPT>(v) || col < J) {  // chunks past the row carry no mass
                        float4 gv = *reinterpret_cast<const float4*>(Gs + col);
                        float4 gl = *reinterpret_cast<const float4*>(Gs + Jp + col);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float t = ex2(expo2(F.x, F.y + comp(gl, c), comp(gv, c), comp(x[v], c), P.k_hi, P.k_lo));
                            comp(x[v], c) = t;
                            rsum += t;
                        }
                    } else {
                        x[v] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                rsum = team_reduce<TW, float, false>(rsum, red, NTEAMS, tm, par);
                const float ph = Ps[lr];
                // every lane forms the update (no divergent branch); one lane stores it
                const float2 Fn = df_sub(F, log2_corr(rsum));
                if (tm.tl == 0) Fnew[lr] = Fn;
                errt = fmaf(ph, fabsf(rsum - 1.0f), errt);
                const float d = __fdividef(ph, rsum);
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    acc[v].x = fmaf(x[v].x, d, acc[v].x);
                    acc[v].y = fmaf(x[v].y, d, acc[v].y);
                    acc[v].z = fmaf(x[v].z, d, acc[v].z);
                    acc[v].w = fmaf(x[v].w, d, acc[v].w);
                }
            }
            __syncwarp();
            if (!EUC && lane == 0) mbar_arrive(&empty[st]);
            ++cseq;
          }
            // end of partition vp: its column partials (teams in order) and row residual.  The
            // FP32 partial is kept for the exact path and added to the column's total as
            // round(partial 2^S_j); a partial too large for the total marks the column.
            if (tm.tl == 0) errf[tm.team] = errt;
            float* cp = P.colpart + (int64_t)vp * Jp;
            cta_col_sum<TW, VPT>(comb, acc, J, Jp, tm, [&](int j, float sum) {
                cp[j] = sum;
                const int sx = SX[j];
                const float x = ldexpf(sum, sx);
                if (sx != 0 && x < 0x1p55f) atomicAdd(acc_s + j, (unsigned long long)__float2ull_rn(x));
                else atomicOr(acc_s + j, 1ull << 63);
            });
            if (tid == 0) {
                float2 e = make_float2(errf[0], 0.f);
                for (int t = 1; t < NTEAMS; ++t) e = df_add(e, errf[t]);
                atomicAdd(acc_s + Jp, (unsigned long long)__float2ull_rn(ldexpf(e.x + e.y, FX_ERR)));
                s_bad = 0;
            }
#pragma unroll
            for (int v = 0; v < VPT; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            errt = 0.f;
            if (vp + 1 < v1) bar_named(CONS_BAR, NC);  // errf is read by thread 0 above
        }
        // the constant per-column values of this thread's first round of column updates are
        // loaded before the barrier, so only the totals cross L2 after it
        constexpr int CU = 3;
        float2 lq0[CU];
        int sx0[CU];
#pragma unroll
        for (int u = 0; u < CU; ++u) {
            const int j = tid + u * NC;
            lq0[u] = j < J ? __ldcg(LQ2 + j) : make_float2(0.f, 0.f);
            sx0[u] = j < J ? __ldcg(SX + j) : 0;
        }
        OTA_BARRIER();
        // Loop test on pi^(s-1): every thread reads the same total of the row residuals.
        const double ed = (double)__ldcg(acc_s + Jp) * 0x1p-50;
        const bool conv = ed <= stop_tol(P.tol);
        if (conv || s - 1 >= P.max_iter) {
            if (b == 0 && tid == 0) {
                P.st->iters = s - 1;
                P.st->err = ed;
                P.st->converged = conv;
            }
            if (P.F_out)
                for (int r = tid; r < nrow; r += NC) P.F_out[r0 + r] = Fold[r];
            *ret_par = (s - 1) & 1;
            if (P.fpart) sk_finalize_sweep<TW, VPT, EUC>(P, S, sh, dyn, r0, nrow, v0, v1, Fold, cseq, g.abort);
            if (tid == 0) s_stop = 1;
            return true;
        }
        // G^s_j = G^(s-1)_j + log2 q^_j - log2 s_j, every column in every CTA (FP32 pairs).  The
        // sum s_j is the fixed-point total T_j 2^-S_j; a marked column, or one whose total is
        // too small to carry 30 bits, is summed exactly from the partitions' FP32 partials.
        {
            double* Gnew = P.G + (s & 1) * Jp;
            int bad = 0;
            // CU columns a thread per round: all loads of a round first (one trip to L2), then
            // the arithmetic
            for (int j0 = tid; j0 < J; j0 += CU * NC) {
                unsigned long long T[CU];
                float2 lq[CU];
                int sx[CU];
#pragma unroll
                for (int u = 0; u < CU; ++u) {
                    const int j = j0 + u * NC;
                    T[u] = j < J ? __ldcg(acc_s + j) : 0ull;
                    lq[u] = j0 == tid ? lq0[u] : (j < J ? __ldcg(LQ2 + j) : make_float2(0.f, 0.f));
                    sx[u] = j0 == tid ? sx0[u] : (j < J ? __ldcg(SX + j) : 0);
                }
#pragma unroll
                for (int u = 0; u < CU; ++u) {
                    const int j = j0 + u * NC;
                    if (j >= J) break;
                    float2 ls;
                    if (!(T[u] >> 63) && T[u] >= (1ull << 30)) {
                        const float th = __ull2float_rn(T[u]);
                        const float tl = (float)((long long)T[u] - (long long)__float2ull_rn(th));
                        ls = df_log2(make_float2(th, tl));
                        ls.x -= (float)sx[u];
                    } else {
                        float2 sum = make_float2(0.f, 0.f);
                        for (int v = 0; v < V; ++v) sum = df_add(sum, __ldcg(P.colpart + (int64_t)v * Jp + j));
                        if (!(sum.x > 0.f) || !isfinite(sum.x)) {
                            bad = 1;
                            continue;
                        }
                        ls = df_log2(sum);
                    }
                    const float2 d = df_add2(lq[u], make_float2(-ls.x, -ls.y));
                    const float2 Gn = df_add2(make_float2(Gs[j], Gs[Jp + j]), d);
                    Gs[j] = Gn.x;
                    Gs[Jp + j] = Gn.y;
                    if ((j >> 5) % nb == b) Gnew[j] = (double)Gn.x + (double)Gn.y;  // the FP64 copy, once
                }
            }
            // this CTA's share of clearing the totals of sweep s + 2 (last read before this
            // iteration's barrier; next written after the next one)
            unsigned long long* acc_z = ACC + (size_t)((s + 2) % 3) * (Jp + 4);
            for (int t = b * NC + tid; t < Jp + 4; t += nb * NC) acc_z[t] = 0ull;
            if (bad) atomicOr(&s_bad, 1);
            bar_named(CONS_BAR, NC);
            if (s_bad) {  // every CTA sees the same totals and takes the same decision
                if (tid == 0) atomicCAS(status, DEV_OK, DEV_ENUMERIC);
                if (tid == 0) s_stop = 1;
                return false;
            }
        }
    }
#undef OTA_BARRIER_CHECK
#undef OTA_BARRIER
}

}  // namespace ota
