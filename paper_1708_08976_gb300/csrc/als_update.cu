// als_update.cu -- the factor update of a CP-ALS step (Section 2.2) in one launch per mode,
// and the Grams of all factors in one launch.
//
//   H = Hadamard_{k != n} G_k,  U_n = M H^{-1},  G_n = U_n^T U_n,  and after the last
//   mode of a sweep the fit (r^2 = ||X||^2 - 2 <M, U_n> + sum_ab prod_k G_k(a, b)).
//
// The shape follows what the FP64 pipe of this part allows (measured with clock64 in one
// CTA): a dependent FP64 FMA takes ~64 cycles, one warp issues at most one FP64
// instruction per ~64 cycles however many of its lanes are active, the SM as a whole peaks
// near one FP64 warp-instruction per ~17 cycles, and an FP64 reciprocal costs ~440 cycles.
// Everything that does not need M runs before griddepcontrol.wait, i.e. (launched with
// programmatic stream serialisation) while the kernel that writes M is still running; what
// is left after M arrives is short and runs on the FP32 pipe.
//  - H = L D L^T is factored in FP64 without a division on its C-step chain.  Step j
//    replaces the trailing entries by 2^-e_j (d_j A(i,k) - A(i,j) A(k,j)), d_j the current
//    pivot and e_j its binary exponent; the scaling is an exact exponent change.  After
//    step j every trailing entry is sigma_{j+1} times the true Schur complement, with
//    sigma_{j+1} = sigma_j * (d_j 2^-e_j) (a factor in [1, 2) per step), so
//    L(i, j) = A(i, j) / d_j and D_j = d_j / sigma_j; the C reciprocals are taken once,
//    in parallel, after the elimination.  H is positive definite iff every pivot is > 0
//    (the pivots are the squares of the Cholesky diagonal, up to the positive sigma_j);
//    otherwise MTK_ENOTPD is raised and U_n is left as it is.
//  - W = L^{-1} by column elimination (C - 1 steps of independent FMAs, one barrier
//    each), then H^{-1} = W^T D^{-1} W, all in FP64.  H^{-1} is kept in shared memory as
//    pairs of FP32 numbers (hi + lo, 48 significant bits).
//  - H^{-1} comes from als_factor_kernel (one CTA), launched ahead of the mode's MTTKRP
//    contraction, which it overlaps on an SM the contraction leaves free.  After M
//    arrives, each row is U_n(i, :) = M(i, :) H^{-1}: every product of an FP32 entry of
//    M and an FP32 half of H^{-1} formed exactly, the C of them summed in double-FP32
//    (about 2^-44 relative), then rounded to FP32 (one warp per row, one column per lane).
//  - Without that kernel (MTTKRPs on the FP32 tensor), every CTA of the update factors H
//    itself (all of them obtain bitwise the same factor) before griddepcontrol.wait, and
//    solves each row by L y = m, z = D^{-1} y, L^T u = z in FP64.
//  - The Gram of the new U_n runs on the FP32 pipe in double-FP32 arithmetic: exact
//    products (p = a*b, q = fma(a, b, -p)) and two-sum accumulation (Knuth, TAOCP vol. 2,
//    4.2.2; Dekker 1971), about 2^-44 relative.  The per-CTA partials are added in a
//    fixed order by a ticket reduction (the last CTA adds all partials when there are at
//    most 32, else groups of 8 CTAs and then the groups) and rounded once to FP64, so results do not depend on scheduling; the last CTA writes
//    G_n, which the next mode's update reads as it is.
#include <string.h>

#include "mtk_internal.cuh"

namespace mtk {
namespace {

size_t rup(size_t x, size_t m) { return (x + m - 1) / m * m; }

constexpr int kUpdThreads = 128;
constexpr int kUpdRows = 4;                                   // rows per pass: one per warp
constexpr int kUpdMaxC = 64;
constexpr int kMaxPairs = kUpdMaxC * (kUpdMaxC + 1) / 2;      // 2080
constexpr int kPairsPerThread = (kMaxPairs + kUpdThreads - 1) / kUpdThreads;
constexpr int kUpdMaxCtas = 128;
constexpr int kAppThreads = 256;                              // the factor update: 8 warps
constexpr int kAppRows = kAppThreads / 32;                    // rows per pass: one per warp
constexpr int kAppPairs = (kMaxPairs + kAppThreads - 1) / kAppThreads;
constexpr int kGroup = 8;                                     // CTAs per first-level group
constexpr int kGramRows = 16;                                 // rows staged per pass (Grams)
constexpr int kGramMaxCtas = 64;                              // per factor
// ticket words: [0, 64) the update kernel (1 + up to 38 groups), then 16 per factor
constexpr int kTicketUpd = 0;
constexpr int kTicketGram = 64;
constexpr int kTicketPerFactor = 16;

// ---- double-FP32 arithmetic -------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += a * b, the product formed exactly
__device__ __forceinline__ void df_madd(float& hi, float& lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float q = fmaf(a, b, -p);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, q));
}
__device__ __forceinline__ void df_renorm(float& hi, float& lo) {
    const float s = __fadd_rn(hi, lo);
    lo = __fsub_rn(lo, __fsub_rn(s, hi));
    hi = s;
}
// (hi, lo) += (bh, bl)
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
    float s, e;
    two_sum(hi, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = s;
    lo = e;
    df_renorm(hi, lo);
}

// w * 2^-e, exact while the result is a normal number; results below the normal range
// are flushed to zero, infinities and NaNs pass through
__device__ __forceinline__ double scale_exp2(double w, int e) {
    long long b = __double_as_longlong(w);
    const int ew = (int)((b >> 52) & 0x7FF);
    if (ew == 0x7FF) return w;
    if (ew == 0) return 0.0;
    const int en = ew - e;
    if (en <= 0) return 0.0;
    if (en >= 0x7FF) return w > 0.0 ? __longlong_as_double(0x7FF0000000000000LL)
                                     : __longlong_as_double((long long)0xFFF0000000000000ULL);
    b = (b & ~(0x7FFLL << 52)) | ((long long)en << 52);
    return __longlong_as_double(b);
}

// lower-triangle index pairs (i, k), i >= k, ordered by column from the last one: the
// entries with k > j are exactly the first (C-1-j)(C-j)/2 of the list
__device__ __forceinline__ void build_pairs(int* tri, int C) {
    for (int k = threadIdx.x; k < C; k += blockDim.x) {
        const int base = (C - 1 - k) * (C - k) / 2;
        for (int i = k; i < C; ++i) tri[base + (i - k)] = (i << 8) | k;
    }
}

// dst[x] = sum over rows b = 0..cnt-1 of src[b][x] (double-FP32, in row order).  A thread
// takes 3 entries x and loads 8 rows of each before adding, so each round of 24 loads is
// one trip to L2 (the sums are short and latency-bound).
__device__ void sum_rows(const float2* __restrict__ src, int cnt, int npairs, float2* __restrict__ dst) {
    constexpr int PX = 3, B = 8;
    const int nt = (int)blockDim.x;
    for (int x0 = threadIdx.x; x0 < npairs; x0 += PX * nt) {
        float h[PX], l[PX];
#pragma unroll
        for (int q = 0; q < PX; ++q) h[q] = l[q] = 0.0f;
        for (int b0 = 0; b0 < cnt; b0 += B) {
            float2 v[PX][B];
#pragma unroll
            for (int q = 0; q < PX; ++q)
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    const int x = x0 + q * nt;
                    v[q][j] = (b0 + j < cnt && x < npairs) ? __ldcg(src + (size_t)(b0 + j) * npairs + x)
                                                            : make_float2(0.0f, 0.0f);
                }
#pragma unroll
            for (int q = 0; q < PX; ++q)
#pragma unroll
                for (int j = 0; j < B; ++j)
                    if (b0 + j < cnt) df_add(h[q], l[q], v[q][j].x, v[q][j].y);
        }
#pragma unroll
        for (int q = 0; q < PX; ++q)
            if (x0 + q * nt < npairs) dst[x0 + q * nt] = make_float2(h[q], l[q]);
    }
}

// Two-level fixed-order reduction of per-CTA partials.  Every thread of the CTA calls it
// after the CTA wrote row `idx` of part[cnt][npairs].  Group g = idx / 8: the last CTA of
// the group to arrive adds the group's rows into gsum[g]; the last group to finish adds
// the groups into fin (npairs entries, may be shared memory).  Returns 1 in that one CTA.
// tk[0] counts finished groups, tk[1 + g] the arrivals in group g; both are left at zero.
// dst[x] = sum over rows b = 0..cnt-1 (cnt <= 32) of src[b][x], all rows of a thread's
// entries loaded at once (one trip to L2)
__device__ void sum_rows32(const float2* __restrict__ src, int cnt, int npairs, float2* __restrict__ dst) {
    for (int x = threadIdx.x; x < npairs; x += blockDim.x) {
        float2 v[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) v[b] = b < cnt ? __ldcg(src + (size_t)b * npairs + x) : make_float2(0.0f, 0.0f);
        float h = 0.0f, l = 0.0f;
#pragma unroll
        for (int b = 0; b < 32; ++b)
            if (b < cnt) df_add(h, l, v[b].x, v[b].y);
        dst[x] = make_float2(h, l);
    }
}

__device__ int ticket_reduce(float2* part, float2* gsum, float2* fin, unsigned int* tk, int idx, int cnt,
                             int npairs, int* flag) {
    __threadfence();
    __syncthreads();
    if (cnt <= 32) {
        // one level: the last CTA to arrive adds every row, in row order
        if (threadIdx.x == 0) *flag = (atomicAdd(&tk[0], 1u) == (unsigned)(cnt - 1)) ? 1 : 0;
        __syncthreads();
        if (!*flag) return 0;
        __threadfence();
        sum_rows32(part, cnt, npairs, fin);
        if (threadIdx.x == 0) tk[0] = 0u;
        __syncthreads();
        return 1;
    }
    const int g = idx / kGroup, ng = (cnt + kGroup - 1) / kGroup;
    const int members = (cnt - kGroup * g) < kGroup ? (cnt - kGroup * g) : kGroup;
    if (threadIdx.x == 0) *flag = (atomicAdd(&tk[1 + g], 1u) == (unsigned)(members - 1)) ? 1 : 0;
    __syncthreads();
    if (!*flag) return 0;
    __threadfence();
    sum_rows(part + (size_t)kGroup * g * npairs, members, npairs, gsum + (size_t)g * npairs);
    if (threadIdx.x == 0) tk[1 + g] = 0u;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *flag = (atomicAdd(&tk[0], 1u) == (unsigned)(ng - 1)) ? 1 : 0;
    __syncthreads();
    if (!*flag) return 0;
    __threadfence();
    sum_rows(gsum, ng, npairs, fin);
    if (threadIdx.x == 0) tk[0] = 0u;
    __syncthreads();
    return 1;
}

// G (C x C, FP64, both triangles) from the reduced double-FP32 pair sums
__device__ void write_gram(const float2* fin, const int* tri, int npairs, int C, double* G) {
    for (int x = threadIdx.x; x < npairs; x += blockDim.x) {
        const float2 v = fin[x];
        const double g = (double)v.x + (double)v.y;
        const int i = tri[x] >> 8, k = tri[x] & 255;
        G[i * C + k] = g;
        G[k * C + i] = g;
    }
}

// the same with the columns of U scaled by sc: G(i, k) sc_i sc_k (exact scales: FP32 numbers)
__device__ void write_gram_scaled(const float2* fin, const int* tri, int npairs, int C, const float* sc, double* G) {
    for (int x = threadIdx.x; x < npairs; x += blockDim.x) {
        const float2 v = fin[x];
        const int i = tri[x] >> 8, k = tri[x] & 255;
        const double g = ((double)v.x + (double)v.y) * ((double)sc[i] * (double)sc[k]);
        G[i * C + k] = g;
        G[k * C + i] = g;
    }
}

// index of (a, b) in the pair list (build_pairs order)
__device__ __forceinline__ int pair_index(int a, int b, int C) {
    const int i = a > b ? a : b, k = a > b ? b : a;
    return (C - 1 - k) * (C - k) / 2 + (i - k);
}

struct UpdParams {
    const double* G[MTK_MAXN];   // Grams of the factors (entry n not read)
    int N, C, n;
    const float* M;              // In x C
    int64_t In;
    float* Un;                   // In x C, overwritten (left as it is when H is not pd)
    int64_t rows;                // rows per CTA, a multiple of kAppRows
    int gram;                    // 1: the Gram of U_n is reduced here and written to Gn
    double* Gn;
    float2* part;                // [grid][npairs] this CTA's partial Gram
    float2* gsum;                // [groups][npairs]
    double* dots;                // [grid] partial <M, U_n> (with the fit)
    unsigned int* tk;            // tickets, zero on entry and on exit
    const double* normX2;        // with gram: the fit (else null)
    double* fit;
    double* r2;
    uint32_t* status;
    const float2* hinv;          // H^{-1} formed by als_factor_kernel (C x C pairs), then its not-pd
                                 // flag (an int at hinv + C*C); null: H is factored here
    int normalize;               // with gram, without the fit: U_n and G_n scaled to unit columns
};

// ---- the factorisation, on shared memory, by all threads of the CTA ------------------------
// A = H = Hadamard_{k != n} G_k (the loads of one factor issued together)
__device__ void form_h(const double* const* G, int N, int n, int C, double* A) {
    for (int e0 = threadIdx.x; e0 < C * C; e0 += 4 * blockDim.x) {
        double h[4];
        bool first = true;
        for (int k = 0; k < N; ++k) {
            if (k == n) continue;
            double g[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = e0 + q * (int)blockDim.x;
                g[q] = e < C * C ? G[k][e] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) h[q] = first ? g[q] : h[q] * g[q];
            first = false;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = e0 + q * (int)blockDim.x;
            if (e < C * C) A[e] = h[q];
        }
    }
    __syncthreads();
}

// Division-free L D L^T of A (lower triangle), one barrier per step.  Returns true when H
// is not positive definite (the same answer in every thread).  Otherwise L is left in both
// triangles of A (A[i][k] = A[k][i] = L(i, k), i > k) and dinv[k] = D_k^{-1}.
__device__ bool ldl(double* A, int C, const int* tri, double* dinv, double* rcp, double* red) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nt = blockDim.x;
    for (int j = 0; j < C; ++j) {
        const double d = A[j * C + j];
        const int ed = (int)((__double_as_longlong(d) >> 52) & 0x7FF);
        if (!(d > 0.0) || ed == 0 || ed == 0x7FF) return true;
        const int ej = ed - 1023;
        const int m = C - 1 - j;
        const int cnt = m * (m + 1) / 2;
        for (int x = t; x < cnt; x += nt) {
            const int i = tri[x] >> 8, k = tri[x] & 255;
            const double v = A[i * C + j] * A[k * C + j];
            A[i * C + k] = scale_exp2(fma(d, A[i * C + k], -v), ej);
        }
        __syncthreads();
    }
    // sigma_j = prod_{m<j} mant(d_m) (exclusive scan), D_j^{-1} = sigma_j / d_j
    double s_own = 1.0, r_own = 0.0;
    if (t < C) {
        const double d = A[t * C + t];
        s_own = __longlong_as_double((__double_as_longlong(d) & 0x000FFFFFFFFFFFFFLL) | (1023LL << 52));
        r_own = 1.0 / d;
        rcp[t] = r_own;
    }
    double incl = s_own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl *= y;
    }
    if (t == 31) red[0] = incl;
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 1.0;
    __syncthreads();
    if (warp == 1) excl *= red[0];
    if (t < C) dinv[t] = excl * r_own;
    __syncthreads();
    const int npairs = C * (C + 1) / 2;
    for (int x = t; x < npairs; x += nt) {
        const int i = tri[x] >> 8, k = tri[x] & 255;
        if (i > k) {
            const double l = A[i * C + k] * rcp[k];
            A[i * C + k] = l;
            A[k * C + i] = l;
        }
    }
    __syncthreads();
    return false;
}

// H^{-1} = W^T D^{-1} W with W = L^{-1} (column elimination, C - 1 steps of independent
// FMAs, one barrier each), kept as FP32 pairs (hi + lo, 48 significant bits), both
// triangles, row-major [k][c].  W: C x C doubles of scratch.
__device__ void ldl_inverse(const double* A, double* W, const double* dinv, const int* tri, float2* Hv, int C) {
    const int t = threadIdx.x, nt = blockDim.x;
    for (int e = t; e < C * C; e += nt) W[e] = (e / C == e % C) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k + 1 < C; ++k) {
        const int w = k + 1, cnt = (C - 1 - k) * w;
        for (int x = t; x < cnt; x += nt) {
            const int q = x / w;
            const int i = k + 1 + q, c = x - q * w;
            W[i * C + c] = fma(-A[i * C + k], W[k * C + c], W[i * C + c]);
        }
        __syncthreads();
    }
    const int npairs = C * (C + 1) / 2;
    for (int x = t; x < npairs; x += nt) {
        const int a = tri[x] >> 8, b = tri[x] & 255;
        double s0 = 0.0, s1 = 0.0;
        int k = a;
        for (; k + 1 < C; k += 2) {
            s0 = fma(W[k * C + a] * dinv[k], W[k * C + b], s0);
            s1 = fma(W[(k + 1) * C + a] * dinv[k + 1], W[(k + 1) * C + b], s1);
        }
        if (k < C) s0 = fma(W[k * C + a] * dinv[k], W[k * C + b], s0);
        const double h = s0 + s1;
        const float hh = (float)h;
        const float2 v = make_float2(hh, (float)(h - (double)hh));
        Hv[a * C + b] = v;
        Hv[b * C + a] = v;
    }
    __syncthreads();
}

// ---- H^{-1} alone, one CTA (launched ahead of a long kernel that it may overlap) -------
struct FactorParams {
    const double* G[MTK_MAXN];
    int N, C, n;
    float2* hinv;                // C x C pairs, then the not-pd flag (int)
    uint32_t* status;
};

// dynamic shared memory: A[C*C], W[C*C] (doubles), Hv[C*C] (float2)
__global__ void __launch_bounds__(kAppThreads) als_factor_kernel(const __grid_constant__ FactorParams p) {
    // the next kernel of the stream (launched with programmatic serialisation) may start now
    allow_dependent_launch();
    extern __shared__ double dsm[];
    __shared__ double dinv[kUpdMaxC], rcp[kUpdMaxC];
    __shared__ double red[kAppThreads / 32];
    __shared__ int tri[kMaxPairs];
    const int C = p.C;
    double* A = dsm;
    double* W = A + C * C;
    float2* Hv = reinterpret_cast<float2*>(W + C * C);
    build_pairs(tri, C);
    form_h(p.G, p.N, p.n, C, A);
    const bool bad = ldl(A, C, tri, dinv, rcp, red);
    if (!bad) ldl_inverse(A, W, dinv, tri, Hv, C);
    for (int e = threadIdx.x; e < C * C && !bad; e += blockDim.x) p.hinv[e] = Hv[e];
    if (threadIdx.x == 0) *reinterpret_cast<int*>(p.hinv + C * C) = bad ? 1 : 0;
    if (bad && threadIdx.x == 0) set_status(p.status, MTK_ENOTPD);
}

// ---- the update ------------------------------------------------------------------------------
// dynamic shared memory: A[C*C] (doubles), Hv[C*C] and fin[npairs] (float2)
__global__ void __launch_bounds__(kAppThreads)
als_update_kernel(const __grid_constant__ UpdParams p) {
    extern __shared__ double dsm[];
    __shared__ double dinv[kUpdMaxC], rcp[kUpdMaxC];
    __shared__ double red[kAppThreads / 32];
    __shared__ int tri[kMaxPairs];
    __shared__ float ur[kAppRows][kUpdMaxC];
    __shared__ float nsc[kUpdMaxC];
    __shared__ int flag;

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int C = p.C, N = p.N, n = p.n;
    const int npairs = C * (C + 1) / 2;
    double* A = dsm;
    float2* Hv = reinterpret_cast<float2*>(A + C * C);
    float2* fin = Hv + C * C;

    build_pairs(tri, C);
    // ---- the inverse from als_factor_kernel, or L D L^T here (before M is ready)
    const bool pre = p.hinv != nullptr;
    bool bad;
    if (pre) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        bad = *reinterpret_cast<const volatile int*>(p.hinv + C * C) != 0;
        for (int e = t; e < C * C && !bad; e += kAppThreads) Hv[e] = p.hinv[e];
        __syncthreads();
    } else {
        form_h(p.G, N, n, C, A);
        bad = ldl(A, C, tri, dinv, rcp, red);
        if (bad && blockIdx.x == 0 && t == 0) set_status(p.status, MTK_ENOTPD);
        // ---- M is written by the previous kernel
        asm volatile("griddepcontrol.wait;" ::: "memory");
    }

    const bool gram = p.gram != 0;
    const bool fit = gram && p.normX2 != nullptr;
    const int64_t r0 = (int64_t)blockIdx.x * p.rows;
    const int64_t r1 = (r0 + p.rows < p.In) ? r0 + p.rows : p.In;
    float gh[kAppPairs], gl[kAppPairs];
#pragma unroll
    for (int q = 0; q < kAppPairs; ++q) gh[q] = gl[q] = 0.0f;
    double dot = 0.0;
    const int j0 = lane, j1 = lane + 32;
    for (int64_t rb = r0; rb < r1; rb += kAppRows) {
        const int64_t i = rb + warp;
        float u0 = 0.0f, u1 = 0.0f;
        if (i < r1) {
            const float* mrow = p.M + i * C;
            float* urow = p.Un + i * C;
            const float m0 = j0 < C ? mrow[j0] : 0.0f;
            const float m1 = j1 < C ? mrow[j1] : 0.0f;
            if (!bad && pre) {
                // U_n(i, :) = M(i, :) H^{-1}: products of an FP32 entry and an FP32 pair,
                // each formed exactly, summed in double-FP32 (about 2^-44 relative)
                float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
                if (C > 32) {
                    for (int k = 0; k < C; ++k) {
                        const float mk = __shfl_sync(0xffffffffu, k < 32 ? m0 : m1, k & 31);
                        const float2 w = Hv[k * C + j0];
                        df_madd(h0, l0, mk, w.x);
                        l0 = fmaf(mk, w.y, l0);
                        if (j1 < C) {
                            const float2 v = Hv[k * C + j1];
                            df_madd(h1, l1, mk, v.x);
                            l1 = fmaf(mk, v.y, l1);
                        }
                    }
                } else {
                    // one column per lane (the second column is past C for every lane)
                    for (int k = 0; k < C; ++k) {
                        const float mk = __shfl_sync(0xffffffffu, m0, k);
                        if (j0 < C) {
                            const float2 w = Hv[k * C + j0];
                            df_madd(h0, l0, mk, w.x);
                            l0 = fmaf(mk, w.y, l0);
                        }
                    }
                }
                u0 = __fadd_rn(h0, l0);
                u1 = __fadd_rn(h1, l1);
            } else if (!bad) {
                // L y = m, z = D^{-1} y, L^T u = z in FP64, one column per lane, the solved
                // entry broadcast by a shuffle
                // (the second column per lane only when C > 32: a uniform branch, so that the
                // FP64 pipe, narrow on this part, issues no dead instructions)
                double s0 = (double)m0, s1 = (double)m1;
                if (C > 32) {
                    for (int k = 0; k < C; ++k) {
                        const double y = __shfl_sync(0xffffffffu, k < 32 ? s0 : s1, k & 31);
                        if (j0 > k) s0 = fma(-A[k * C + j0], y, s0);
                        if (j1 > k && j1 < C) s1 = fma(-A[k * C + j1], y, s1);
                    }
                    s0 *= dinv[j0];
                    if (j1 < C) s1 *= dinv[j1];
                    for (int k = C - 1; k >= 0; --k) {
                        const double y = __shfl_sync(0xffffffffu, k < 32 ? s0 : s1, k & 31);
                        if (j0 < k) s0 = fma(-A[k * C + j0], y, s0);
                        if (j1 < k && j1 < C) s1 = fma(-A[k * C + j1], y, s1);
                    }
                } else {
                    for (int k = 0; k < C; ++k) {
                        const double y = __shfl_sync(0xffffffffu, s0, k);
                        if (j0 > k && j0 < C) s0 = fma(-A[k * C + j0], y, s0);
                    }
                    if (j0 < C) s0 *= dinv[j0];
                    for (int k = C - 1; k >= 0; --k) {
                        const double y = __shfl_sync(0xffffffffu, s0, k);
                        if (j0 < k) s0 = fma(-A[k * C + j0], y, s0);
                    }
                }
                u0 = (float)s0;
                u1 = (float)s1;
            }
            if (!bad) {
                if (j0 < C) urow[j0] = u0;
                if (j1 < C) urow[j1] = u1;
            } else {
                if (j0 < C) u0 = urow[j0];
                if (j1 < C) u1 = urow[j1];
            }
            if (fit) {
                if (j0 < C) dot = fma((double)m0, (double)u0, dot);
                if (j1 < C) dot = fma((double)m1, (double)u1, dot);
            }
        }
        if (!gram) continue;
        if (j0 < C) ur[warp][j0] = u0;
        if (j1 < C) ur[warp][j1] = u1;
        __syncthreads();
        const int nr = (r1 - rb) < kAppRows ? (int)(r1 - rb) : kAppRows;
#pragma unroll
        for (int q = 0; q < kAppPairs; ++q) {
            const int x = t + q * kAppThreads;
            if (x < npairs) {
                const int a = tri[x] >> 8, b = tri[x] & 255;
                for (int r = 0; r < nr; ++r) df_madd(gh[q], gl[q], ur[r][a], ur[r][b]);
            }
        }
        __syncthreads();
    }
    if (!gram) return;

    // ---- partial Gram (and partial <M, U_n>) of this CTA, then the fixed-order reduction
    float2* prow = p.part + (size_t)blockIdx.x * npairs;
#pragma unroll
    for (int q = 0; q < kAppPairs; ++q) {
        const int x = t + q * kAppThreads;
        if (x < npairs) {
            df_renorm(gh[q], gl[q]);
            prow[x] = make_float2(gh[q], gl[q]);
        }
    }
    if (fit) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
        if (lane == 0) red[warp] = dot;
        __syncthreads();
        if (t == 0) {
            double sd = 0.0;
            for (int w = 0; w < kAppThreads / 32; ++w) sd += red[w];
            p.dots[blockIdx.x] = sd;
        }
    }
    if (!ticket_reduce(p.part, p.gsum, fin, p.tk + kTicketUpd, (int)blockIdx.x, (int)gridDim.x, npairs, &flag))
        return;
    if (p.normalize && !fit && !bad) {
        // the last CTA scales U_n to unit columns, s_c = fp32(1 / ||U_n(:, c)||) from the
        // new Gram's diagonal (1 for a zero column), and writes G_n of the scaled factor
        // (with H not positive definite U_n stays as it was, unscaled)
        for (int c = t; c < C; c += kAppThreads) {
            const float2 w = fin[pair_index(c, c, C)];
            const double g = (double)w.x + (double)w.y;
            nsc[c] = g > 0.0 ? (float)(1.0 / sqrt(g)) : 1.0f;
        }
        __syncthreads();
        for (int64_t i = warp; i < p.In; i += kAppThreads / 32) {
            float* urow = p.Un + i * C;               // rows of every CTA: read through L2
            if (j0 < C) urow[j0] = __fmul_rn(__ldcg(urow + j0), nsc[j0]);
            if (j1 < C) urow[j1] = __fmul_rn(__ldcg(urow + j1), nsc[j1]);
        }
        write_gram_scaled(fin, tri, npairs, C, nsc, p.Gn);
        return;
    }
    write_gram(fin, tri, npairs, C, p.Gn);
    if (!fit) return;
    // ---- fit: y2 = sum_ab prod_k G_k(a, b) with the new G_n (fin); <M, U_n> from the
    // partials
    double v = 0.0;
    for (int e0 = t; e0 < C * C; e0 += 4 * kAppThreads) {
        double h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = e0 + q * kAppThreads;
            if (e < C * C) {
                const float2 w = fin[pair_index(e / C, e % C, C)];
                h[q] = (double)w.x + (double)w.y;
            } else {
                h[q] = 0.0;
            }
        }
        for (int k = 0; k < N; ++k) {
            if (k == n) continue;
            double g[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = e0 + q * kAppThreads;
                g[q] = e < C * C ? p.G[k][e] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) h[q] *= g[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) v += h[q];
    }
    double ds = 0.0;
    for (int b = t; b < (int)gridDim.x; b += kAppThreads) ds += __ldcg(p.dots + b);
    v -= 2.0 * ds;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (t == 0) {
        const double nx2 = *p.normX2;
        double y = 0.0;
        for (int w = 0; w < kAppThreads / 32; ++w) y += red[w];
        const double r2 = nx2 + y;
        if (p.r2) *p.r2 = r2;
        if (p.fit) *p.fit = 1.0 - sqrt(r2 > 0.0 ? r2 : 0.0) / sqrt(nx2);
    }
}

// ---- Grams of all factors in one launch: CTAs [first[k], first[k+1]) take factor k
struct GramAllParams {
    const float* U[MTK_MAXN];
    int64_t I[MTK_MAXN];
    int64_t rows[MTK_MAXN];
    int first[MTK_MAXN + 1];
    int N, C;
    double* G[MTK_MAXN];
    float2* part;                // [grid][npairs]
    float2* gsum;                // [N][8][npairs]
    unsigned int* tk;
};

__global__ void __launch_bounds__(kUpdThreads) gram_all_kernel(const __grid_constant__ GramAllParams p) {
    __shared__ int tri[kMaxPairs];
    __shared__ float ur[kGramRows][kUpdMaxC];
    __shared__ float2 fin[kMaxPairs];
    __shared__ int flag;
    const int C = p.C, npairs = C * (C + 1) / 2;
    int f = 0;
    while (f + 1 < p.N && (int)blockIdx.x >= p.first[f + 1]) ++f;
    const int idx = (int)blockIdx.x - p.first[f], cnt = p.first[f + 1] - p.first[f];
    const float* U = p.U[f];
    const int64_t r0 = (int64_t)idx * p.rows[f];
    const int64_t r1 = (r0 + p.rows[f] < p.I[f]) ? r0 + p.rows[f] : p.I[f];
    build_pairs(tri, C);
    float gh[kPairsPerThread], gl[kPairsPerThread];
#pragma unroll
    for (int q = 0; q < kPairsPerThread; ++q) gh[q] = gl[q] = 0.0f;
    for (int64_t rb = r0; rb < r1; rb += kGramRows) {
        const int nr = (r1 - rb) < kGramRows ? (int)(r1 - rb) : kGramRows;
        __syncthreads();
        for (int e = threadIdx.x; e < nr * C; e += blockDim.x) ur[e / C][e % C] = U[rb * C + e];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPairsPerThread; ++q) {
            const int x = threadIdx.x + q * kUpdThreads;
            if (x < npairs) {
                const int a = tri[x] >> 8, b = tri[x] & 255;
                for (int r = 0; r < nr; ++r) df_madd(gh[q], gl[q], ur[r][a], ur[r][b]);
            }
        }
    }
    float2* prow = p.part + (size_t)blockIdx.x * npairs;
#pragma unroll
    for (int q = 0; q < kPairsPerThread; ++q) {
        const int x = threadIdx.x + q * kUpdThreads;
        if (x < npairs) {
            df_renorm(gh[q], gl[q]);
            prow[x] = make_float2(gh[q], gl[q]);
        }
    }
    if (!ticket_reduce(p.part + (size_t)p.first[f] * npairs, p.gsum + (size_t)f * kGroup * npairs, fin,
                       p.tk + kTicketGram + f * kTicketPerFactor, idx, cnt, npairs, &flag))
        return;
    write_gram(fin, tri, npairs, C, p.G[f]);
}

int gram_ctas(int64_t I, int64_t* rows) {
    int64_t P = (I + kGramRows - 1) / kGramRows;
    if (P > kGramMaxCtas) P = kGramMaxCtas;
    if (P < 1) P = 1;
    const int64_t r = (I + P - 1) / P;
    if (rows) *rows = r;
    return (int)((I + r - 1) / r);
}

size_t pair_bytes(int C) { return (size_t)(C * (C + 1) / 2) * sizeof(float2); }

}  // namespace

bool als_update_supported(int C) { return C >= 1 && C <= kUpdMaxC; }

size_t als_ticket_bytes() { return 2048; }

int als_update_ctas(int64_t In, int64_t* rows) {
    int64_t P = (In + kAppRows - 1) / kAppRows;
    int64_t r = kAppRows;
    if (P > kUpdMaxCtas) {
        r = ((In + kUpdMaxCtas - 1) / kUpdMaxCtas + kAppRows - 1) / kAppRows * kAppRows;
        P = (In + r - 1) / r;
    }
    if (rows) *rows = r;
    return (int)P;
}

int als_update_max_ctas(const int64_t* dims, int N) {
    int P = 1;
    for (int k = 0; k < N; ++k) {
        const int q = als_update_ctas(dims[k], nullptr);
        if (q > P) P = q;
    }
    return P;
}

// the per-CTA partial Grams, the ticket groups' sums, the partial dots
size_t als_update_scratch_bytes(int Pmax, int C) {
    const int ng = (Pmax + kGroup - 1) / kGroup;
    return rup((size_t)Pmax * pair_bytes(C), 256) + rup((size_t)ng * pair_bytes(C), 256) +
           rup((size_t)Pmax * sizeof(double), 256);
}

size_t gram_all_scratch_bytes(const int64_t* I, int N, int C) {
    int64_t P = 0;
    for (int k = 0; k < N; ++k) P += gram_ctas(I[k], nullptr);
    return rup((size_t)P * pair_bytes(C), 256) + rup((size_t)N * kGroup * pair_bytes(C), 256);
}

cudaError_t launch_als_update(const AlsUpdateArgs& a, cudaStream_t s) {
    UpdParams p;
    memset(&p, 0, sizeof(p));
    for (int k = 0; k < a.N && k < MTK_MAXN; ++k) p.G[k] = a.G[k];
    p.N = a.N;
    p.C = a.C;
    p.n = a.n;
    p.M = a.M;
    p.In = a.In;
    p.Un = a.Un;
    const int P = als_update_ctas(a.In, &p.rows);
    if (P > a.Pmax) return cudaErrorInvalidValue;
    const int ng = (a.Pmax + kGroup - 1) / kGroup;
    char* w = static_cast<char*>(a.scratch);
    p.gram = a.Gn ? 1 : 0;
    p.Gn = a.Gn;
    p.part = reinterpret_cast<float2*>(w);
    w += rup((size_t)a.Pmax * pair_bytes(a.C), 256);
    p.gsum = reinterpret_cast<float2*>(w);
    w += rup((size_t)ng * pair_bytes(a.C), 256);
    p.dots = reinterpret_cast<double*>(w);
    p.tk = a.tickets;
    p.normX2 = a.Gn ? a.normX2 : nullptr;
    p.fit = a.fit;
    p.r2 = a.r2;
    p.status = a.status;
    p.hinv = static_cast<const float2*>(a.hinv);
    p.normalize = a.normalize && a.Gn && !a.normX2 ? 1 : 0;
    const size_t smem = (size_t)a.C * a.C * sizeof(double) + (size_t)a.C * a.C * sizeof(float2) + pair_bytes(a.C);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(als_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)P);
    cfg.blockDim = dim3(kAppThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.programmatic ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, als_update_kernel, p);
    note_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

size_t als_hinv_bytes(int C) { return rup((size_t)C * C * sizeof(float2) + sizeof(int), 256); }

cudaError_t launch_als_factor(const double* const* G, int N, int C, int n, void* hinv, uint32_t* status,
                              cudaStream_t s) {
    FactorParams p;
    memset(&p, 0, sizeof(p));
    for (int k = 0; k < N && k < MTK_MAXN; ++k) p.G[k] = G[k];
    p.N = N;
    p.C = C;
    p.n = n;
    p.hinv = static_cast<float2*>(hinv);
    p.status = status;
    const size_t smem = 2 * (size_t)C * C * sizeof(double) + (size_t)C * C * sizeof(float2);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(als_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    als_factor_kernel<<<1, kAppThreads, smem, s>>>(p);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gram_all(const float* const* U, const int64_t* I, int N, int C, double* const* G,
                            void* scratch, unsigned int* tickets, cudaStream_t s) {
    GramAllParams p;
    memset(&p, 0, sizeof(p));
    int P = 0;
    for (int k = 0; k < N; ++k) {
        p.U[k] = U[k];
        p.I[k] = I[k];
        p.G[k] = G[k];
        p.first[k] = P;
        P += gram_ctas(I[k], &p.rows[k]);
    }
    p.first[N] = P;
    p.N = N;
    p.C = C;
    char* w = static_cast<char*>(scratch);
    p.part = reinterpret_cast<float2*>(w);
    w += rup((size_t)P * (int64_t)pair_bytes(C), 256);
    p.gsum = reinterpret_cast<float2*>(w);
    p.tk = tickets;
    gram_all_kernel<<<P, kUpdThreads, 0, s>>>(p);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace mtk
