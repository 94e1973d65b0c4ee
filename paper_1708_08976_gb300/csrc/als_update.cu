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
//  - H = L D L^T is factored in FP64 without a division on its C-step chain.  Step j
//    replaces the trailing entries by 2^-e_j (d_j A(i,k) - A(i,j) A(k,j)), d_j the current
//    pivot and e_j its binary exponent; the scaling is an exact exponent change.  After
//    step j every trailing entry is sigma_{j+1} times the true Schur complement, with
//    sigma_{j+1} = sigma_j * (d_j 2^-e_j) (a factor in [1, 2) per step), so
//    L(i, j) = A(i, j) / d_j and D_j = d_j / sigma_j; the C reciprocals are taken once,
//    in parallel, after the elimination.  H is positive definite iff every pivot is > 0
//    (the pivots are the squares of the Cholesky diagonal, up to the positive sigma_j);
//    otherwise MTK_ENOTPD is raised and U_n is left as it is.
//  - Each row of U_n solves L y = m, z = D^{-1} y, L^T u = z in FP64 (one warp per row,
//    one column per lane, the solved entry broadcast by a shuffle).
//  - Every CTA factors H itself (all of them obtain bitwise the same factor), so the
//    update needs no second launch.  Launched with programmatic stream serialisation,
//    the factorisation runs before griddepcontrol.wait, i.e. while the kernel that
//    writes M is still running.
//  - The Gram sums run on the FP32 pipe in double-FP32 arithmetic: exact products
//    (p = a*b, q = fma(a, b, -p)) and two-sum accumulation (Knuth, TAOCP vol. 2,
//    4.2.2; Dekker 1971), about 2^-44 relative.  The per-CTA partials are added in a
//    fixed order by a two-level ticket reduction (groups of 8 CTAs, then the groups) and
//    rounded once to FP64, so results do not depend on scheduling.
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
constexpr int kUpdMaxCtas = 304;
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
__device__ int ticket_reduce(float2* part, float2* gsum, float2* fin, unsigned int* tk, int idx, int cnt,
                             int npairs, int* flag) {
    __threadfence();
    __syncthreads();
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

// index of (a, b) in the pair list (build_pairs order)
__device__ __forceinline__ int pair_index(int a, int b, int C) {
    const int i = a > b ? a : b, k = a > b ? b : a;
    return (C - 1 - k) * (C - k) / 2 + (i - k);
}

struct UpdParams {
    const double* G[MTK_MAXN];   // Grams of the factors (entries n and, with pprev, nprev not read)
    int N, C, n;
    const float* M;              // In x C
    int64_t In;
    float* Un;                   // In x C, overwritten (left as it is when H is not pd)
    int64_t rows;                // rows per CTA, a multiple of kUpdRows
    int gmode;                   // 0: no Gram of U_n; 1: partial Grams only; 2: G_n (and the fit)
    float2* part;                // [grid][npairs] this CTA's partial Gram (gmode >= 1)
    const float2* pprev;         // the previous update's partials (or null): G_nprev is reduced
    int Pprev, nprev;            // from them here, and written to Gprev by CTA 0
    double* Gprev;
    double* Gn;                  // gmode 2: the Gram of the new U_n
    float2* gsum;                // gmode 2: [groups][npairs]
    double* dots;                // gmode 2 with fit: [grid] partial <M, U_n>
    unsigned int* tk;            // gmode 2: tickets, zero on entry and on exit
    const double* normX2;        // gmode 2: the fit (else null)
    double* fit;
    double* r2;
    uint32_t* status;
};

// dynamic shared memory: A[C*C] doubles, then fin and fprev, C(C+1)/2 float2 each
__global__ void __launch_bounds__(kUpdThreads)
als_update_kernel(const __grid_constant__ UpdParams p) {
    extern __shared__ double dsm[];
    __shared__ double dinv[kUpdMaxC], rcp[kUpdMaxC];
    __shared__ double red[kUpdThreads / 32];
    __shared__ int tri[kMaxPairs];
    __shared__ float ur[kUpdRows][kUpdMaxC];
    __shared__ int flag;

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int C = p.C, N = p.N, n = p.n;
    const int npairs = C * (C + 1) / 2;
    double* A = dsm;
    float2* fin = reinterpret_cast<float2*>(dsm + C * C);
    float2* fprev = fin + npairs;

    build_pairs(tri, C);
    __syncthreads();
    // ---- G of the previous mode from its update's partials (written before the kernel
    // that precedes this one started)
    const bool prev = p.pprev != nullptr;
    if (prev) {
        sum_rows(p.pprev, p.Pprev, npairs, fprev);
        __syncthreads();
        if (blockIdx.x == 0) write_gram(fprev, tri, npairs, C, p.Gprev);
    }
    // ---- H = Hadamard_{k != n} G_k; the loads of one factor are issued together
    for (int e0 = t; e0 < C * C; e0 += 8 * kUpdThreads) {
        double h[8];
        bool first = true;
        for (int k = 0; k < N; ++k) {
            if (k == n) continue;
            double g[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = e0 + q * kUpdThreads;
                if (e < C * C) {
                    if (prev && k == p.nprev) {
                        const float2 v = fprev[pair_index(e / C, e % C, C)];
                        g[q] = (double)v.x + (double)v.y;
                    } else {
                        g[q] = p.G[k][e];
                    }
                } else {
                    g[q] = 0.0;
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) h[q] = first ? g[q] : h[q] * g[q];
            first = false;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (e0 + q * kUpdThreads < C * C) A[e0 + q * kUpdThreads] = h[q];
    }
    __syncthreads();

    // ---- division-free L D L^T (lower triangle), one barrier per step
    bool bad = false;
    for (int j = 0; j < C; ++j) {
        const double d = A[j * C + j];
        const int ed = (int)((__double_as_longlong(d) >> 52) & 0x7FF);
        if (!(d > 0.0) || ed == 0 || ed == 0x7FF) {     // same value in every thread
            bad = true;
            break;
        }
        const int ej = ed - 1023;
        const int m = C - 1 - j;
        const int cnt = m * (m + 1) / 2;
#pragma unroll 3
        for (int x = t; x < cnt; x += kUpdThreads) {
            const int i = tri[x] >> 8, k = tri[x] & 255;
            const double v = A[i * C + j] * A[k * C + j];
            A[i * C + k] = scale_exp2(fma(d, A[i * C + k], -v), ej);
        }
        __syncthreads();
    }
    if (bad && blockIdx.x == 0 && t == 0) set_status(p.status, MTK_ENOTPD);
    if (!bad) {
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
        // L(i, k) = A(i, k) / d_k for i > k, kept in both triangles: A[k][i] = A[i][k] = L(i, k)
#pragma unroll 4
        for (int x = t; x < npairs; x += kUpdThreads) {
            const int i = tri[x] >> 8, k = tri[x] & 255;
            if (i > k) {
                const double l = A[i * C + k] * rcp[k];
                A[i * C + k] = l;
                A[k * C + i] = l;
            }
        }
        __syncthreads();
    }

    // ---- M is written by the previous kernel
    asm volatile("griddepcontrol.wait;" ::: "memory");

    const bool gram = p.gmode >= 1;
    const bool fit = p.gmode == 2 && p.normX2 != nullptr;
    const int64_t r0 = (int64_t)blockIdx.x * p.rows;
    const int64_t r1 = (r0 + p.rows < p.In) ? r0 + p.rows : p.In;
    float gh[kPairsPerThread], gl[kPairsPerThread];
#pragma unroll
    for (int q = 0; q < kPairsPerThread; ++q) gh[q] = gl[q] = 0.0f;
    double dot = 0.0;
    const int j0 = lane, j1 = lane + 32;
    for (int64_t rb = r0; rb < r1; rb += kUpdRows) {
        const int64_t i = rb + warp;
        float u0 = 0.0f, u1 = 0.0f;
        if (i < r1) {
            const float* mrow = p.M + i * C;
            float* urow = p.Un + i * C;
            const float m0 = j0 < C ? mrow[j0] : 0.0f;
            const float m1 = j1 < C ? mrow[j1] : 0.0f;
            if (!bad) {
                double s0 = (double)m0, s1 = (double)m1;
                if (C <= 32) {
                    for (int k = 0; k < C; ++k) {             // L y = m
                        const double y = __shfl_sync(0xffffffffu, s0, k);
                        if (j0 > k && j0 < C) s0 = fma(-A[k * C + j0], y, s0);
                    }
                    s0 *= dinv[j0 < C ? j0 : 0];              // z = D^{-1} y
                    for (int k = C - 1; k >= 0; --k) {        // L^T u = z
                        const double y = __shfl_sync(0xffffffffu, s0, k);
                        if (j0 < k) s0 = fma(-A[k * C + j0], y, s0);
                    }
                } else {
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
                        if (j1 < k) s1 = fma(-A[k * C + j1], y, s1);
                    }
                }
                u0 = (float)s0;
                u1 = (float)s1;
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
        const int nr = (r1 - rb) < kUpdRows ? (int)(r1 - rb) : kUpdRows;
#pragma unroll
        for (int q = 0; q < kPairsPerThread; ++q) {
            const int x = t + q * kUpdThreads;
            if (x < npairs) {
                const int a = tri[x] >> 8, b = tri[x] & 255;
                for (int r = 0; r < nr; ++r) df_madd(gh[q], gl[q], ur[r][a], ur[r][b]);
            }
        }
        __syncthreads();
    }
    if (!gram) return;

    // ---- partial Gram (and partial <M, U_n>) of this CTA
    float2* prow = p.part + (size_t)blockIdx.x * npairs;
#pragma unroll
    for (int q = 0; q < kPairsPerThread; ++q) {
        const int x = t + q * kUpdThreads;
        if (x < npairs) {
            df_renorm(gh[q], gl[q]);
            prow[x] = make_float2(gh[q], gl[q]);
        }
    }
    if (p.gmode == 1) return;
    if (fit) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
        if (lane == 0) red[warp] = dot;
        __syncthreads();
        if (t == 0) p.dots[blockIdx.x] = (red[0] + red[1]) + (red[2] + red[3]);
    }
    if (!ticket_reduce(p.part, p.gsum, fin, p.tk + kTicketUpd, (int)blockIdx.x, (int)gridDim.x, npairs, &flag))
        return;
    write_gram(fin, tri, npairs, C, p.Gn);
    if (!fit) return;
    // ---- fit: y2 = sum_ab prod_k G_k(a, b) with the new G_n (fin) and, when it was reduced
    // here, the previous mode's G (fprev; CTA 0's global copy may not be written yet);
    // <M, U_n> from the partials
    double v = 0.0;
    for (int e0 = t; e0 < C * C; e0 += 8 * kUpdThreads) {
        double h[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = e0 + q * kUpdThreads;
            if (e < C * C) {
                const float2 w = fin[pair_index(e / C, e % C, C)];
                h[q] = (double)w.x + (double)w.y;
            } else {
                h[q] = 0.0;
            }
        }
        for (int k = 0; k < N; ++k) {
            if (k == n) continue;
            double g[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = e0 + q * kUpdThreads;
                if (e >= C * C) {
                    g[q] = 0.0;
                } else if (prev && k == p.nprev) {
                    const float2 w = fprev[pair_index(e / C, e % C, C)];
                    g[q] = (double)w.x + (double)w.y;
                } else {
                    g[q] = p.G[k][e];
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) h[q] *= g[q];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) v += h[q];
    }
    double ds = 0.0;
    for (int b = t; b < (int)gridDim.x; b += kUpdThreads) ds += __ldcg(p.dots + b);
    v -= 2.0 * ds;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (t == 0) {
        const double nx2 = *p.normX2;
        const double r2 = nx2 + ((red[0] + red[1]) + (red[2] + red[3]));
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
    int64_t P = (In + kUpdRows - 1) / kUpdRows;
    int64_t r = kUpdRows;
    if (P > kUpdMaxCtas) {
        r = ((In + kUpdMaxCtas - 1) / kUpdMaxCtas + kUpdRows - 1) / kUpdRows * kUpdRows;
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

// two partial buffers (consecutive updates alternate), the ticket groups' sums, the dots
size_t als_update_scratch_bytes(int Pmax, int C) {
    const int ng = (Pmax + kGroup - 1) / kGroup;
    return 2 * rup((size_t)Pmax * pair_bytes(C), 256) + rup((size_t)ng * pair_bytes(C), 256) +
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
    if (P > a.Pmax || (a.prevP > a.Pmax)) return cudaErrorInvalidValue;
    const size_t pb = rup((size_t)a.Pmax * pair_bytes(a.C), 256);
    const int ng = (a.Pmax + kGroup - 1) / kGroup;
    char* w = static_cast<char*>(a.scratch);
    float2* buf[2] = {reinterpret_cast<float2*>(w), reinterpret_cast<float2*>(w + pb)};
    p.gmode = a.gmode;
    p.part = buf[a.parity & 1];
    if (a.prevP > 0) {
        p.pprev = buf[(a.parity & 1) ^ 1];
        p.Pprev = a.prevP;
        p.nprev = a.nprev;
        p.Gprev = a.Gprev;
    }
    p.Gn = a.Gn;
    p.gsum = reinterpret_cast<float2*>(w + 2 * pb);
    p.dots = reinterpret_cast<double*>(w + 2 * pb + rup((size_t)ng * pair_bytes(a.C), 256));
    p.tk = a.tickets;
    p.normX2 = a.gmode == 2 ? a.normX2 : nullptr;
    p.fit = a.fit;
    p.r2 = a.r2;
    p.status = a.status;
    const size_t smem = (size_t)a.C * a.C * sizeof(double) + 2 * pair_bytes(a.C);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(als_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)P);
    cfg.blockDim = dim3(kUpdThreads);
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
