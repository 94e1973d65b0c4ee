// krp.cu -- row-parallel Khatri-Rao product (Section 4.1, Algorithm 1).
//
// K = U_0 kr ... kr U_{Z-1}, row j <-> multi-index (a_0, ..., a_{Z-1}) with the
// last operand's index fastest (Section 2.1 row rule).  K is row-major, so the
// J_{Z-1} rows that share one "prefix" (a_0..a_{Z-2}) form one contiguous run
// of J_{Z-1}*C floats.
//
// Parallel variant (Section 4.1.2): every warp owns a contiguous range of rows and
// writes them four at a time (4 C floats, a whole number of 16-byte words): lane q
// stores word q of each group of four rows with one 16-byte store.  The row and column
// of each of the lane's four floats are therefore fixed, and from one group to the next
// the lane's rows move by 4: their last-operand index advances by a counter, and the
// prefix product P(p, c) = U_0(a_0, c) * ... * U_{Z-2}(a_{Z-2}, c) that Algorithm 1
// keeps is held in a register per float, formed again only when the float's row enters
// a new prefix (every J_{Z-1} rows).  Each entry then costs one load of U_{Z-1} and one
// multiply: the prefix work is shared by the J_{Z-1} rows of a run.  The kernel is bound
// by the HBM write of K.
//
// The naive comparator (Section 5.2) walks the same rows but forms every entry from all
// Z operands (Z loads and Z - 1 multiplies per entry), its digits (a_0..a_{Z-1})
// advanced by mixed-radix increments.
//
// Lanes take 16-byte words q = lane and q = lane + 32 of each group (C <= 64); wider
// outputs and outputs that are not 16-byte aligned take the generic loop (scalar
// stores, digits per float).
#include "mtk_internal.cuh"

namespace mtk {
namespace {

constexpr int kKrpThreads = 256;
constexpr int kKrpWarps = kKrpThreads / 32;

struct KrpArgs {
    int Z, C;
    const float* U[MTK_MAXN];
    int64_t rows[MTK_MAXN];
    int64_t J;        // total rows
    float* K;
};

// groups of four rows [g0, g1) of warp w of nw in all: a balanced split
__device__ __forceinline__ void warp_groups(int64_t J, int64_t w, int64_t nw, int64_t& g0, int64_t& g1) {
    const int64_t G = (J + 3) / 4;
    g0 = G * w / nw;
    g1 = G * (w + 1) / nw;
}

// digits of row j over the operands (last operand fastest), each kept as its row's
// offset d * C into the operand (every operand has rows * C < 2^31 on this path)
template <int ZM>
__device__ __forceinline__ void row_offsets(const KrpArgs& a, int Z, int64_t j, int* o) {
#pragma unroll
    for (int z = ZM - 1; z >= 0; --z) {
        if (z >= Z) continue;
        const int64_t q = j / a.rows[z];
        o[z] = (int)(j - q * a.rows[z]) * a.C;
        j = q;
    }
}

// P(p, c) from the prefix rows' offsets o[0..Z-2]
template <int ZM>
__device__ __forceinline__ float prefix_value(const KrpArgs& a, int Z, const int* o, int c) {
    float v = 1.0f;
#pragma unroll
    for (int z = 0; z < ZM - 1; ++z)
        if (z < Z - 1) v *= __ldg(a.U[z] + o[z] + c);
    return v;
}

// the last operand's digit wrapped: carry into the prefix digits (mixed radix)
template <int ZM>
__device__ __forceinline__ void prefix_carry(const KrpArgs& a, int Z, int* o) {
#pragma unroll
    for (int z = ZM - 2; z >= 0; --z) {
        if (z >= Z - 1) continue;
        o[z] += a.C;
        if (o[z] < (int)a.rows[z] * a.C) break;
        o[z] = 0;
    }
}

// Fast path: C <= 64, K 16-byte aligned.  REUSE: Algorithm 1; else the naive comparator.
template <int ZT, bool REUSE>
__global__ void __launch_bounds__(kKrpThreads) krp_words_kernel(const __grid_constant__ KrpArgs a) {
    constexpr int ZM = ZT > 0 ? ZT : MTK_MAXN;
    const int Z = ZT > 0 ? ZT : a.Z;
    const int C = a.C;
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * kKrpWarps + (threadIdx.x >> 5);
    int64_t g0, g1;
    warp_groups(a.J, w, (int64_t)gridDim.x * kKrpWarps, g0, g1);
    if (g0 >= g1) return;
    const int64_t Jl = a.rows[Z - 1];
    const float* Ul = a.U[Z - 1];
    for (int q = lane; q < C; q += 32) {
        // the lane's four floats of word q: row offset ri (0..3) and column ci in a group
        int ri[4], ci[4];
        int o[4][ZM];               // offsets of the float's row in every operand (d * C)
        float pv[4];                // REUSE: P(prefix, ci)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int f = 4 * q + e;
            ri[e] = f / C;
            ci[e] = f - ri[e] * C;
            row_offsets<ZM>(a, Z, 4 * g0 + ri[e], o[e]);
            pv[e] = REUSE ? prefix_value<ZM>(a, Z, o[e], ci[e]) : 1.0f;
        }
        const int JlC = (int)Jl * C, step = 4 * C;
        float* dst = a.K + 4 * g0 * C + 4 * q;
        for (int64_t g = g0; g < g1; ++g) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (REUSE) {
                    v[e] = pv[e] * __ldg(Ul + o[e][Z - 1] + ci[e]);
                } else {
                    float prod = __ldg(Ul + o[e][Z - 1] + ci[e]);
#pragma unroll
                    for (int z = 0; z < ZM - 1; ++z)
                        if (z < Z - 1) prod *= __ldg(a.U[z] + o[e][z] + ci[e]);
                    v[e] = prod;
                }
            }
            if (4 * g + 3 < a.J) {
                *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * g + ri[e] < a.J) dst[e] = v[e];
            }
            dst += 4 * C;
            // next group: every row moves by 4
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int& ol = o[e][Z - 1];
                ol += step;
                if (ol >= JlC) {
                    do {
                        ol -= JlC;
                        prefix_carry<ZM>(a, Z, o[e]);
                    } while (ol >= JlC);
                    if (REUSE && g + 1 < g1) pv[e] = prefix_value<ZM>(a, Z, o[e], ci[e]);
                }
            }
        }
    }
}

// Generic loop: any C and alignment; one float per thread step, digits per float (the
// same products for both forms).
__global__ void __launch_bounds__(kKrpThreads) krp_generic_kernel(const __grid_constant__ KrpArgs a) {
    const int64_t n = a.J * a.C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = e / a.C;
        const int c = (int)(e - j * a.C);
        float v = 1.0f;
        for (int z = a.Z - 1; z >= 0; --z) {
            const int64_t q = j / a.rows[z];
            v *= __ldg(a.U[z] + (j - q * a.rows[z]) * a.C + c);
            j = q;
        }
        a.K[e] = v;
    }
}

template <int ZT>
void words_launch(const KrpArgs& a, bool reuse, int grid, cudaStream_t s) {
    if (reuse) krp_words_kernel<ZT, true><<<grid, kKrpThreads, 0, s>>>(a);
    else krp_words_kernel<ZT, false><<<grid, kKrpThreads, 0, s>>>(a);
}

}  // namespace

cudaError_t launch_krp(const float* const* U, const int64_t* rows, int Z, int C, float* K,
                       int reuse, cudaStream_t s) {
    KrpArgs a;
    a.Z = Z;
    a.C = C;
    a.J = 1;
    for (int z = 0; z < MTK_MAXN; ++z) { a.U[z] = nullptr; a.rows[z] = 1; }
    for (int z = 0; z < Z; ++z) { a.U[z] = U[z]; a.rows[z] = rows[z]; a.J *= rows[z]; }
    a.K = K;
    if (a.J == 0) return cudaSuccess;
    bool fast = (reinterpret_cast<uintptr_t>(K) & 15) == 0 && C <= 64;
    for (int z = 0; z < Z; ++z)
        if (rows[z] * C + 4 * (int64_t)C >= ((int64_t)1 << 31)) fast = false;
    if (fast) {
        // warps: up to 64 per SM, each with at least 16 groups of four rows
        const int64_t groups = (a.J + 3) / 4;
        int64_t warps = (groups + 15) / 16;
        const int64_t cap = (int64_t)num_sms() * 64;
        if (warps > cap) warps = cap;
        const int grid = (int)((warps + kKrpWarps - 1) / kKrpWarps);
        switch (Z) {
            case 1: words_launch<1>(a, reuse != 0, grid, s); break;
            case 2: words_launch<2>(a, reuse != 0, grid, s); break;
            case 3: words_launch<3>(a, reuse != 0, grid, s); break;
            case 4: words_launch<4>(a, reuse != 0, grid, s); break;
            default: words_launch<0>(a, reuse != 0, grid, s); break;
        }
    } else {
        const int64_t n = a.J * C;
        int64_t blocks = (n + kKrpThreads - 1) / kKrpThreads;
        const int grid = (int)(blocks < num_sms() * 16 ? blocks : num_sms() * 16);
        krp_generic_kernel<<<grid, kKrpThreads, 0, s>>>(a);
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace mtk
