// krp.cu -- row-parallel Khatri-Rao product (Section 4.1, Algorithm 1).
//
// K = U_0 kr ... kr U_{Z-1}, row j <-> multi-index (a_0, ..., a_{Z-1}) with the
// last operand's index fastest (Section 2.1 row rule).  K is row-major, so the
// J_{Z-1} rows that share one "prefix" (a_0..a_{Z-2}) form one contiguous run
// of J_{Z-1}*C floats.
//
// Parallel variant (Section 4.1.2): each CTA owns a contiguous block of rows.
// It first forms, once per CTA, the prefix products P(p, :) = U_0(a_0,:) * ... *
// U_{Z-2}(a_{Z-2},:) of the prefixes its block touches and keeps them in shared
// memory (the partial Hadamard products that Algorithm 1 keeps in its matrix
// P), then streams its rows as K(j, :) = P(p, :) * U_{Z-1}(a_{Z-1}, :): one
// multiply per output entry, the prefix work amortised over the J_{Z-1} rows
// that share it.  The kernel is HBM-write-bound; stores are coalesced over the
// flat output.
// The naive comparator (Section 5.2) forms every entry from all Z operands.
#include "mtk_internal.cuh"

namespace mtk {
namespace {

struct KrpArgs {
    int Z, C;
    const float* U[MTK_MAXN];
    int64_t rows[MTK_MAXN];
    int64_t J;        // total rows
    float* K;
};

constexpr int kKrpSmemFloats = 8192;   // prefix products per CTA (32 KB)

__global__ void __launch_bounds__(256) krp_reuse_kernel(const __grid_constant__ KrpArgs a) {
    __shared__ float P[kKrpSmemFloats];
    const int C = a.C, Z = a.Z;
    const int64_t Jl = a.rows[Z - 1];                  // rows of the last operand
    const int64_t RB = (kKrpSmemFloats / C) & ~3LL;    // rows per block (multiple of 4)
    const int64_t nblk = (a.J + RB - 1) / RB;
    const int64_t Jp2 = (Z >= 2) ? a.rows[Z - 2] : 1;  // rows of the second-to-last operand
    for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int64_t j0 = blk * RB;
        const int64_t j1 = (j0 + RB < a.J) ? j0 + RB : a.J;
        const int64_t p0 = j0 / Jl, p1 = (j1 - 1) / Jl;
        const int np = (int)(p1 - p0 + 1);            // <= RB prefixes
        __syncthreads();
        // prefix products: P(p) = Q(p / Jp2) * U_{Z-2}(p % Jp2) with Q the product of
        // operands 0..Z-3 (shared by Jp2 consecutive prefixes)
        for (int e = threadIdx.x; e < np * C; e += blockDim.x) {
            const int pl = e / C, c = e % C;
            const int64_t pg = p0 + pl;
            float v = 1.0f;
            if (Z >= 2) {
                int64_t q = pg / Jp2;
                v = __ldg(a.U[Z - 2] + (pg % Jp2) * C + c);
                for (int z = Z - 3; z >= 0; --z) {     // digits of q, operand Z-3 fastest
                    const int64_t d = q % a.rows[z];
                    q /= a.rows[z];
                    v *= __ldg(a.U[z] + d * C + c);
                }
            }
            P[pl * C + c] = v;
        }
        __syncthreads();
        // stream the block's rows: flat index e = j*C + c, tracked incrementally
        const float* Ul = a.U[Z - 1];
        const int64_t e0 = j0 * C, e1 = j1 * C;
        int64_t e = e0 + threadIdx.x;
        int64_t j = e / C;
        int c = (int)(e % C);
        const int step = blockDim.x;
        const int64_t dj = step / C;
        const int dc = step % C;
        for (; e < e1; e += step) {
            const int64_t pg = j / Jl, t = j - pg * Jl;
            a.K[e] = P[(int)(pg - p0) * C + c] * __ldg(Ul + t * C + c);
            j += dj;
            c += dc;
            if (c >= C) { c -= C; ++j; }
        }
    }
}

__global__ void __launch_bounds__(256) krp_naive_kernel(const __grid_constant__ KrpArgs a) {
    const int64_t n = a.J * a.C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = e / a.C;
        const int c = (int)(e % a.C);
        float v = 1.0f;
        for (int z = a.Z - 1; z >= 0; --z) {
            const int64_t d = j % a.rows[z];
            j /= a.rows[z];
            v *= __ldg(a.U[z] + d * a.C + c);
        }
        a.K[e] = v;
    }
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
    if (reuse) {
        const int64_t RB = (kKrpSmemFloats / C) & ~3LL;
        int64_t nblk = (a.J + RB - 1) / RB;
        int grid = (int)(nblk < 152 * 8 ? nblk : 152 * 8);
        krp_reuse_kernel<<<grid, 256, 0, s>>>(a);
        note_launches(1);
    } else {
        const int64_t n = a.J * C;
        int64_t blocks = (n + 255) / 256;
        int grid = (int)(blocks < 152 * 16 ? blocks : 152 * 16);
        krp_naive_kernel<<<grid, 256, 0, s>>>(a);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace mtk
