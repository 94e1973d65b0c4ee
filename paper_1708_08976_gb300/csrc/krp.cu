// krp.cu -- row-parallel Khatri-Rao product (Section 4.1, Algorithm 1).
//
// K = U_0 kr ... kr U_{Z-1}, row j <-> multi-index (a_0, ..., a_{Z-1}) with the
// last operand's index fastest (Section 2.1 row rule).  K is row-major, so the
// J_{Z-1} rows that share one "prefix" (a_0..a_{Z-2}) form one contiguous run
// of J_{Z-1}*C floats.
//
// Parallel variant (Section 4.1.2): each CTA owns a tile of consecutive rows.  It
// first forms, once per tile, the prefix products P(p, :) = U_0(a_0,:) * ... *
// U_{Z-2}(a_{Z-2},:) of the prefixes the tile touches and keeps them in shared
// memory (the partial Hadamard products that Algorithm 1 keeps in its matrix P),
// then streams the tile's rows as K(j, :) = P(p, :) * U_{Z-1}(a_{Z-1}, :): one
// multiply per output entry, the prefix work amortised over the J_{Z-1} rows that
// share it.
//
// The kernel is bound by the HBM write of K.  A warp writes four consecutive rows
// (4 C floats, a whole number of 16-byte words) per step: lane q stores word q of the
// four rows with one 16-byte store, so every store instruction covers one contiguous
// run of the output.  Which row and column each of the lane's four floats belongs to
// is fixed for the lane; the rows' (prefix, last index) pairs advance by counters, so
// the streaming loop has no integer division.  An output that is not 16-byte aligned
// takes the same loop with scalar stores.
//
// The naive comparator (Section 5.2) runs the same loop but forms every entry from
// all Z operands (Z - 1 multiplies per entry, no shared prefix products).
#include "mtk_internal.cuh"

namespace mtk {
namespace {

constexpr int kKrpThreads = 256;
constexpr int kKrpWarps = kKrpThreads / 32;
constexpr int kKrpTileFloats = 16384;      // output floats per tile (64 KB)
constexpr int kKrpMaxTileRows = 4096;

struct KrpArgs {
    int Z, C;
    const float* U[MTK_MAXN];
    int64_t rows[MTK_MAXN];
    int64_t J;        // total rows
    int64_t RT;       // rows per tile, a multiple of 4
    float* K;
    int vec;          // K is 16-byte aligned: 16-byte stores
};

// The (row, column) of float i of 16-byte word q inside a group of four rows (4 C floats
// = C words), packed as row << 16 | column.
__device__ __forceinline__ int word_float(int q, int i, int C) {
    const int e = 4 * q + i;
    const int r = e / C;
    return (r << 16) | (e - r * C);
}

// Row cursor: row jb as (pb, tb) = (jb / Jl, jb % Jl), advanced by a constant number
// of rows S = qS * Jl + rS without division.
struct Cursor {
    int64_t pb, tb;
};
__device__ __forceinline__ void cursor_advance(Cursor& c, int64_t qS, int64_t rS, int64_t Jl) {
    c.pb += qS;
    c.tb += rS;
    if (c.tb >= Jl) {
        c.tb -= Jl;
        ++c.pb;
    }
}
// (p, t) of row jb + r, 0 <= r < 4
__device__ __forceinline__ void cursor_row(const Cursor& c, int r, int64_t Jl, int64_t& p, int64_t& t) {
    p = c.pb;
    t = c.tb + r;
    while (t >= Jl) {
        t -= Jl;
        ++p;
    }
}

// dynamic shared memory: the tile's prefix products, [prefixes][C]
__global__ void __launch_bounds__(kKrpThreads) krp_reuse_kernel(const __grid_constant__ KrpArgs a) {
    extern __shared__ float P[];
    const int C = a.C, Z = a.Z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t Jl = a.rows[Z - 1];                  // rows of the last operand
    const int64_t Jp2 = (Z >= 2) ? a.rows[Z - 2] : 1;  // rows of the second-to-last operand
    const float* Ul = a.U[Z - 1];
    const int64_t ntiles = (a.J + a.RT - 1) / a.RT;
    const int64_t S = 4 * kKrpWarps;                   // rows per step of a warp
    const int64_t qS = S / Jl, rS = S % Jl;
    int rc0[4];                                        // this lane's word q = lane
#pragma unroll
    for (int i = 0; i < 4; ++i) rc0[i] = word_float(lane, i, C);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t j0 = tile * a.RT;
        const int64_t j1 = (j0 + a.RT < a.J) ? j0 + a.RT : a.J;
        const int64_t p0 = j0 / Jl, p1 = (j1 - 1) / Jl;
        const int np = (int)(p1 - p0 + 1);
        __syncthreads();
        // prefix products: P(p) = Q(p / Jp2) * U_{Z-2}(p % Jp2), Q the product of operands
        // 0..Z-3 at the digits of p / Jp2 (operand Z-3 fastest)
        for (int e = threadIdx.x; e < np * C; e += kKrpThreads) {
            const int pl = e / C, c = e - pl * C;
            const int64_t pg = p0 + pl;
            float v = 1.0f;
            if (Z >= 2) {
                int64_t q = pg / Jp2;
                v = __ldg(a.U[Z - 2] + (pg - q * Jp2) * C + c);
                for (int z = Z - 3; z >= 0; --z) {
                    const int64_t nq = q / a.rows[z];
                    v *= __ldg(a.U[z] + (q - nq * a.rows[z]) * C + c);
                    q = nq;
                }
            }
            P[e] = v;
        }
        __syncthreads();
        // stream the tile: warp w takes the groups of four rows w, w + 8, ...
        Cursor cur;
        {
            const int64_t jb = j0 + 4 * warp;
            cur.pb = jb / Jl;
            cur.tb = jb - cur.pb * Jl;
        }
        for (int64_t jb = j0 + 4 * warp; jb < j1; jb += S) {
            const int64_t nr = (j1 - jb) < 4 ? (j1 - jb) : 4;    // rows of this group
            float* dst = a.K + jb * C;
            for (int q = lane; q < C; q += 32) {
                float v[4];
                int ri[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int rc = q == lane ? rc0[i] : word_float(q, i, C);
                    ri[i] = rc >> 16;
                    const int ci = rc & 0xFFFF;
                    v[i] = 0.0f;
                    if (ri[i] < nr) {
                        int64_t p, t;
                        cursor_row(cur, ri[i], Jl, p, t);
                        v[i] = P[(int)(p - p0) * C + ci] * __ldg(Ul + t * C + ci);
                    }
                }
                if (a.vec && nr == 4) {
                    *reinterpret_cast<float4*>(dst + 4 * q) = make_float4(v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (ri[i] < nr) dst[4 * q + i] = v[i];
                }
            }
            cursor_advance(cur, qS, rS, Jl);
        }
    }
}

// Naive comparator: every entry from all Z operands.  The row's digits (a_0..a_{Z-1})
// advance with the group by mixed-radix addition of the step's digits.
template <int ZT>
__global__ void __launch_bounds__(kKrpThreads) krp_naive_kernel(const __grid_constant__ KrpArgs a) {
    const int C = a.C;
    constexpr int ZM = ZT > 0 ? ZT : MTK_MAXN;
    const int Z = ZT > 0 ? ZT : a.Z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t S = 4 * (int64_t)kKrpWarps * gridDim.x;  // rows per step of a warp
    int64_t sd[ZM], d[ZM];
    {
        int64_t s = S, j = 4 * ((int64_t)blockIdx.x * kKrpWarps + warp);
#pragma unroll
        for (int z = ZM - 1; z >= 0; --z) {
            if (z >= Z) continue;
            const int64_t r = a.rows[z];
            sd[z] = s % r;
            s /= r;
            d[z] = j % r;
            j /= r;
        }
    }
    int rc0[4];                                        // this lane's word q = lane
#pragma unroll
    for (int i = 0; i < 4; ++i) rc0[i] = word_float(lane, i, C);
    for (int64_t jb = 4 * ((int64_t)blockIdx.x * kKrpWarps + warp); jb < a.J; jb += S) {
        const int64_t nr = (a.J - jb) < 4 ? (a.J - jb) : 4;
        float* dst = a.K + jb * C;
        for (int q = lane; q < C; q += 32) {
            float v[4];
            int ri[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rc = q == lane ? rc0[i] : word_float(q, i, C);
                ri[i] = rc >> 16;
                const int ci = rc & 0xFFFF;
                v[i] = 0.0f;
                if (ri[i] < nr) {
                    // digits of row jb + ri: add ri to the last digit, carry upwards
                    int64_t e[ZM];
                    int64_t carry = ri[i];
#pragma unroll
                    for (int z = ZM - 1; z >= 0; --z) {
                        if (z >= Z) continue;
                        int64_t x = d[z] + carry;
                        carry = 0;
                        while (x >= a.rows[z]) {
                            x -= a.rows[z];
                            ++carry;
                        }
                        e[z] = x;
                    }
                    float prod = 1.0f;
#pragma unroll
                    for (int z = 0; z < ZM; ++z)
                        if (z < Z) prod *= __ldg(a.U[z] + e[z] * C + ci);
                    v[i] = prod;
                }
            }
            if (a.vec && nr == 4) {
                *reinterpret_cast<float4*>(dst + 4 * q) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (ri[i] < nr) dst[4 * q + i] = v[i];
            }
        }
        // next group: d += sd (mixed radix, every digit of sd below its radix)
        int64_t carry = 0;
#pragma unroll
        for (int z = ZM - 1; z >= 0; --z) {
            if (z >= Z) continue;
            int64_t x = d[z] + sd[z] + carry;
            carry = 0;
            if (x >= a.rows[z]) {
                x -= a.rows[z];
                carry = 1;
            }
            d[z] = x;
        }
    }
}

template <int ZT>
void naive_launch(const KrpArgs& a, int grid, cudaStream_t s) {
    krp_naive_kernel<ZT><<<grid, kKrpThreads, 0, s>>>(a);
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
    a.vec = (reinterpret_cast<uintptr_t>(K) & 15) == 0 ? 1 : 0;
    if (a.J == 0) return cudaSuccess;
    int64_t RT = (kKrpTileFloats / C) & ~(int64_t)3;
    if (RT < 4) RT = 4;
    if (RT > kKrpMaxTileRows) RT = kKrpMaxTileRows;
    a.RT = RT;
    if (reuse) {
        // a tile of RT rows touches at most RT / J_{Z-1} + 2 prefixes
        const int64_t Jl = rows[Z - 1];
        int64_t np = RT / Jl + 2;
        if (np > RT) np = RT;
        const size_t smem = (size_t)np * C * sizeof(float);
        if (smem > 48 * 1024) {
            const cudaError_t e =
                cudaFuncSetAttribute(krp_reuse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        const int64_t ntiles = (a.J + RT - 1) / RT;
        const int grid = (int)(ntiles < num_sms() * 4 ? ntiles : num_sms() * 4);
        krp_reuse_kernel<<<grid, kKrpThreads, smem, s>>>(a);
        note_launches(1);
    } else {
        const int64_t groups = (a.J + 3) / 4;
        const int64_t blocks = (groups + kKrpWarps - 1) / kKrpWarps;
        const int grid = (int)(blocks < num_sms() * 8 ? blocks : num_sms() * 8);
        switch (Z) {
            case 1: naive_launch<1>(a, grid, s); break;
            case 2: naive_launch<2>(a, grid, s); break;
            case 3: naive_launch<3>(a, grid, s); break;
            case 4: naive_launch<4>(a, grid, s); break;
            default: naive_launch<0>(a, grid, s); break;
        }
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace mtk
