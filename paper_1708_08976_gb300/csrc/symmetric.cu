// symmetric.cu -- tensors symmetric in modes 0 and 1, stored packed (the paper's 3-D fMRI
// variant, Section 5.3.3: a symmetric pair of region modes of size n0 kept as one mode of the
// entries of one triangle, which halves the tensor).
//
// Packed layout, with diagonal (diag = 1): X(a, b, r) with a >= b (r = the flat index of
// modes 2..N-1) is kept at Xp[p + Pp r], p = a (a + 1) / 2 + b, n0 (n0 + 1) / 2 rows.
// Without it (diag = 0, the paper's n0 (n0 - 1) / 2 = 19,900 rows for n0 = 200: the
// diagonal of a correlation tensor is the constant 1 and carries nothing): a > b only,
// p = a (a - 1) / 2 + b, and the tensor is taken to be zero on its diagonal.  Either way
// Pp, the packed mode's size, is the row count rounded up to a multiple of 8 (so that the
// packed mode is a 16-byte aligned contiguous index), and from 2048 rows on to a multiple of
// 64 (at most 3% more), so that the rows (p, r) of the MN-major view of modes 0 and 1 start
// on 128-byte boundaries: with Pp = 20,104 their 128-byte pieces straddled two L2 lines,
// and that contraction ran at 0.79 of the copy bandwidth.  The padding rows hold zeros.
//
// The MTTKRP of the full tensor then reads only the packed entries:
//  - n >= 2: sum_{a, b} X(a, b, .) U_0(a, c) U_1(b, c) = sum_p Xp(p, .) W(p, c) with
//    W(p(a, b), c) = U_0(a, c) U_1(b, c) + U_0(b, c) U_1(a, c) for a > b and
//    U_0(a, c) U_1(a, c) for a = b: the MTTKRP of the packed tensor with W as its first
//    factor (sym_pair_kernel forms W);
//  - n = 0: M(a, c) = sum_b V(p(max(a, b), min(a, b)), c) U_1(b, c) with V the mode-0
//    MTTKRP of the packed tensor (sym_ttv_kernel; without diagonal the b = a term is
//    left out); n = 1 the same with U_0.
#include "mtk_internal.cuh"

namespace mtk {
namespace {

// a (a + 1) / 2 + b; the packed row of (a, b), a >= b, is tri_index(a - off, b) with
// off = 1 - diag
__device__ __forceinline__ int64_t tri_index(int64_t a, int64_t b) { return a * (a + 1) / 2 + b; }

// inverse of tri_index (p < n0 (n0 + 1) / 2) -> (a, b), a >= b: a first guess from an
// FP32 square root, made exact by integer steps
__device__ __forceinline__ void tri_pair(int64_t p, int64_t& a, int64_t& b) {
    int64_t s = (int64_t)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    if (s < 0) s = 0;
    while (s * (s + 1) / 2 > p) --s;
    while ((s + 1) * (s + 2) / 2 <= p) ++s;
    a = s;
    b = p - s * (s + 1) / 2;
}

__host__ __device__ __forceinline__ int64_t tri_rows(int64_t n0, int diag) {
    return diag ? n0 * (n0 + 1) / 2 : n0 * (n0 - 1) / 2;
}

// Xp from the full tensor X (n0 x n0 x rest, natural order): one thread per packed entry
__global__ void __launch_bounds__(256) sym_pack_kernel(const float* __restrict__ X, int64_t n0, int diag, int64_t Pp,
                                                       int64_t rest, float* __restrict__ Xp) {
    const int64_t P0 = tri_rows(n0, diag);
    const int64_t total = Pp * rest;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / Pp, p = e - r * Pp;
        float v = 0.0f;
        if (p < P0) {
            int64_t a, b;
            tri_pair(p, a, b);
            a += 1 - diag;
            v = X[a + n0 * b + n0 * n0 * r];
        }
        Xp[e] = v;
    }
}

// The same, by bands of 32 rows a of one slice r, for n0 <= kBandMaxN: the band's entries
// X(a, b, r), b <= a, are read with a fastest (128-byte runs), staged in shared memory and
// written row by row of a (each packed row contiguous, the band's rows one contiguous range
// of Xp), with no index decoding per entry.  The last band also writes the zero padding.
constexpr int kBandRows = 32;
constexpr int kBandMaxN = 320;
__global__ void __launch_bounds__(256) sym_pack_band_kernel(const float* __restrict__ X, int n0, int diag,
                                                            int64_t Pp, float* __restrict__ Xp) {
    __shared__ float T[kBandMaxN][kBandRows + 1];
    const int a0 = blockIdx.x * kBandRows;
    const int a1 = a0 + kBandRows < n0 ? a0 + kBandRows : n0;
    const int64_t r = blockIdx.y;
    const float* src = X + (int64_t)n0 * n0 * r;
    const int nb = diag ? a1 : a1 - 1;                   // columns b < nb hold the band's entries
    for (int e = threadIdx.x; e < nb * kBandRows; e += blockDim.x) {
        const int b = e / kBandRows, ao = e - b * kBandRows;
        if (a0 + ao < a1) T[b][ao] = src[(a0 + ao) + (int64_t)n0 * b];
    }
    __syncthreads();
    // one warp per row a of the band, lanes along its packed row (b = 0..a, or 0..a-1)
    float* dst = Xp + Pp * r;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int ao = warp; ao < a1 - a0; ao += (int)(blockDim.x >> 5)) {
        const int a = a0 + ao;
        const int len = diag ? a + 1 : a;
        float* row = dst + tri_rows(a, diag);           // the packed rows of the rows before a
        for (int b = lane; b < len; b += 32) row[b] = T[b][ao];
    }
    if (a1 == n0)
        for (int64_t p = tri_rows(n0, diag) + threadIdx.x; p < Pp; p += blockDim.x) dst[p] = 0.0f;
}

// W (Pp x C, row-major): the pair products of U_0 and U_1, symmetrised; zero padding rows
__global__ void __launch_bounds__(256) sym_pair_kernel(const float* __restrict__ U0, const float* __restrict__ U1,
                                                       int64_t n0, int diag, int64_t Pp, int C, float* __restrict__ W) {
    const int64_t P0 = tri_rows(n0, diag);
    const int64_t total = Pp * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / C;
        const int c = (int)(e - p * C);
        float v = 0.0f;
        if (p < P0) {
            int64_t a, b;
            tri_pair(p, a, b);
            a += 1 - diag;
            const float x = U0[a * C + c] * U1[b * C + c];
            v = a == b ? x : fmaf(U0[b * C + c], U1[a * C + c], x);
        }
        W[e] = v;
    }
}

// M(a, c) = sum_b V(p(max(a, b), min(a, b)), c) U(b, c): one warp per (a, c), lanes over
// b in order of b, then a fixed-order warp reduction
__global__ void __launch_bounds__(256) sym_ttv_kernel(const float* __restrict__ V, const float* __restrict__ U,
                                                      int64_t n0, int diag, int C, float* __restrict__ M) {
    const int lane = threadIdx.x & 31;
    const int off = 1 - diag;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = wid; item < n0 * C; item += nw) {
        const int64_t a = item / C;
        const int c = (int)(item - a * C);
        float s = 0.0f;
        for (int64_t b = lane; b < n0; b += 32) {
            if (off && b == a) continue;
            const int64_t p = a >= b ? tri_index(a - off, b) : tri_index(b - off, a);
            s = fmaf(V[p * C + c], U[b * C + c], s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) M[a * C + c] = s;
    }
}

int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int64_t sym_packed_rows(int64_t n0, int diag) {
    const int64_t rows = tri_rows(n0, diag);
    const int64_t m = rows >= 2048 ? 64 : 8;
    return (rows + m - 1) / m * m;
}

cudaError_t launch_sym_pack(const float* X, int64_t n0, int diag, int64_t rest, float* Xp, cudaStream_t s) {
    const int64_t Pp = sym_packed_rows(n0, diag);
    if (n0 <= kBandMaxN && rest <= 65535) {
        const dim3 grid((unsigned)((n0 + kBandRows - 1) / kBandRows), (unsigned)rest);
        sym_pack_band_kernel<<<grid, 256, 0, s>>>(X, (int)n0, diag, Pp, Xp);
        note_launches(1);
        return cudaGetLastError();
    }
    sym_pack_kernel<<<grid_for(Pp * rest, 256), 256, 0, s>>>(X, n0, diag, Pp, rest, Xp);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sym_pair(const float* U0, const float* U1, int64_t n0, int diag, int C, float* W, cudaStream_t s) {
    const int64_t Pp = sym_packed_rows(n0, diag);
    sym_pair_kernel<<<grid_for(Pp * C, 256), 256, 0, s>>>(U0, U1, n0, diag, Pp, C, W);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sym_ttv(const float* V, const float* U, int64_t n0, int diag, int C, float* M, cudaStream_t s) {
    sym_ttv_kernel<<<grid_for(n0 * C, 8), 256, 0, s>>>(V, U, n0, diag, C, M);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace mtk
