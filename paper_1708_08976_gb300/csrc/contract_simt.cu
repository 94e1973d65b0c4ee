// contract_simt.cu -- FP32 CUDA-core contraction D(i,c) = sum_k X3(k, i) W(k, c).
//
// This is the plain-FP32 form of the 1-step MTTKRP (Algorithms 2/3): the mode-n
// matricization is consumed in place as R row-major I x L blocks (Fig. 2), and
// the KRP rows W(k, :) are generated on chip from the factor rows (Algorithm 3
// forms K_R(j,:) kr K_L per block; here a block of 32 consecutive k is formed in
// shared memory and never written to HBM).  With a single materialised factor
// the same kernel is the GEMM of the materialised-KRP path and of the 2-step
// partial MTTKRP (Algorithm 4).
//
// Decomposition: grid = (i-tiles of 64, contraction splits S, column blocks of
// 32).  Each CTA owns a contiguous k-range (the private partial result of
// Algorithm 3), stages X tiles with 4-byte cp.async (zero-filled outside the
// tensor) through a 3-deep ring, and accumulates an 8 x 4 register tile per
// thread; four k-groups per CTA are summed in shared memory in fixed order.
// Partials of the S splits are summed in split order by split_reduce_kernel
// (the parallel reduction of Algorithm 3), so results are deterministic.
#include "mtk_internal.cuh"

namespace mtk {
namespace {

constexpr int BK = 32;        // k per stage
constexpr int BI = 64;        // i per CTA tile
constexpr int NKG = 4;        // k-groups per CTA
constexpr int STAGES = 3;
constexpr int XP = BI + 4;    // padded row pitch of the X stage (floats)
constexpr int WP = 32 + 4;    // padded row pitch of the W stage

struct __align__(16) SimtSmem {
    union {
        struct {
            float xs[STAGES][BK][XP];
            float ws[2][BK][WP];
            float qs[2][32];
        } pipe;
        float red[NKG][BI][32];
    };
};

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
    unsigned saddr = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    int sz = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(saddr), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Q(q, c) = prod over tail factors of tail[t](digit_t(q), c)
__device__ __forceinline__ float tail_product(const KrpOperand& W, int64_t q, int c, int C) {
    float p = 1.0f;
    for (int t = 0; t < W.ntail; ++t) {
        const int64_t rad = W.tail_rad[t];
        const int64_t d = q % rad;
        q /= rad;
        p *= __ldg(W.tail[t] + d * C + c);
    }
    return p;
}

__global__ void __launch_bounds__(256)
contract_simt_kernel(const __grid_constant__ ContractParams p) {
    __shared__ SimtSmem sm;
    const int nCg = blockDim.x / 32;             // column groups of 4
    const int Cb = nCg * 4;                      // columns handled (>= real columns)
    const int t = threadIdx.x, nth = blockDim.x;
    const int tc = t % nCg, ti = (t / nCg) % 8, kg = t / (nCg * 8);
    const int64_t i0 = (int64_t)blockIdx.x * BI;
    const int sp = blockIdx.y;
    const int c0 = blockIdx.z * 32;
    const int C = p.C;
    const int64_t L = p.L, I = p.I;
    const int64_t kb = (int64_t)sp * p.kchunk;
    const int64_t ke = (kb + p.kchunk < p.K) ? kb + p.kchunk : p.K;
    const int nst = (int)((ke - kb + BK - 1) / BK);
    const bool kfast = L > 1;
    const KrpOperand& W = p.W;

    // uniform trackers of the stage start: (l, r) for X, (d0, q) for W
    int64_t xl = kb % L, xr = kb / L;            // X issue tracker
    int64_t wd = kb % W.rad0, wq = kb / W.rad0;  // W generation tracker
    int64_t qcached = -1;
    const int64_t qtot = p.K / W.rad0;           // number of q values (rows of Q)

    auto issue_x = [&](int s) {
        float* dst = &sm.pipe.xs[s % STAGES][0][0];
        const int64_t ks = kb + (int64_t)s * BK;
        for (int e = t; e < BK * BI; e += nth) {
            int kk, ii;
            if (kfast) { kk = e % BK; ii = e / BK; } else { ii = e % BI; kk = e / BI; }
            const int64_t k = ks + kk, i = i0 + ii;
            const bool valid = (k < ke) && (i < I);
            int64_t off = 0;
            if (valid) {
                if (L == 1) {
                    off = k * I;
                } else {
                    int64_t l = xl + kk, r = xr;
                    while (l >= L) { l -= L; ++r; }
                    off = l + L * I * r;
                }
                off += L * i;
            }
            cp_async4(dst + kk * XP + ii, p.X + off, valid);
        }
        cp_async_commit();
        if (L > 1) { xl += BK; while (xl >= L) { xl -= L; ++xr; } }
    };

    // W stage s into ws[s & 1]; needs Q rows for wq, wq+1 in qs
    auto gen_w = [&](int s) {
        float* dst = &sm.pipe.ws[s & 1][0][0];
        const int64_t ks = kb + (int64_t)s * BK;
        for (int e = t; e < BK * Cb; e += nth) {
            const int kk = e / Cb, cc = e % Cb;
            const int c = c0 + cc;
            float w = 0.0f;
            if (ks + kk < ke && c < C) {
                int64_t d = wd + kk;
                int which = 0;
                if (W.ntail > 0 && d >= W.rad0) { d -= W.rad0; which = 1; }
                w = __ldg(W.f0 + d * C + c);
                if (W.ntail > 0) w *= sm.pipe.qs[which][cc];
            }
            dst[kk * WP + cc] = w;
        }
    };
    auto advance_w = [&]() {
        wd += BK;
        while (wd >= W.rad0) { wd -= W.rad0; ++wq; }
    };
    // refresh the cached Q rows if the stage's q changed (uniform branch)
    auto refresh_q = [&]() {
        if (W.ntail > 0 && wq != qcached) {
            __syncthreads();
            for (int e = t; e < 2 * 32; e += nth) {
                const int which = e / 32, cc = e % 32, c = c0 + cc;
                sm.pipe.qs[which][cc] = (c < C && wq + which < qtot) ? tail_product(W, wq + which, c, C) : 0.0f;
            }
            qcached = wq;
            __syncthreads();
        }
    };

    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;

    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nst) issue_x(s); else cp_async_commit();
    }
    if (nst > 0) { refresh_q(); gen_w(0); }

    for (int s = 0; s < nst; ++s) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        if (s + STAGES - 1 < nst) issue_x(s + STAGES - 1); else cp_async_commit();

        const float* xs = &sm.pipe.xs[s % STAGES][0][0];
        const float* ws = &sm.pipe.ws[s & 1][0][0];
#pragma unroll
        for (int j = 0; j < BK / NKG; ++j) {
            const int kk = kg + NKG * j;
            const float4 xa = *reinterpret_cast<const float4*>(xs + kk * XP + ti * 8);
            const float4 xb = *reinterpret_cast<const float4*>(xs + kk * XP + ti * 8 + 4);
            const float4 w = *reinterpret_cast<const float4*>(ws + kk * WP + tc * 4);
            const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xv[a], wv[b], acc[a][b]);
        }
        if (s + 1 < nst) {
            advance_w();
            refresh_q();
            gen_w(s + 1);
        }
    }
    cp_async_wait<0>();
    __syncthreads();

    // fixed-order reduction over the k-groups
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) sm.red[kg][ti * 8 + a][tc * 4 + b] = acc[a][b];
    __syncthreads();
    for (int e = t; e < BI * Cb; e += nth) {
        const int ii = e / Cb, cc = e % Cb;
        const int64_t i = i0 + ii;
        const int c = c0 + cc;
        if (i >= I || c >= C) continue;
        float v = sm.red[0][ii][cc];
#pragma unroll
        for (int g = 1; g < NKG; ++g) v += sm.red[g][ii][cc];
        if (p.S == 1) p.out[i * p.out_si + c * p.out_sc] = v;
        else p.part[((int64_t)sp * I + i) * C + c] = v;
    }
}

__global__ void split_reduce_kernel(const float* __restrict__ part, int S, int64_t I, int C,
                                    float* __restrict__ out, int64_t si, int64_t sc) {
    const int64_t n = I * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.0f;
        for (int s = 0; s < S; ++s) v += part[(int64_t)s * n + e];
        const int64_t i = e / C, c = e % C;
        out[i * si + c * sc] = v;
    }
}

}  // namespace

cudaError_t launch_contract_simt(const ContractParams& p, int c_blocks, int i_tiles,
                                 cudaStream_t s) {
    const int Cfirst = p.C < 32 ? p.C : 32;
    const int nCg = (Cfirst + 3) / 4;
    dim3 grid(i_tiles, p.S, c_blocks);
    contract_simt_kernel<<<grid, nCg * 32, 0, s>>>(p);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_split_reduce(const float* part, int S, int64_t I, int C, float* out,
                                int64_t si, int64_t sc, cudaStream_t s) {
    const int64_t n = I * C;
    int blocks = (int)((n + 255) / 256);
    if (blocks > num_sms() * 8) blocks = num_sms() * 8;
    if (blocks < 1) blocks = 1;
    split_reduce_kernel<<<blocks, 256, 0, s>>>(part, S, I, C, out, si, sc);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace mtk
