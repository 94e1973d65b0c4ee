// multi_ttv.cu -- second step of the 2-step MTTKRP (Section 4.3, Algorithm 4).
//
// right ordering (after R = X_(0:n) K_R):   M(i,c) = sum_l T[l + L*i + L*I*c] * K_L(l,c)
//   One warp per output entry: the warp reads the contiguous run T[L*i + L*I*c ..+L)
//   with coalesced loads, multiplies by the strided column K_L(:,c) (L1-resident) and
//   reduces with warp shuffles in a fixed tree.
// left ordering (after L = X_(0:n-1)^T K_L): M(i,c) = sum_r T[i + I*r + I*R*c] * K_R(r,c)
//   A block takes 32 consecutive i (one per lane: coalesced column-major reads of T) of
//   one column c; its 8 warps take r = w, w + 8, ... (K_R(r,c) broadcast within a warp)
//   and their sums are added in warp order.
// Both orderings are deterministic.  Both are HBM-bound on T.  Both let the next kernel
// of the stream start early (its own griddepcontrol.wait still waits for them to finish).
#include "mtk_internal.cuh"

namespace mtk {
namespace {

__global__ void __launch_bounds__(256)
multi_ttv_right_kernel(const float* __restrict__ T, int64_t L, int64_t I,
                       const float* __restrict__ KL, int C, float* __restrict__ M) {
    allow_dependent_launch();
    const int lane = threadIdx.x & 31;
    const int64_t nw = I * C;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t w = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x / 32); w < nw;
         w += warps_total) {
        const int64_t i = w / C;
        const int c = (int)(w % C);
        const float* t = T + L * i + L * I * c;
        float s = 0.0f;
        for (int64_t l = lane; l < L; l += 32) s = fmaf(t[l], __ldg(KL + l * C + c), s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) M[i * C + c] = s;
    }
}

__global__ void __launch_bounds__(256)
multi_ttv_left_kernel(const float* __restrict__ T, int64_t I, int64_t R,
                      const float* __restrict__ KR, int C, float* __restrict__ M) {
    allow_dependent_launch();
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nib = (I + 31) / 32;
    for (int64_t b = blockIdx.x; b < nib * C; b += gridDim.x) {
        const int c = (int)(b / nib);
        const int64_t i = (b - (int64_t)c * nib) * 32 + lane;
        float s = 0.0f;
        if (i < I) {
            const float* t = T + i + I * R * c;
            for (int64_t r = w; r < R; r += 8) s = fmaf(t[I * r], __ldg(KR + r * C + c), s);
        }
        red[w][lane] = s;
        __syncthreads();
        if (w == 0 && i < I) {
            float a = red[0][lane];
#pragma unroll
            for (int k = 1; k < 8; ++k) a += red[k][lane];
            M[i * C + c] = a;
        }
        __syncthreads();
    }
}

// One mode of a C-batched tensor contracted with a factor (the dimension tree beyond
// N = 4: the modes >= 2 of the left partial): out(a, b, c) = sum_j T(a, j, b, c) K(j, c),
// T and out in natural order with c slowest; out_rowmajor: out as [a + A b][c] instead.
// One thread per output, consecutive a in consecutive threads (coalesced when A > 1); the
// sum over j runs in order.
__global__ void __launch_bounds__(256)
ttv_mode_kernel(const float* __restrict__ T, int64_t A, int64_t J, int64_t B,
                const float* __restrict__ K, int C, float* __restrict__ out, int out_rowmajor) {
    allow_dependent_launch();
    const int64_t n = A * B * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ab = e % (A * B);
        const int c = (int)(e / (A * B));
        const int64_t b = ab / A, a = ab - b * A;
        const float* t = T + a + A * J * (b + B * (int64_t)c);
        float s = 0.0f;
        for (int64_t j = 0; j < J; ++j) s = fmaf(t[A * j], __ldg(K + j * C + c), s);
        if (out_rowmajor) out[ab * C + c] = s;
        else out[e] = s;
    }
}

}  // namespace

cudaError_t launch_ttv_mode(const float* T, int64_t A, int64_t J, int64_t B, const float* K, int C, float* out,
                            int out_rowmajor, cudaStream_t s) {
    const int64_t n = A * B * C;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
    if (blocks < 1) blocks = 1;
    ttv_mode_kernel<<<(int)blocks, 256, 0, s>>>(T, A, J, B, K, C, out, out_rowmajor);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_multi_ttv(const float* T, int64_t L, int64_t I, int64_t R, const float* Ko,
                             int C, int right, float* M, cudaStream_t s) {
    if (right) {
        const int64_t nw = I * C;
        int64_t blocks = (nw + 7) / 8;
        int grid = (int)(blocks < num_sms() * 16 ? blocks : num_sms() * 16);
        multi_ttv_right_kernel<<<grid, 256, 0, s>>>(T, L, I, Ko, C, M);
        note_launches(1);
    } else {
        const int64_t blocks = (I + 31) / 32 * C;
        int grid = (int)(blocks < num_sms() * 8 ? blocks : num_sms() * 8);
        multi_ttv_left_kernel<<<grid, 256, 0, s>>>(T, I, R, Ko, C, M);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace mtk
