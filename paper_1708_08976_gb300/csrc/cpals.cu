// cpals.cu -- the non-MTTKRP parts of a CP-ALS factor update (Section 2.2):
//   G_k = U_k^T U_k (FP32 products, FP64 accumulation), H = Hadamard_{k != n} G_k,
//   U_n = M H^{-1} through an FP64 Cholesky factorisation (the reading of the
//   pseudoinverse for positive-definite H), ||X||^2 and the fit.
// All reductions use fixed trees and fixed chunk orders, so results do not
// depend on scheduling.
#include "mtk_internal.cuh"

namespace mtk {
namespace {

constexpr int kGramRows = 8;        // rows of U staged per step
constexpr int64_t kGramChunk = 8;     // rows per CTA, at least (many CTAs: the FP64 rate per
constexpr int64_t kGramMaxChunks = 256;  // SM is low), at most this many chunks

// partial Gram of rows [chunk*rpc, ...) for the pairs of block blockIdx.y
// (1024 pairs per block, 4 per thread); out = part + chunk*C*C (or G if one chunk)
__global__ void __launch_bounds__(256)
gram_partial_kernel(const float* __restrict__ U, int64_t I, int C, int64_t rpc, double* __restrict__ out) {
    extern __shared__ float us[];                 // kGramRows x C
    const int64_t r0 = (int64_t)blockIdx.x * rpc;
    const int64_t r1 = (r0 + rpc < I) ? r0 + rpc : I;
    const int npairs = C * C;
    const int pbase = blockIdx.y * 1024;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t rb = r0; rb < r1; rb += kGramRows) {
        const int nr = (int)((r1 - rb) < kGramRows ? (r1 - rb) : kGramRows);
        __syncthreads();
        for (int e = threadIdx.x; e < nr * C; e += blockDim.x) us[e] = U[rb * C + e];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = pbase + threadIdx.x + q * blockDim.x;
            if (e < npairs) {
                const int a = e / C, b = e % C;
                double s = acc[q];
                for (int r = 0; r < nr; ++r) s += (double)us[r * C + a] * (double)us[r * C + b];
                acc[q] = s;
            }
        }
    }
    for (int q = 0; q < 4; ++q) {
        const int e = pbase + threadIdx.x + q * blockDim.x;
        if (e < npairs) out[(int64_t)blockIdx.x * npairs + e] = acc[q];
    }
}

__global__ void gram_reduce_kernel(const double* __restrict__ part, int nchunks, int C,
                                   double* __restrict__ G) {
    const int npairs = C * C;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < npairs; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nchunks; ++k) s += part[(int64_t)k * npairs + e];
        G[e] = s;
    }
}

struct GramList {
    const double* G[MTK_MAXN];
};

// H = Hadamard_{k != n} G_k, its Cholesky factor H = L L^T and the inverse
// H^{-1} = L^{-T} L^{-1}, all FP64, one CTA.  Scratch layout (doubles): work[C*C]
// (used when the matrix does not fit in shared memory), diag[C], Hinv[C*C].
__global__ void __launch_bounds__(256)
chol_kernel(const __grid_constant__ GramList gl, int N, int C, int n, double* __restrict__ Hbuf,
            int* __restrict__ flag, uint32_t* status, int use_smem) {
    extern __shared__ double hs[];
    double* A = use_smem ? hs : Hbuf;
    double* diag = Hbuf + (size_t)C * C;
    double* Hinv = diag + C;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
        double h = 1.0;
        for (int k = 0; k < N; ++k)
            if (k != n) h *= gl.G[k][e];
        A[e] = h;
    }
    __syncthreads();
    // right-looking Cholesky, column j at a time (lower triangle)
    for (int j = 0; j < C; ++j) {
        if (threadIdx.x == 0) {
            const double d = A[j * C + j];
            if (!(d > 0.0)) bad = 1;
            A[j * C + j] = (d > 0.0) ? sqrt(d) : 1.0;
        }
        __syncthreads();
        if (bad) break;
        const double ljj = A[j * C + j];
        for (int i = j + 1 + threadIdx.x; i < C; i += blockDim.x) A[i * C + j] /= ljj;
        __syncthreads();
        // trailing update of the lower triangle: A(i,k) -= L(i,j) L(k,j), j < k <= i
        const int m = C - j - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = j + 1 + e / m, k = j + 1 + e % m;
            if (k <= i) A[i * C + k] -= A[i * C + j] * A[k * C + j];
        }
        __syncthreads();
    }
    if (!bad) {
        // W = L^{-1} by forward substitution, one thread per column j: W(i, j) for i > j is
        // kept at A[j*C + i] (the strict upper triangle is free), W(j, j) in diag[j]
        for (int j = threadIdx.x; j < C; j += blockDim.x) {
            const double wjj = 1.0 / A[j * C + j];
            for (int i = j + 1; i < C; ++i) {
                double sum = A[i * C + j] * wjj;
                for (int k = j + 1; k < i; ++k) sum += A[i * C + k] * A[j * C + k];
                A[j * C + i] = -sum / A[i * C + i];
            }
            diag[j] = wjj;
        }
        __syncthreads();
        // Hinv(a, b) = sum_{k >= max(a,b)} W(k, a) W(k, b)
        for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
            const int a = e / C, b = e % C;
            const int k0 = a > b ? a : b;
            double sum = 0.0;
            for (int k = k0; k < C; ++k) {
                const double wa = (k == a) ? diag[a] : A[a * C + k];
                const double wb = (k == b) ? diag[b] : A[b * C + k];
                sum += wa * wb;
            }
            Hinv[e] = sum;
        }
    }
    if (threadIdx.x == 0) {
        *flag = bad ? 0 : 1;
        if (bad) set_status(status, MTK_ENOTPD);
    }
}

// U_n(i, b) = sum_a M(i, a) Hinv(a, b), FP64 accumulation, one thread per output entry;
// nothing is written when H was not positive definite
__global__ void __launch_bounds__(256)
apply_inverse_kernel(const double* __restrict__ Hinv, const int* __restrict__ flag, const float* __restrict__ M,
                     int64_t In, int C, float* __restrict__ Un) {
    extern __shared__ double hsh[];
    const bool in_smem = C <= 64;
    if (in_smem)
        for (int e = threadIdx.x; e < C * C; e += blockDim.x) hsh[e] = Hinv[e];
    __syncthreads();
    if (*flag == 0) return;
    const double* H = in_smem ? hsh : Hinv;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < In * C;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / C;
        const int b = (int)(e % C);
        const float* m = M + i * C;
        double sum = 0.0;
        for (int a = 0; a < C; ++a) sum += (double)m[a] * H[a * C + b];
        Un[e] = (float)sum;
    }
}

// entries per CTA: a multiple of 1024 giving at most 1216 CTAs (8 per SM of this part) of at
// least 4096 entries; a function of I alone, so the fixed-order sum does not depend on the
// device.  (1 M entries per CTA left a 134 MB tensor to 32 CTAs and took 314 us.)
int64_t norm2_chunk(int64_t I) {
    int64_t nb = (I + 4095) / 4096;
    if (nb > 1216) nb = 1216;
    if (nb < 1) nb = 1;
    return ((I + nb - 1) / nb + 1023) / 1024 * 1024;
}

__global__ void __launch_bounds__(256)
norm2_partial_kernel(const float* __restrict__ X, int64_t I, int64_t chunk, double* __restrict__ part) {
    __shared__ double red[256];
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = (a + chunk < I) ? a + chunk : I;
    // exact squares, compensated FP32 sums of 64 entries, a double-FP32 total (SquareSum):
    // no FP64 arithmetic in the loop (this part's FP64 pipe is narrow)
    SquareSum sq;
    int cnt = 0;
    const bool vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    if (vec) {
        // a is a multiple of 4 (the chunk is), so X + a stays 16-byte aligned; four 16-byte
        // loads in flight per thread
        const int64_t nv = (b - a) / 4;
        const float4* xv = reinterpret_cast<const float4*>(X + a);
        for (int64_t v0 = threadIdx.x; v0 < nv; v0 += 4 * (int64_t)blockDim.x) {
            float4 q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t v = v0 + u * (int64_t)blockDim.x;
                q[u] = v < nv ? __ldcs(xv + v) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                sq.add(q[u].x);
                sq.add(q[u].y);
                sq.add(q[u].z);
                sq.add(q[u].w);
            }
            if (++cnt == 4) {
                sq.flush();
                cnt = 0;
            }
        }
        for (int64_t e = a + nv * 4 + threadIdx.x; e < b; e += blockDim.x) sq.add(X[e]);
    } else {
        for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
            sq.add(X[e]);
            if (++cnt == 64) {
                sq.flush();
                cnt = 0;
            }
        }
    }
    red[threadIdx.x] = sq.value();
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// one warp: lane l adds part[l], part[l + 32], ... in order, then a fixed shuffle tree
__global__ void sum_chunks_kernel(const double* __restrict__ part, int n, double* out) {
    const int l = threadIdx.x;
    double s = 0.0;
    for (int k = l; k < n; k += 32) s += part[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (l == 0 && blockIdx.x == 0) *out = s;
}

// r2 = ||X||^2 - 2 <M, U> + sum_{a,b} prod_k G_k(a,b)  (= ||X - [[U]]||^2 when M is the
// MTTKRP of the mode U belongs to), fit = 1 - sqrt(max(0, r2)) / ||X||, and the loss
// 0.5 r2 rounded to FP32
__global__ void __launch_bounds__(256)
residual_kernel(const double* __restrict__ normX2, const float* __restrict__ M,
                const float* __restrict__ U, int64_t I, const __grid_constant__ GramList gl, int N,
                int C, double* r2_out, double* fit, float* loss) {
    __shared__ double red[256];
    double inner = 0.0;
    for (int64_t e = threadIdx.x; e < I * C; e += blockDim.x) inner += (double)M[e] * (double)U[e];
    double y2 = 0.0;
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
        double h = 1.0;
        for (int k = 0; k < N; ++k) h *= gl.G[k][e];
        y2 += h;
    }
    red[threadIdx.x] = y2 - 2.0 * inner;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nx2 = *normX2;
        const double r2 = nx2 + red[0];
        if (r2_out) *r2_out = r2;
        if (fit) *fit = 1.0 - sqrt(r2 > 0.0 ? r2 : 0.0) / sqrt(nx2);
        if (loss) *loss = (float)(0.5 * r2);
    }
}

// grad(i, b) = scale * (sum_a U(i,a) H(a,b) - M(i,b)),  H = Hadamard_{k != n} G_k
__global__ void __launch_bounds__(256)
gradient_kernel(const float* __restrict__ U, const float* __restrict__ M,
                const __grid_constant__ GramList gl, int N, int C, int n, int64_t In,
                const float* __restrict__ scale, float* __restrict__ grad) {
    extern __shared__ double Hs[];
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
        double h = 1.0;
        for (int k = 0; k < N; ++k)
            if (k != n) h *= gl.G[k][e];
        Hs[e] = h;
    }
    __syncthreads();
    const double sc = scale ? (double)*scale : 1.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < In * C;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / C;
        const int b = (int)(e % C);
        double s = 0.0;
        for (int a = 0; a < C; ++a) s += (double)U[i * C + a] * Hs[a * C + b];
        grad[e] = (float)(sc * (s - (double)M[e]));
    }
}

}  // namespace

int gram_chunks(int64_t I) {
    const int64_t n = (I + kGramChunk - 1) / kGramChunk;
    return (int)(n < kGramMaxChunks ? n : kGramMaxChunks);
}

cudaError_t launch_gram(const float* U, int64_t I, int C, double* G, double* part, int nchunks,
                        cudaStream_t s) {
    const size_t smem = (size_t)kGramRows * C * sizeof(float);
    const unsigned pblocks = (unsigned)((C * C + 1023) / 1024);
    const int64_t rpc = (I + nchunks - 1) / (nchunks > 0 ? nchunks : 1);
    if (nchunks <= 1) {
        gram_partial_kernel<<<dim3(1, pblocks), 256, smem, s>>>(U, I, C, I, G);
        note_launches(1);
    } else {
        gram_partial_kernel<<<dim3(nchunks, pblocks), 256, smem, s>>>(U, I, C, rpc, part);
        note_launches(1);
        gram_reduce_kernel<<<(C * C + 255) / 256, 256, 0, s>>>(part, nchunks, C, G);
        note_launches(1);
    }
    return cudaGetLastError();
}

size_t solve_scratch_doubles(int C) { return 2 * (size_t)C * C + C; }

cudaError_t launch_chol_solve(const double* const* G, int N, int C, int n, const float* M,
                              int64_t In, float* Un, double* Hbuf, int* flag, uint32_t* status,
                              cudaStream_t s) {
    GramList gl;
    for (int k = 0; k < MTK_MAXN; ++k) gl.G[k] = (k < N) ? G[k] : nullptr;
    const size_t hbytes = (size_t)C * C * sizeof(double);
    // C <= 64 takes the one-launch update of als_update.cu; this path serves larger ranks
    const int chol_smem = hbytes <= 200 * 1024;
    if (chol_smem) {
        cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hbytes);
    }
    chol_kernel<<<1, 256, chol_smem ? hbytes : 0, s>>>(gl, N, C, n, Hbuf, flag, status, chol_smem);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double* Hinv = Hbuf + (size_t)C * C + C;
    const size_t smem = C <= 64 ? hbytes : 0;
    int64_t blocks = (In * C + 255) / 256;
    int grid = (int)(blocks < num_sms() * 4 ? blocks : num_sms() * 4);
    apply_inverse_kernel<<<grid, 256, smem, s>>>(Hinv, flag, M, In, C, Un);
    note_launches(1);
    return cudaGetLastError();
}

int norm2_chunks(int64_t I) {
    const int64_t c = norm2_chunk(I);
    return (int)((I + c - 1) / c);
}

cudaError_t launch_norm2(const float* X, int64_t I, double* part, int nchunks, double* out,
                         cudaStream_t s) {
    norm2_partial_kernel<<<nchunks, 256, 0, s>>>(X, I, norm2_chunk(I), part);
    note_launches(1);
    sum_chunks_kernel<<<1, 32, 0, s>>>(part, nchunks, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_residual(const double* normX2, const float* M, const float* U, int64_t I,
                            const double* const* G, int N, int C, double* r2, double* fit,
                            cudaStream_t s, float* loss) {
    GramList gl;
    for (int k = 0; k < MTK_MAXN; ++k) gl.G[k] = (k < N) ? G[k] : nullptr;
    residual_kernel<<<1, 256, 0, s>>>(normX2, M, U, I, gl, N, C, r2, fit, loss);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gradient(const float* U, const float* M, const double* const* G, int N, int C,
                            int n, int64_t In, const float* scale, float* grad, cudaStream_t s) {
    GramList gl;
    for (int k = 0; k < MTK_MAXN; ++k) gl.G[k] = (k < N) ? G[k] : nullptr;
    const size_t smem = (size_t)C * C * sizeof(double);
    cudaFuncSetAttribute(gradient_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int64_t blocks = (In * C + 255) / 256;
    int grid = (int)(blocks < num_sms() * 4 ? blocks : num_sms() * 4);
    gradient_kernel<<<grid, 256, smem, s>>>(U, M, gl, N, C, n, In, scale, grad);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace mtk
