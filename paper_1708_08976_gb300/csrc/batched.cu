// batched.cu -- many independent MTTKRPs (Section 2.2) in one persistent launch.
//
// Each problem p is one mode-n MTTKRP of its own N-way tensor (N <= 4), with its own
// dims and rank C_p <= 32.  On the 3-way view of the mode (Fig. 2) the problem is
//     M(i, c) = sum_k X3(k, i) W(k, c),   X3(k, i) = X[l + L i + L I r],  k = l + L r,
// W(k, c) = prod_z F_z(digit_z(k), c) over the mode's factor list (first factor fastest,
// Section 2.1 row rule).  The work is cut into units (problem, tile of rows, chunk of k);
// a persistent grid walks the unit list (two CTAs per SM, static round robin), each unit
// accumulates its partial M in registers with FP32 FMAs on the CUDA cores and writes it
// to a slab; one reduce launch then adds the slabs of every problem in slab order
// (deterministic).  The whole batch is two launches, which the caller can capture in a
// CUDA graph.  Uneven, unaligned dims are the norm here (no 16-byte row strides), so the
// tensor is read with plain coalesced loads.
//
// Register blocking: 256 threads, each a 4 x 4 block of (rows, columns); a tile is
// BI = 4096 / CB rows x CB columns with CB = C rounded up to 8, 16 or 32, and 16 k-values
// deep.  Per k, a thread reads 4 tensor values and 4 KRP values from shared memory for 16
// FMAs; the next tile is loaded into registers while the current one is multiplied.
#include <string.h>

#include "mtk_internal.cuh"

namespace mtk {
namespace {

constexpr int BT_KQ = 64;                 // k-chunks of units are multiples of this
constexpr int BT_THREADS = 256;

struct BItem {
    const float* X;
    const float* f[3];       // factor list of the mode, first = fastest digit of k
    float* part;             // slabs [nchunks][I][C] (or the output when nchunks == 1)
    float* out;              // M, I x C row-major
    int rad[3];
    int nf;
    int L, I, R;             // 3-way view
    int C, CB;
    int ntiles, nchunks;
    int kchunk;              // k per unit (multiple of BT_KQ)
    int unit0;               // first unit of this problem
};

__device__ __forceinline__ int find_item(const BItem* it, int P, int u) {
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (it[mid].unit0 <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int CB>
__device__ void run_unit(const BItem& bi, int tile, int chunk, float* xs, float* ws) {
    constexpr int BT_KT = 16;                // k per staged tile
    constexpr int BI = 4096 / CB;
    constexpr int TR = BI / 4;               // threads along rows
    constexpr int XPT = BT_KT * BI / BT_THREADS;    // tensor values staged per thread per tile
    constexpr int WPT = (BT_KT * CB + BT_THREADS - 1) / BT_THREADS;
    // the problem's fields in registers (the descriptor lives in the parameter space)
    const float* __restrict__ X = bi.X;
    const int L = bi.L, I = bi.I, C = bi.C, nf = bi.nf;
    const float* f0 = bi.f[0];
    const float* f1 = bi.f[1];
    const float* f2 = bi.f[2];
    const uint32_t r0 = (uint32_t)bi.rad[0], r1 = (uint32_t)bi.rad[1];
    const int nchunks = bi.nchunks;
    float* part = bi.part;
    float* outp = bi.out;
    const int t = threadIdx.x;
    const int tr = t % TR, tc = t / TR;      // 4 rows at 4*tr, 4 columns at 4*tc
    const int i0 = tile * BI;
    const int64_t k0 = (int64_t)chunk * bi.kchunk;
    int64_t k1 = k0 + bi.kchunk;
    const int64_t K = (int64_t)L * bi.R;
    if (k1 > K) k1 = K;
    const int64_t LI = (int64_t)L * I;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] = 0.0f;

    // staged values of the next tile (loaded while the current one is multiplied)
    float xr[XPT], wr[WPT];
    auto load = [&](int64_t kb) {
        if (L == 1) {
#pragma unroll
            for (int j = 0; j < XPT; ++j) {
                const int e = t + BT_THREADS * j;
                const int i = e % BI, kk = e / BI;
                const int64_t k = kb + kk;
                xr[j] = (k < k1 && i0 + i < I) ? __ldg(X + (i0 + i) + (int64_t)I * k) : 0.0f;
            }
        } else {
            // this thread's k in the tile is fixed (e % BT_KT == t % BT_KT): split it once
            const int kk = t % BT_KT;
            const uint32_t k = (uint32_t)(kb + kk);
            const uint32_t r = k / (uint32_t)L, l = k - r * (uint32_t)L;
            const float* xk = X + l + LI * r;
            const bool kin = (int64_t)(kb + kk) < k1;
#pragma unroll
            for (int j = 0; j < XPT; ++j) {
                const int i = t / BT_KT + (BT_THREADS / BT_KT) * j;
                xr[j] = (kin && i0 + i < I) ? __ldg(xk + (int64_t)L * (i0 + i)) : 0.0f;
            }
        }
#pragma unroll
        for (int j = 0; j < WPT; ++j) {
            const int e = t + BT_THREADS * j;
            const int c = e % CB, kk = e / CB;
            const int64_t k = kb + kk;
            float w = 0.0f;
            if (e < BT_KT * CB && k < k1 && c < C) {
                const uint32_t u = (uint32_t)k;
                const uint32_t q0 = u / r0;
                w = __ldg(f0 + (int64_t)(u - q0 * r0) * C + c);
                if (nf > 1) {
                    const uint32_t q1 = q0 / r1;
                    w *= __ldg(f1 + (int64_t)(q0 - q1 * r1) * C + c);
                    if (nf > 2) w *= __ldg(f2 + (int64_t)q1 * C + c);
                }
            }
            wr[j] = w;
        }
    };
    auto store = [&]() {
        if (L == 1) {
#pragma unroll
            for (int j = 0; j < XPT; ++j) {
                const int e = t + BT_THREADS * j;
                xs[(e / BI) * (BI + 4) + (e % BI)] = xr[j];
            }
        } else {
            const int kk = t % BT_KT;
#pragma unroll
            for (int j = 0; j < XPT; ++j) xs[kk * (BI + 4) + t / BT_KT + (BT_THREADS / BT_KT) * j] = xr[j];
        }
#pragma unroll
        for (int j = 0; j < WPT; ++j) {
            const int e = t + BT_THREADS * j;
            if (e < BT_KT * CB) ws[e] = wr[j];
        }
    };

    if (k0 < k1) load(k0);
    for (int64_t kb = k0; kb < k1; kb += BT_KT) {
        __syncthreads();
        store();
        __syncthreads();
        if (kb + BT_KT < k1) load(kb + BT_KT);
#pragma unroll
        for (int kk = 0; kk < BT_KT; ++kk) {
            const float4 xv = *reinterpret_cast<const float4*>(xs + kk * (BI + 4) + 4 * tr);
            const float4 wv = *reinterpret_cast<const float4*>(ws + kk * CB + 4 * tc);
            const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
            const float wa[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[a][q] = fmaf(xa[a], wa[q], acc[a][q]);
        }
    }
    // write the partial (or the result when the problem has one chunk)
    float* dst = nchunks == 1 ? outp : part + (int64_t)chunk * I * C;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + 4 * tr + a;
        if (i >= I) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = 4 * tc + q;
            if (c < C) dst[(int64_t)i * C + c] = acc[a][q];
        }
    }
}

template <int MAXP>
struct BatchParams {
    int P, nunits;
    BItem it[MAXP];
};

template <int MAXP>
__global__ void __launch_bounds__(BT_THREADS, 2) mttkrp_batched_kernel(const __grid_constant__ BatchParams<MAXP> a) {
    // xs: 16 x (BI + 4) floats (BI <= 512); ws: 16 x CB floats
    __shared__ __align__(16) float xs[16 * (512 + 4)];
    __shared__ __align__(16) float ws[16 * 32];
    for (int u = blockIdx.x; u < a.nunits; u += gridDim.x) {
        const int p = find_item(a.it, a.P, u);
        const BItem& b = a.it[p];
        const int local = u - b.unit0;
        const int tile = local % b.ntiles, chunk = local / b.ntiles;
        if (b.CB == 8) run_unit<8>(b, tile, chunk, xs, ws);
        else if (b.CB == 16) run_unit<16>(b, tile, chunk, xs, ws);
        else run_unit<32>(b, tile, chunk, xs, ws);
    }
}

// M of every problem = sum of its slabs in slab order
template <int MAXP>
__global__ void __launch_bounds__(256) batched_reduce_kernel(const __grid_constant__ BatchParams<MAXP> a) {
    const int p = blockIdx.y;
    if (p >= a.P) return;
    const BItem& b = a.it[p];
    if (b.nchunks <= 1) return;
    const int64_t n = (int64_t)b.I * b.C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.0f;
        for (int s = 0; s < b.nchunks; ++s) v += b.part[(int64_t)s * n + e];
        b.out[e] = v;
    }
}

constexpr int kMaxP = 192;                 // problems per launch (kernel parameter space)

int64_t round_up64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

int batched_max_problems() { return kMaxP; }

// Plan of one problem: view, tiles, chunks.  kchunk_target: k per unit (0 = automatic).
// Taken: N <= 4, C <= 32, contraction length I^L I^R < 2^31.
bool batched_plan_item(const int64_t* dims, int N, int n, int C, int64_t kchunk_target, int ctas,
                       int* ntiles, int* nchunks, int* kchunk, int* CB) {
    if (N < 2 || N > 4 || n < 0 || n >= N || C < 1 || C > 32) return false;
    int64_t L = 1, R = 1;
    for (int k = 0; k < n; ++k) L *= dims[k];
    for (int k = n + 1; k < N; ++k) R *= dims[k];
    const int64_t I = dims[n];
    const int64_t lim = ((int64_t)1 << 31) - 1;
    if (L > lim || R > lim || I > lim || L * R > lim) return false;
    *CB = C <= 8 ? 8 : (C <= 16 ? 16 : 32);
    const int BI = 4096 / *CB;
    *ntiles = (int)((I + BI - 1) / BI);
    const int64_t K = L * R;
    int64_t kc = kchunk_target;
    if (kc <= 0) {
        // about 2 units per CTA over this problem alone, at least 4 k-tiles per unit
        int64_t units = 2 * (int64_t)ctas / *ntiles;
        if (units < 1) units = 1;
        kc = (K + units - 1) / units;
    }
    kc = round_up64(kc < BT_KQ ? BT_KQ : kc, BT_KQ);
    if (kc > K) kc = round_up64(K, BT_KQ);
    if (kc > lim) kc = lim / BT_KQ * BT_KQ;
    *kchunk = (int)kc;
    *nchunks = (int)((K + kc - 1) / kc);
    return true;
}

// automatic k per unit for a whole batch: about 4 units per CTA over all problems
static int64_t batch_kchunk(const BatchedProblem* probs, int P, int64_t kchunk_target, int ctas) {
    if (kchunk_target > 0) return kchunk_target;
    int64_t work = 0;
    for (int p = 0; p < P; ++p) {
        const BatchedProblem& q = probs[p];
        if (q.N < 2 || q.N > 4 || q.n < 0 || q.n >= q.N || q.C < 1 || q.C > 32) continue;
        int64_t K = 1;
        for (int k = 0; k < q.N; ++k)
            if (k != q.n) K *= q.dims[k];
        const int CB = q.C <= 8 ? 8 : (q.C <= 16 ? 16 : 32);
        work += K * ((q.dims[q.n] + 4096 / CB - 1) / (4096 / CB));
    }
    int64_t kc = work / (4 * (int64_t)(ctas > 0 ? ctas : 1));
    return kc < BT_KQ ? BT_KQ : kc;
}

cudaError_t launch_batched(const BatchedProblem* probs, int P, int64_t kchunk_target, int ctas, float* scratch,
                           cudaStream_t s) {
    if (P > kMaxP) return cudaErrorInvalidValue;
    kchunk_target = batch_kchunk(probs, P, kchunk_target, ctas);
    BatchParams<kMaxP>* a = new BatchParams<kMaxP>;
    memset(a, 0, sizeof(*a));
    a->P = P;
    int units = 0;
    int64_t off = 0;
    int maxchunks = 1, maxrows = 0;
    for (int p = 0; p < P; ++p) {
        const BatchedProblem& q = probs[p];
        BItem& b = a->it[p];
        int ntiles, nchunks, kchunk, CB;
        if (!batched_plan_item(q.dims, q.N, q.n, q.C, kchunk_target, ctas, &ntiles, &nchunks, &kchunk, &CB)) {
            delete a;
            return cudaErrorInvalidValue;
        }
        int64_t L = 1, R = 1;
        for (int k = 0; k < q.n; ++k) L *= q.dims[k];
        for (int k = q.n + 1; k < q.N; ++k) R *= q.dims[k];
        b.X = q.X;
        b.nf = 0;
        for (int k = 0; k < q.N; ++k) {
            if (k == q.n) continue;
            b.f[b.nf] = q.U[k];
            b.rad[b.nf] = (int)q.dims[k];
            ++b.nf;
        }
        b.out = q.M;
        b.L = (int)L;
        b.I = (int)q.dims[q.n];
        b.R = (int)R;
        b.C = q.C;
        b.CB = CB;
        b.ntiles = ntiles;
        b.nchunks = nchunks;
        b.kchunk = kchunk;
        b.unit0 = units;
        units += ntiles * nchunks;
        if (nchunks > 1) {
            b.part = scratch + off;
            off += round_up64((int64_t)nchunks * b.I * b.C, 64);
        }
        if (nchunks > maxchunks) maxchunks = nchunks;
        if (b.I * b.C > maxrows) maxrows = b.I * b.C;
    }
    a->nunits = units;
    int grid = units < ctas ? units : ctas;
    if (grid < 1) grid = 1;
    mttkrp_batched_kernel<kMaxP><<<grid, BT_THREADS, 0, s>>>(*a);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && maxchunks > 1) {
        int bx = (maxrows + 255) / 256;
        if (bx > 16) bx = 16;
        batched_reduce_kernel<kMaxP><<<dim3(bx, P), 256, 0, s>>>(*a);
        note_launches(1);
        e = cudaGetLastError();
    }
    delete a;
    return e;
}

size_t batched_scratch_floats(const BatchedProblem* probs, int P, int64_t kchunk_target, int ctas) {
    kchunk_target = batch_kchunk(probs, P, kchunk_target, ctas);
    int64_t off = 0;
    for (int p = 0; p < P; ++p) {
        const BatchedProblem& q = probs[p];
        int ntiles, nchunks, kchunk, CB;
        if (!batched_plan_item(q.dims, q.N, q.n, q.C, kchunk_target, ctas, &ntiles, &nchunks, &kchunk, &CB))
            return (size_t)-1;
        if (nchunks > 1) off += round_up64((int64_t)nchunks * q.dims[q.n] * q.C, 64);
    }
    return (size_t)off;
}

}  // namespace mtk
