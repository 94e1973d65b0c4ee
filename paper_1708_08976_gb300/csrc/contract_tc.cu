// contract_tc.cu -- tensor-core (tcgen05 / TMEM) form of the MTTKRP contraction
//     D(i, c) = sum_k X3(k, i) W(k, c)
// on the 3-way view of the tensor (Fig. 2: the mode-n matricization is R row-major
// I x L blocks, consumed in place; the tensor is never reordered).
//
// Block structure (Algorithm 3).  The parallel 1-step algorithm forms, for each
// block j, K_R(j,:) kr K_L and multiplies it with the block of X_(n); equivalently
// it multiplies the block by the fixed K_L and scales column c by K_R(j, c).  Here
// the factor list of the mode (first factor = fastest digit of k) is split into a
// head (the first few factors, whose KRP has rad0 rows) and a tail.  Every run of
// rad0 consecutive k shares one tail row q, so
//     D(i, c) = sum_q Q(q, c) * sum_{d0} X3(q*rad0 + d0, i) * H(d0, c)
// with H the head KRP and Q(q, c) = prod_t tail_t(digit_t(q), c).  The inner sums
// run on the tensor cores against H, which is the same for every run: a prep
// kernel writes H once per call, split into BF16 pieces, as an image of the
// swizzled shared-memory B operand (one slice per 64-k stage, runs padded to a
// multiple of 64), and each stage fetches its slice with one cp.async.bulk copy
// (the image is L2-resident).  The scale Q is applied when the accumulator is
// drained from TMEM, which happens at least every two stages.
//
// Precision (split products).  Each FP32 tensor entry x is split into BF16 pieces
// x = x_1 + x_2 (+ x_3) by round-to-nearest on the successive remainders, each head
// entry into three (the bf16x3 / bf16x6 schemes of Henry, Tang and Heinecke, ARITH
// 2019).  One MMA per tensor piece multiplies it with all three H pieces, stacked
// along N, so every cross product is formed.  Tensor-core FP32 accumulation does
// not round to nearest, and its error grows with the number of accumulation
// steps; draining TMEM into FP32 registers (round-to-nearest adds) every <= 2
// stages keeps each accumulation chain at <= 8 (2 pieces) or 12 (3 pieces) MMA
// steps per k-quarter-stage group.
//
// Tile: MMA M = 128 rows of i (the CTA owns BI <= 128 of them), N = 3 * CP (CP = C
// rounded up to 16), K = 64 per stage (one 128-byte swizzle row of BF16).  The
// tensor operand A is K-major when k runs along the contiguous mode (I^L > 1) and
// MN-major when i is the contiguous index (mode 0, I^L = 1); B is K-major.
//
// Warp roles: CONV_WARPS converter warps copy the tensor with 16-byte cp.async into
// a thread-private staging ring in shared memory (several stages in flight without
// holding registers), split it, store the pieces, and drain the accumulator; one
// thread of the last warp issues tcgen05.mma.
//
// Every mbarrier wait is bounded (1 s of %globaltimer by default, or the caller's limit);
// on expiry the kernel sets MTK_ETIMEOUT in the status word and every role stops.  Before
// the CTA frees its TMEM and leaves, each role waits (with a 1 s limit that an abort does
// not shorten) for the asynchronous work it started: the TMA producer for its last tile
// loads, the converter warp that issues the B-image copies for those copies, and the MMA
// issuer for its MMAs (one final commit).  Nothing then lands in shared memory or TMEM
// after the CTA has exited.
#include "contract_tc_kernel.cuh"

namespace mtk {

// every variant is instantiated in the translation unit of its (PX, MN) pair
extern template cudaError_t tc_launch<2, true, true>(const tcd::TcParams&, const CUtensorMap&, dim3,
                                                      size_t, cudaStream_t);
extern template cudaError_t tc_launch<2, true, false>(const tcd::TcParams&, const CUtensorMap&, dim3,
                                                      size_t, cudaStream_t);
extern template cudaError_t tc_launch<2, false, true>(const tcd::TcParams&, const CUtensorMap&, dim3,
                                                      size_t, cudaStream_t);
extern template cudaError_t tc_launch<2, false, false>(const tcd::TcParams&, const CUtensorMap&, dim3,
                                                      size_t, cudaStream_t);
extern template cudaError_t tc_launch<3, true, true>(const tcd::TcParams&, const CUtensorMap&, dim3,
                                                      size_t, cudaStream_t);
extern template cudaError_t tc_launch<3, true, false>(const tcd::TcParams&, const CUtensorMap&, dim3,
                                                      size_t, cudaStream_t);
extern template cudaError_t tc_launch<3, false, true>(const tcd::TcParams&, const CUtensorMap&, dim3,
                                                      size_t, cudaStream_t);
extern template cudaError_t tc_launch<3, false, false>(const tcd::TcParams&, const CUtensorMap&, dim3,
                                                      size_t, cudaStream_t);

using namespace tcd;

namespace {

using namespace tc;

// ---- B image: the head KRP split into three BF16 pieces, in stage slices --------
struct ImgArgs {
    int head, C, CP, N;
    const float* fac[MTK_MAXN];
    int64_t frad[MTK_MAXN];
    int64_t rad0, rad0p;
    uint8_t* img;
};

__global__ void __launch_bounds__(256) tc_image_kernel(const __grid_constant__ ImgArgs a) {
    const int64_t items = (a.rad0p / 8) * a.CP;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(it % a.CP);
        const int64_t k0 = (it / a.CP) * 8;           // first padded k of the octet
        int64_t dig[MTK_MAXN];
        int64_t rem = k0;
        for (int z = 0; z < a.head; ++z) { dig[z] = rem % a.frad[z]; rem /= a.frad[z]; }
        float w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float v = 0.0f;
            if (k0 + j < a.rad0 && c < a.C) {
                v = 1.0f;
                for (int z = 0; z < a.head; ++z) v *= __ldg(a.fac[z] + dig[z] * a.C + c);
            }
            w[j] = v;
            for (int z = 0; z < a.head; ++z) {        // increment the mixed-radix digits
                if (++dig[z] < a.frad[z]) break;
                dig[z] = 0;
            }
        }
        uint2 lo4[3], hi4[3];
        split4<3>(make_float4(w[0], w[1], w[2], w[3]), lo4);
        split4<3>(make_float4(w[4], w[5], w[6], w[7]), hi4);
        const int64_t stage = k0 / TC_BK;
        const int oct = (int)((k0 % TC_BK) / 8);
        uint8_t* base = a.img + stage * (int64_t)(a.N * 128);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int n = q * a.CP + c;
            const uint32_t off = (uint32_t)((n >> 3) * 1024 + (n & 7) * 128 + (((oct ^ (n & 7)) & 7) << 4));
            *reinterpret_cast<uint4*>(base + off) = make_uint4(lo4[q].x, lo4[q].y, hi4[q].x, hi4[q].y);
        }
    }
}

int tile_rows(int64_t I) {
    const int64_t tiles = (I + TC_M - 1) / TC_M;
    int64_t bi = (I + tiles - 1) / tiles;
    bi = (bi + 7) & ~7LL;
    return (int)(bi > TC_M ? TC_M : bi);
}

// TMA staging applies when the boxes below are legal and never straddle a run of l:
// K-major: 8-float boxes at l multiples of 8 (I^L and the head rows divisible by 8);
// MN-major: (BI x 64) boxes along (i, r).  Coordinates must fit in 32 bits.
bool tma_eligible(const ContractParams& p, const TcPlan& pl) {
#ifdef MTK_TC_CPASYNC_ONLY
    return false;
#endif
    if (CONV_WARPS != 8) return false;
    const int64_t lim = ((int64_t)1 << 31) - TC_BK;
    if (p.L == 1) return p.I % 4 == 0 && pl.BI <= 256 && p.I < lim && p.R < lim;
    return p.L % 8 == 0 && pl.rad0 % 8 == 0 && pl.BI % 4 == 0 && pl.BI <= 256 && p.L < lim && p.I < lim &&
           p.R < lim;
}

bool encode_xmap(const ContractParams& p, const TcPlan& pl, CUtensorMap* map) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    CUresult r;
    if (p.L == 1) {
        const cuuint64_t dims[2] = {(cuuint64_t)p.I, (cuuint64_t)p.R};
        const cuuint64_t strides[1] = {(cuuint64_t)p.I * 4};
        const cuuint32_t box[2] = {(cuuint32_t)pl.BI, (cuuint32_t)TC_BK};
        const cuuint32_t es[2] = {1, 1};
        r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p.X), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[3] = {(cuuint64_t)p.L, (cuuint64_t)p.I, (cuuint64_t)p.R};
        const cuuint64_t strides[2] = {(cuuint64_t)p.L * 4, (cuuint64_t)p.L * p.I * 4};
        const cuuint32_t box[3] = {pl.linear ? (cuuint32_t)TC_BK : 8u, (cuuint32_t)pl.BI, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(p.X), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS;
}

}  // namespace

// declared in tc_ptx.cuh
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }();
    return fn;
}

bool contract_tc_shape_ok(int64_t L, int64_t I, int C, int precision) {
    if (precision != MTK_PREC_BF16X2 && precision != MTK_PREC_BF16X3) return false;
    if (C < 1 || C > MAX_CB) return false;
    if (L == 1) return I % 4 == 0 && I < (int64_t(1) << 24);   // 16-byte loads along i
    return L % 4 == 0;                                          // 16-byte loads along k
}

TcPlan contract_tc_plan(const int64_t* frad, int nfac, int64_t L, int64_t I, int C) {
    TcPlan pl;
    memset(&pl, 0, sizeof(pl));
    // head: fewest leading factors with >= 64 rows, <= 1/32 padding and a row count
    // divisible by 4 (keeps the 16-byte tensor loads aligned); else all factors
    int64_t prod = 1;
    int m = 0;
    while (m < nfac) {
        prod *= frad[m];
        ++m;
        const int64_t padded = (prod + TC_BK - 1) / TC_BK * TC_BK;
        if (prod >= TC_BK && (padded - prod) * 32 <= prod && prod % 4 == 0) break;
    }
    if (nfac == 0) { prod = 1; m = 0; }
    int64_t K = 1;
    for (int z = 0; z < nfac; ++z) K *= frad[z];
    pl.head = m;
    pl.rad0 = prod;
    pl.rad0p = (prod + TC_BK - 1) / TC_BK * TC_BK;
    pl.nruns = K / prod;
    // runs are contiguous in memory when i is the contiguous index or the head lies
    // inside the modes left of n (rad0 divides I^L)
    pl.linear = (L == 1 || L % prod == 0) ? 1 : 0;
    // small I: pack U runs into the 128 MMA rows (needs contiguous runs)
    pl.U = 1;
    if (pl.linear && I <= TC_M / 2 && pl.nruns > 1 && (L > 1 || I % 8 == 0)) {
        int64_t u = TC_M / I;
        if (u > pl.nruns) u = pl.nruns;
        pl.U = (int)u;
    }
    pl.BI = pl.U > 1 ? (int)I : tile_rows(I);
    pl.Kp = ((pl.nruns + pl.U - 1) / pl.U) * pl.rad0p;
    pl.CP = (C + 15) & ~15;
    pl.N = 3 * pl.CP;
    pl.image_bytes = (size_t)(pl.rad0p / TC_BK) * pl.N * 128;
    return pl;
}

bool contract_tc_supported(const ContractParams& p, int precision) {
    if (!contract_tc_shape_ok(p.L, p.I, p.C, precision)) return false;
    if ((reinterpret_cast<uintptr_t>(p.X) & 15) != 0) return false;
    if (p.kchunk <= 0 || p.kchunk % TC_BK != 0) return false;
    if (p.nfac < 1) return false;
    return true;
}

cudaError_t launch_contract_tc(const ContractParams& p, int precision, void* image, cudaStream_t s) {
    const TcPlan pl = contract_tc_plan(p.frad, p.nfac, p.L, p.I, p.C);
    TcParams tp;
    memset(&tp, 0, sizeof(tp));
    tp.p = p;
    tp.wait_ns = p.wait_ns ? p.wait_ns : kWaitNs;
    tp.stall = p.stall;
    tp.bimg = static_cast<const uint8_t*>(image);
    tp.ntail = p.nfac - pl.head;
    for (int z = pl.head; z < p.nfac; ++z) {
        tp.tail[z - pl.head] = p.fac[z];
        tp.tail_rad[z - pl.head] = p.frad[z];
    }
    tp.rad0 = pl.rad0;
    tp.rad0p = pl.rad0p;
    tp.Kp = pl.Kp;
    tp.nruns = pl.nruns;
    tp.BI = pl.BI;
    tp.U = pl.U;
    tp.CP = pl.CP;
    tp.N = pl.N;
    tp.linear = pl.linear;
    tp.nslabs = p.S * pl.U;
    tp.mn_major = p.L == 1 ? 1 : 0;
    const int px = precision == MTK_PREC_BF16X3 ? 3 : 2;
    tp.b_off = px * PIECE_BYTES;
    tp.b_bytes = pl.N * 128;
    tp.stage_bytes = tp.b_off + ((tp.b_bytes + 1023) & ~1023);
    tp.stages = MTK_TC_AB_STAGES;
    const int stg_stage = 2 * RPT * CONV_THREADS * 16;           // 32 KB of staging per stage
    const int budget = 222 * 1024;
    while (tp.stages > 2 && budget - tp.stages * tp.stage_bytes < 2 * stg_stage) --tp.stages;
    int P = (budget - tp.stages * tp.stage_bytes) / stg_stage;
    if (P > MAX_STAGING) P = MAX_STAGING;
    if (P < 2) P = 2;
    tp.P = P;
    tp.stg_off = tp.stages * tp.stage_bytes;
    int cols = 32;
    while (cols < 2 * pl.N) cols <<= 1;
    tp.tmem_cols = cols;
    // kind::f16 instruction descriptor: D = F32 (bits 4-5), A = B = BF16 (bits 7-9,
    // 10-12), A major (bit 15), B K-major, N >> 3 (bits 17-22), M >> 4 (bits 24-28)
    tp.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)tp.mn_major << 15) |
               ((uint32_t)(pl.N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

    // 1) the B image of the head
    ImgArgs ia;
    memset(&ia, 0, sizeof(ia));
    ia.head = pl.head;
    ia.C = p.C;
    ia.CP = pl.CP;
    ia.N = pl.N;
    for (int z = 0; z < pl.head; ++z) { ia.fac[z] = p.fac[z]; ia.frad[z] = p.frad[z]; }
    ia.rad0 = pl.rad0;
    ia.rad0p = pl.rad0p;
    ia.img = static_cast<uint8_t*>(image);
    const int64_t items = (pl.rad0p / 8) * pl.CP;
    int64_t blocks = (items + 255) / 256;
    int grid_img = (int)(blocks < num_sms() * 8 ? blocks : num_sms() * 8);
    tc_image_kernel<<<grid_img, 256, 0, s>>>(ia);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    // 2) the contraction
    const size_t smem = (size_t)tp.stg_off + (size_t)tp.P * stg_stage + 1024;
    const int64_t tiles = (p.I + tp.BI - 1) / tp.BI;
    const dim3 grid((unsigned)tiles, (unsigned)p.S);
    const bool mn = tp.mn_major != 0;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    const bool tma = tma_eligible(p, pl) && encode_xmap(p, pl, &map);
    tp.kwide = (tma && !mn && pl.linear) ? 1 : 0;
    if (tma) {
        if (px == 3) return mn ? tc_launch<3, true, true>(tp, map, grid, smem, s)
                               : tc_launch<3, false, true>(tp, map, grid, smem, s);
        return mn ? tc_launch<2, true, true>(tp, map, grid, smem, s)
                  : tc_launch<2, false, true>(tp, map, grid, smem, s);
    }
    if (px == 3) return mn ? tc_launch<3, true, false>(tp, map, grid, smem, s)
                           : tc_launch<3, false, false>(tp, map, grid, smem, s);
    return mn ? tc_launch<2, true, false>(tp, map, grid, smem, s)
              : tc_launch<2, false, false>(tp, map, grid, smem, s);
}

cudaError_t launch_tc_image(const float* const* fac, const int64_t* frad, int head, int C, int CP,
                            int64_t rad0, int64_t rad0p, void* image, cudaStream_t s) {
    ImgArgs ia;
    memset(&ia, 0, sizeof(ia));
    ia.head = head;
    ia.C = C;
    ia.CP = CP;
    ia.N = 3 * CP;
    for (int z = 0; z < head; ++z) { ia.fac[z] = fac[z]; ia.frad[z] = frad[z]; }
    ia.rad0 = rad0;
    ia.rad0p = rad0p;
    ia.img = static_cast<uint8_t*>(image);
    const int64_t items = (rad0p / 8) * CP;
    const int64_t blocks = (items + 255) / 256;
    const int grid = (int)(blocks < num_sms() * 8 ? blocks : num_sms() * 8);
    tc_image_kernel<<<grid, 256, 0, s>>>(ia);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace mtk
