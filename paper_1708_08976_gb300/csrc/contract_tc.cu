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
// Warp roles (288 threads): 8 converter warps load the tensor with coalesced
// 16-byte loads straight into registers (one stage ahead), split it, store the
// pieces, and drain the accumulator; one thread of warp 8 issues tcgen05.mma.
// The tensor goes through registers rather than TMA because the split needs it
// there; a TMA stage would add a shared-memory write and read per entry.
//
// Every mbarrier wait is bounded (1 s of %globaltimer); on expiry the kernel sets
// MTK_ETIMEOUT in the status word, stops, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <string.h>

#include "mtk_internal.cuh"

namespace mtk {
namespace {

constexpr int TC_BK = 64;                    // k per stage
constexpr int TC_M = 128;                    // MMA M
constexpr int CONV_WARPS = 8;
constexpr int CONV_THREADS = CONV_WARPS * 32;
constexpr int NTHREADS = CONV_THREADS + 32;  // + the MMA warp
constexpr int MAX_STAGES = 4;
constexpr int GROUP = 2;                     // stages per accumulation chain
constexpr int PIECE_BYTES = TC_M * 128;      // one BF16 piece of the 128 x 64 tensor tile
constexpr int MAX_CB = 64;                   // columns per launch
constexpr unsigned long long kWaitNs = 1000000000ull;

struct TcParams {
    ContractParams p;
    const uint8_t* bimg;    // B image: (rad0p / 64) slices of N x 128 bytes
    int ntail;
    const float* tail[MTK_MAXN];
    int64_t tail_rad[MTK_MAXN];
    int64_t rad0, rad0p, Kp;
    int BI, CP, N, stages, mn_major, stage_bytes, b_off, b_bytes, tmem_cols;
    uint32_t idesc;
};

// ---- PTX wrappers ---------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false if the limit expired or another thread flagged an abort
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long limit_ns) {
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > limit_ns) return false;
        }
    }
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// shared-memory matrix descriptor, 128-byte swizzle (tcgen05 format: version 1 at
// bits 46-47, layout type 2 = SWIZZLE_128B at bits 61-63)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- FP32 -> BF16 pieces ----------------------------------------------------------
__device__ __forceinline__ uint32_t pack2(float a, float b, float& ra, float& rb) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    ra = a - hf.x;     // exact (Sterbenz)
    rb = b - hf.y;
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack2_last(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// split 4 consecutive values into NP pieces of 4 BF16 (8 bytes each)
template <int NP>
__device__ __forceinline__ void split4(const float4 v, uint2* out) {
    float a = v.x, b = v.y, c = v.z, d = v.w;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        if (q + 1 < NP) {
            float ra, rb, rc, rd;
            out[q].x = pack2(a, b, ra, rb);
            out[q].y = pack2(c, d, rc, rd);
            a = ra; b = rb; c = rc; d = rd;
        } else {
            out[q].x = pack2_last(a, b);
            out[q].y = pack2_last(c, d);
        }
    }
}

// offsets inside one 128-byte-swizzled operand (bytes); 2-byte elements
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
    const int chunk = k >> 3, within = (k & 7) * 2;
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + (((chunk ^ (row & 7)) & 7) << 4) + within);
}
__device__ __forceinline__ uint32_t mnmajor_off(int i, int k) {    // 128 rows of i x 64 k
    const int a = i >> 6, g = k >> 3, kr = k & 7, chunk = (i & 63) >> 3;
    return (uint32_t)((g * 2 + a) * 1024 + kr * 128 + (((chunk ^ kr) & 7) << 4) + (i & 7) * 2);
}

__device__ __forceinline__ float4 ldg_stream(const float* ptr) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(ptr));
    return v;
}

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

__device__ __forceinline__ float tail_product(const TcParams& tp, int64_t q, int c, int C) {
    float prod = 1.0f;
    for (int t = 0; t < tp.ntail; ++t) {
        const int64_t rad = tp.tail_rad[t];
        const int64_t d = q % rad;
        q /= rad;
        prod *= __ldg(tp.tail[t] + d * C + c);
    }
    return prod;
}

// PX: tensor pieces; NCH: 16-column chunks of the output per converter thread;
// MN: the tensor operand is i-contiguous (I^L == 1)
template <int PX, int NCH, bool MN>
__global__ void __launch_bounds__(NTHREADS, 1)
contract_tc_kernel(const __grid_constant__ TcParams tp) {
    extern __shared__ uint8_t dsm_raw[];
    __shared__ __align__(8) uint64_t full_bar[MAX_STAGES];
    __shared__ __align__(8) uint64_t empty_bar[MAX_STAGES];
    __shared__ __align__(8) uint64_t accf_bar[2];
    __shared__ __align__(8) uint64_t acce_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ float qsh[CONV_WARPS][NCH * 16];     // per-warp tail scale of its columns

    const ContractParams& p = tp.p;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = threadIdx.x;
    uint8_t* dsm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t dsm_s = smem_u32(dsm);
    const int ST = tp.stages;

    const int64_t I = p.I, L = p.L;
    const int C = p.C, CP = tp.CP, N = tp.N;
    const int64_t i0 = (int64_t)blockIdx.x * tp.BI;
    const int rows = (int)((I - i0) < tp.BI ? (I - i0) : tp.BI);
    const int sp = blockIdx.y;
    const int64_t kb = (int64_t)sp * p.kchunk;                 // padded contraction index
    const int64_t ke = (kb + p.kchunk < tp.Kp) ? kb + p.kchunk : tp.Kp;
    const int nst = (int)((ke - kb + TC_BK - 1) / TC_BK);
    const int64_t rad0 = tp.rad0, rad0p = tp.rad0p;
    const int spr = (int)(rad0p / TC_BK);                      // stages per run

    if (t == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(smem_u32(&full_bar[s]), CONV_WARPS);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), CONV_WARPS);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zero the tensor pieces of every stage once: rows (K-major) or i-quads (MN-major)
    // beyond the tile are never written again and must read as zero
    for (int s = 0; s < ST; ++s) {
        uint4* z = reinterpret_cast<uint4*>(dsm + s * tp.stage_bytes);
        for (int e = t; e < tp.b_off / 16; e += NTHREADS) z[e] = make_uint4(0, 0, 0, 0);
    }
    if (warp == CONV_WARPS) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(tp.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == CONV_WARPS) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0 && nst > 0) {
            constexpr uint32_t a_lbo = MN ? 1024u : 16u;
            constexpr uint32_t a_sbo = MN ? 2048u : 1024u;
            constexpr uint32_t a_kstep = MN ? 4096u : 32u;
            int sir = (int)((kb % rad0p) / TC_BK);             // stage index within its run
            int g = 0;
            bool first = true, ok = true;
            uint32_t b = 0;
            for (int s = 0; s < nst; ++s) {
                const int slot = s % ST;
                if (!mbar_wait(smem_u32(&full_bar[slot]), (uint32_t)((s / ST) & 1), &abort_flag, kWaitNs)) {
                    ok = false;
                    break;
                }
                if (first) {
                    b = (uint32_t)(g & 1);
                    if (g >= 2 && !mbar_wait(smem_u32(&acce_bar[b]), (uint32_t)(((g >> 1) - 1) & 1), &abort_flag,
                                             kWaitNs)) {
                        ok = false;
                        break;
                    }
                }
                tc_fence_after();
                const uint32_t st = dsm_s + (uint32_t)(slot * tp.stage_bytes);
                const uint32_t dcol = tmem + b * (uint32_t)N;
#pragma unroll
                for (int kk = 0; kk < TC_BK / 16; ++kk) {
                    const uint64_t bdesc = make_desc(st + tp.b_off + kk * 32, 16, 1024);
#pragma unroll
                    for (int pc = 0; pc < PX; ++pc) {
                        const uint64_t adesc = make_desc(st + pc * PIECE_BYTES + kk * a_kstep, a_lbo, a_sbo);
                        mma_bf16(dcol, adesc, bdesc, tp.idesc, (first && kk == 0 && pc == 0) ? 0u : 1u);
                    }
                }
                if (s + ST < nst) mma_commit(smem_u32(&empty_bar[slot]));
                const bool last = ((sir + 1) % GROUP == 0) || (sir + 1 == spr) || (s == nst - 1);
                if (last) {
                    mma_commit(smem_u32(&accf_bar[b]));
                    ++g;
                }
                first = last;
                if (++sir == spr) sir = 0;
            }
            if (!ok) {
                abort_flag = 1;
                set_status(p.status, MTK_ETIMEOUT);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ converters
        // K-major: thread owns rows r_j = (t>>4) + 16 j and the k-quad 4*(t&15) of each
        // stage.  MN-major: float4 f_j = t + 256 j of the (rows/4 i-quads) x 64 k stage.
        const int kq = t & 15;
        const int r0 = t >> 4;
        const int nq = rows >> 2;
        int32_t moff[8];                                 // MN-major: i + I*k within a stage
        uint32_t msoff[8];
        int mkl[8];
        if constexpr (MN) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int f = t + CONV_THREADS * j;
                const int iq = nq > 0 ? f % nq : 0, kl = nq > 0 ? f / nq : TC_BK;
                const bool v = nq > 0 && kl < TC_BK;
                mkl[j] = v ? kl : TC_BK;
                moff[j] = v ? (int32_t)(4 * iq + I * kl) : 0;
                msoff[j] = v ? mnmajor_off(4 * iq, kl) : 0u;
            }
        }
        const uint32_t ksoff0 = kmajor_off(r0, 4 * kq);      // K-major: row r0, + 2048 per j
        // load tracker: padded position of the next stage to load, its run q and offset d0
        int64_t ld_k = kb, ld_q = kb / rad0p, ld_d0 = kb % rad0p;
        // (l, r) of the real index q*rad0 + d0 + 4*kq of this thread's k-quad (K-major)
        int64_t xl = 0, xr = 0;
        if constexpr (!MN) {
            const int64_t k0 = ld_q * rad0 + ld_d0 + 4 * kq;
            xl = k0 % L;
            xr = k0 / L;
        }
        auto load_stage = [&](float4 (&v)[8]) {
            if constexpr (!MN) {
                const bool kval = (ld_d0 + 4 * kq < rad0) && (ld_k + 4 * kq < ke);
                const float* base = p.X + xl + L * I * xr + L * (i0 + r0);
                const int64_t jstep = 16 * L;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    v[j] = (kval && r0 + 16 * j < rows) ? ldg_stream(base + j * jstep)
                                                        : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const float* base = p.X + i0 + I * (ld_q * rad0 + ld_d0);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    v[j] = (mkl[j] < TC_BK && ld_d0 + mkl[j] < rad0 && ld_k + mkl[j] < ke)
                               ? ldg_stream(base + moff[j])
                               : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            // advance to the next stage (skipping the padding at the end of a run)
            const int64_t delta = (ld_d0 + TC_BK == rad0p) ? (rad0 - ld_d0) : TC_BK;
            if constexpr (!MN) {
                xl += delta;
                while (xl >= L) { xl -= L; ++xr; }
            }
            ld_k += TC_BK;
            ld_d0 += TC_BK;
            if (ld_d0 == rad0p) { ld_d0 = 0; ++ld_q; }
        };

        // production tracker (stage index within its run)
        int pr_sir = (int)((kb % rad0p) / TC_BK);
        int64_t pr_q = kb / rad0p;

        auto produce = [&](const float4 (&v)[8], int s) -> bool {
            const int slot = s % ST;
            if (s >= ST) {
                if (!mbar_wait(smem_u32(&empty_bar[slot]), (uint32_t)(((s / ST) - 1) & 1), &abort_flag, kWaitNs)) {
                    abort_flag = 1;
                    set_status(p.status, MTK_ETIMEOUT);
                    return false;
                }
            }
            uint8_t* st = dsm + slot * tp.stage_bytes;
            if (warp == 0 && lane == 0) {
                const uint32_t fb = smem_u32(&full_bar[slot]);
                mbar_expect_tx(fb, (uint32_t)tp.b_bytes);
                bulk_copy_g2s(smem_u32(st + tp.b_off), tp.bimg + (int64_t)pr_sir * tp.b_bytes,
                              (uint32_t)tp.b_bytes, fb);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                uint32_t so;
                if constexpr (!MN) {
                    if (r0 + 16 * j >= rows) continue;
                    so = ksoff0 + (uint32_t)(j * 2048);
                } else {
                    if (mkl[j] >= TC_BK) continue;
                    so = msoff[j];
                }
                uint2 pcs[PX];
                split4<PX>(v[j], pcs);
#pragma unroll
                for (int q = 0; q < PX; ++q) *reinterpret_cast<uint2*>(st + q * PIECE_BYTES + so) = pcs[q];
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&full_bar[slot]));
            return true;
        };

        // accumulator drain state
        const int sub = warp & 3, half = warp >> 2;
        float acc[NCH * 16];
#pragma unroll
        for (int e = 0; e < NCH * 16; ++e) acc[e] = 0.0f;
        float* qc = qsh[warp];                           // the columns are warp-uniform
        for (int e = lane; e < NCH * 16; e += 32) qc[e] = 1.0f;
        __syncwarp();
        int64_t q_cached = -1;
        auto drain = [&](int g, int64_t q) -> bool {
            const int b = g & 1;
            if (!mbar_wait(smem_u32(&accf_bar[b]), (uint32_t)((g >> 1) & 1), &abort_flag, kWaitNs)) {
                abort_flag = 1;
                set_status(p.status, MTK_ETIMEOUT);
                return false;
            }
            tc_fence_after();
            if (tp.ntail > 0 && q != q_cached) {
                __syncwarp();
                for (int e = lane; e < NCH * 16; e += 32) {
                    const int c = 16 * half + 32 * (e >> 4) + (e & 15);
                    qc[e] = (c < C) ? tail_product(tp, q, c, C) : 0.0f;
                }
                q_cached = q;
                __syncwarp();
            }
#pragma unroll
            for (int m = 0; m < NCH; ++m) {
                const int cc = 16 * half + 32 * m;
                if (cc < CP) {                            // warp-uniform
                    float sum[16], v[16];
                    const uint32_t ta = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(b * N + cc);
                    tmem_ld16(ta, sum);
                    tmem_ld_wait();
                    tmem_ld16(ta + (uint32_t)CP, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) sum[j] += v[j];
                    tmem_ld16(ta + (uint32_t)(2 * CP), v);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[m * 16 + j] = fmaf(sum[j] + v[j], qc[m * 16 + j], acc[m * 16 + j]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce_bar[b]));
            return true;
        };

        float4 va[8], vb[8];
        int g = 0;
        bool pending = false, ok = true;
        int pend_g = 0;
        int64_t pend_q = 0;
        // one production step: stage s from registers v, then drain the previous group
        auto step = [&](const float4 (&v)[8], int s) -> bool {
            if (!produce(v, s)) return false;
            const bool last = ((pr_sir + 1) % GROUP == 0) || (pr_sir + 1 == spr) || (s == nst - 1);
            const int64_t q_s = pr_q;
            if (++pr_sir == spr) { pr_sir = 0; ++pr_q; }
            if (last) {
                if (pending && !drain(pend_g, pend_q)) return false;
                pend_g = g;
                pend_q = q_s;
                pending = true;
                ++g;
            }
            return true;
        };
        if (nst > 0) load_stage(va);
        for (int s = 0; s < nst && ok; s += 2) {
            if (s + 1 < nst) load_stage(vb);
            if (!step(va, s)) { ok = false; break; }
            if (s + 1 >= nst) break;
            if (s + 2 < nst) load_stage(va);
            if (!step(vb, s + 1)) { ok = false; break; }
        }
        if (ok && pending) ok = drain(pend_g, pend_q);

        // ------------------------------------------------------------ epilogue
        const int row = sub * 32 + lane;
        if (ok && row < rows) {
            const int64_t i = i0 + row;
#pragma unroll
            for (int m = 0; m < NCH; ++m)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = 16 * half + 32 * m + j;
                    if (c < C) {
                        if (p.S == 1) p.out[i * p.out_si + c * p.out_sc] = acc[m * 16 + j];
                        else p.part[((int64_t)sp * I + i) * C + c] = acc[m * 16 + j];
                    }
                }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (warp == CONV_WARPS) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tp.tmem_cols));
    }
}

int tile_rows(int64_t I) {
    const int64_t tiles = (I + TC_M - 1) / TC_M;
    int64_t bi = (I + tiles - 1) / tiles;
    bi = (bi + 3) & ~3LL;
    return (int)(bi > TC_M ? TC_M : bi);
}

template <int PX, int NCH, bool MN>
cudaError_t launch_variant(const TcParams& tp, dim3 grid, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(contract_tc_kernel<PX, NCH, MN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    contract_tc_kernel<PX, NCH, MN><<<grid, NTHREADS, smem, s>>>(tp);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

bool contract_tc_shape_ok(int64_t L, int64_t I, int C, int precision) {
    if (precision != MTK_PREC_BF16X2 && precision != MTK_PREC_BF16X3) return false;
    if (C < 1 || C > MAX_CB) return false;
    if (L == 1) return I % 4 == 0 && I < (int64_t(1) << 24);   // 16-byte loads along i
    return L % 4 == 0;                                          // 16-byte loads along k
}

TcPlan contract_tc_plan(const int64_t* frad, int nfac, int64_t I, int C) {
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
    pl.Kp = (K / prod) * pl.rad0p;
    pl.BI = tile_rows(I);
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
    const TcPlan pl = contract_tc_plan(p.frad, p.nfac, p.I, p.C);
    TcParams tp;
    memset(&tp, 0, sizeof(tp));
    tp.p = p;
    tp.bimg = static_cast<const uint8_t*>(image);
    tp.ntail = p.nfac - pl.head;
    for (int z = pl.head; z < p.nfac; ++z) {
        tp.tail[z - pl.head] = p.fac[z];
        tp.tail_rad[z - pl.head] = p.frad[z];
    }
    tp.rad0 = pl.rad0;
    tp.rad0p = pl.rad0p;
    tp.Kp = pl.Kp;
    tp.BI = pl.BI;
    tp.CP = pl.CP;
    tp.N = pl.N;
    tp.mn_major = p.L == 1 ? 1 : 0;
    const int px = precision == MTK_PREC_BF16X3 ? 3 : 2;
    tp.b_off = px * PIECE_BYTES;
    tp.b_bytes = pl.N * 128;
    tp.stage_bytes = tp.b_off + ((tp.b_bytes + 1023) & ~1023);
    tp.stages = (int)((200 * 1024) / tp.stage_bytes);
    if (tp.stages > MAX_STAGES) tp.stages = MAX_STAGES;
    if (tp.stages < 2) tp.stages = 2;
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
    int grid_img = (int)(blocks < 152 * 8 ? blocks : 152 * 8);
    tc_image_kernel<<<grid_img, 256, 0, s>>>(ia);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    // 2) the contraction
    const size_t smem = (size_t)tp.stages * tp.stage_bytes + 1024;
    const int64_t tiles = (p.I + tp.BI - 1) / tp.BI;
    const dim3 grid((unsigned)tiles, (unsigned)p.S);
    const int nch = pl.CP <= 32 ? 1 : 2;
    const bool mn = tp.mn_major != 0;
    if (px == 3) {
        if (nch == 1) return mn ? launch_variant<3, 1, true>(tp, grid, smem, s) : launch_variant<3, 1, false>(tp, grid, smem, s);
        return mn ? launch_variant<3, 2, true>(tp, grid, smem, s) : launch_variant<3, 2, false>(tp, grid, smem, s);
    }
    if (nch == 1) return mn ? launch_variant<2, 1, true>(tp, grid, smem, s) : launch_variant<2, 1, false>(tp, grid, smem, s);
    return mn ? launch_variant<2, 2, true>(tp, grid, smem, s) : launch_variant<2, 2, false>(tp, grid, smem, s);
}

}  // namespace mtk
