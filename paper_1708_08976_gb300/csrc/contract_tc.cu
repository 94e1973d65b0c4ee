// contract_tc.cu -- tensor-core (tcgen05 / TMEM) form of the MTTKRP contraction
//     D(i, c) = sum_k X3(k, i) W(k, c)
// on the 3-way view of the tensor (Fig. 2: the mode-n matricization is R row-major
// I x L blocks, consumed in place), with the Khatri-Rao rows W(k, :) generated on
// chip (Algorithm 3 forms K_R(j,:) kr K_L per block; here 64 consecutive k at a
// time, never written to HBM).
//
// Precision (split products).  The tensor is FP32.  Each entry x is split into
// BF16 pieces x = x_1 + x_2 (+ x_3) by round-to-nearest on the successive
// remainders (the bf16x3 / bf16x6 schemes of Henry, Tang and Heinecke, ARITH
// 2019); every KRP entry w is split into three pieces.  One MMA per tensor piece
// multiplies it against all three W pieces at once (they are stacked along N),
// so every cross product x_a * w_b is formed and accumulated in FP32 in TMEM.
// With 2 tensor pieces the representation error of x is <= 2^-16 |x|; with 3 it
// is <= 2^-24 |x|, the FP32 unit roundoff.
//
// Tile: MMA M = 128 rows of i (the CTA owns BI <= 128 of them), N = 3 * CP
// (CP = C rounded up to 16), K = 64 per stage (one 128-byte swizzle row of BF16).
// Operands in shared memory use the canonical 128-byte-swizzled layouts: the
// KRP operand B is K-major; the tensor operand A is K-major when k runs along the
// contiguous mode (I^L > 1) and MN-major when i is the contiguous index (mode 0,
// I^L = 1).
//
// Warp roles (288 threads): 8 converter warps load the tensor with coalesced
// 16-byte loads straight into registers (one stage prefetched ahead), split it
// into BF16 pieces and store them in the swizzled layout, generate the W
// pieces, then arrive on the stage's "full" mbarrier; one thread of warp 8 issues
// tcgen05.mma and commits to the stage's "empty" mbarrier.  After the last stage
// the converter warps read the accumulator from TMEM (tcgen05.ld), add the three
// W-piece column groups and write the CTA's partial sum.  Staging the tensor
// through TMA instead would add 8 bytes of shared-memory traffic per entry (TMA
// write + read back for the split), on top of ~12 bytes the split and the MMA
// already need.
//
// Every mbarrier wait is bounded (1 s of %globaltimer); on expiry the kernel
// sets MTK_ETIMEOUT in the status word, stops producing and issuing, waits
// (bounded) for its issued MMAs, frees its TMEM and returns.
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
constexpr int STAGES = 2;
constexpr int PIECE_BYTES = TC_M * 128;      // one BF16 piece of the 128 x 64 tensor tile
constexpr int MAX_CB = 64;                   // columns per launch
constexpr unsigned long long kWaitNs = 1000000000ull;

struct TcParams {
    ContractParams p;
    int BI;           // rows of i owned by a CTA (<= 128)
    int CP;           // columns per W piece in the B operand (C rounded up to 16)
    int N;            // MMA N = 3 * CP
    int px;           // tensor pieces (2 or 3)
    int mn_major;     // A is i-contiguous (I^L == 1)
    int stage_bytes;  // bytes per pipeline stage
    int b_off;        // offset of B inside a stage
    int tmem_cols;
    uint32_t idesc;
};

// ---- PTX wrappers ---------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
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

// split 4 consecutive values into NP pieces of 4 BF16 (8 bytes each)
template <int NP>
__device__ __forceinline__ void split4(const float4 v, uint2* out) {
    float a = v.x, b = v.y, c = v.z, d = v.w;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float ra, rb, rc, rd;
        out[q].x = pack2(a, b, ra, rb);
        out[q].y = pack2(c, d, rc, rd);
        a = ra; b = rb; c = rc; d = rd;
    }
}

// offsets inside one 128-byte-swizzled operand (bytes)
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {   // k: element index, 2-byte elements
    const int chunk = k >> 3, within = (k & 7) * 2;
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + (((chunk ^ (row & 7)) & 7) << 4) + within);
}
__device__ __forceinline__ uint32_t mnmajor_off(int i, int k) {    // 128 rows of i x 64 k
    const int a = i >> 6, g = k >> 3, kr = k & 7, chunk = (i & 63) >> 3;
    return (uint32_t)((g * 2 + a) * 1024 + kr * 128 + (((chunk ^ kr) & 7) << 4) + (i & 7) * 2);
}

__device__ __forceinline__ float4 ldg_stream(const float* p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ float tail_product(const KrpOperand& W, int64_t q, int c, int C) {
    float prod = 1.0f;
    for (int t = 0; t < W.ntail; ++t) {
        const int64_t rad = W.tail_rad[t];
        const int64_t d = q % rad;
        q /= rad;
        prod *= __ldg(W.tail[t] + d * C + c);
    }
    return prod;
}

template <int PX>
__global__ void __launch_bounds__(NTHREADS, 1)
contract_tc_kernel(const __grid_constant__ TcParams tp) {
    extern __shared__ uint8_t dsm_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t empty_bar[STAGES];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ float qs_all[CONV_WARPS][2][MAX_CB];   // one copy per converter warp

    const ContractParams& p = tp.p;
    const KrpOperand& W = p.W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = threadIdx.x;
    uint8_t* dsm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t dsm_s = smem_u32(dsm);

    const int64_t I = p.I, L = p.L, K = p.K;
    const int C = p.C, CP = tp.CP;
    const int64_t i0 = (int64_t)blockIdx.x * tp.BI;
    const int rows = (int)((I - i0) < tp.BI ? (I - i0) : tp.BI);
    const int sp = blockIdx.y;
    const int64_t kb = (int64_t)sp * p.kchunk;
    const int64_t ke = (kb + p.kchunk < K) ? kb + p.kchunk : K;
    const int nst = (int)((ke - kb + TC_BK - 1) / TC_BK);

    if (t == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&full_bar[s]), CONV_WARPS);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&done_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zero every stage once: rows of A beyond `rows` and columns of B beyond the real
    // W pieces are never written again and must read as zero
    {
        uint4* z = reinterpret_cast<uint4*>(dsm);
        const int n16 = STAGES * tp.stage_bytes / 16;
        for (int e = t; e < n16; e += NTHREADS) z[e] = make_uint4(0, 0, 0, 0);
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
        if (lane == 0) {
            const uint32_t a_lbo = tp.mn_major ? 1024u : 16u;
            const uint32_t a_sbo = tp.mn_major ? 2048u : 1024u;
            const uint32_t a_kstep = tp.mn_major ? 4096u : 32u;
            bool ok = true;
            for (int s = 0; s < nst; ++s) {
                const int slot = s % STAGES;
                if (!mbar_wait(smem_u32(&full_bar[slot]), (uint32_t)((s / STAGES) & 1), &abort_flag, kWaitNs)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t st = dsm_s + (uint32_t)(slot * tp.stage_bytes);
#pragma unroll
                for (int kk = 0; kk < TC_BK / 16; ++kk) {
                    const uint64_t bdesc = make_desc(st + tp.b_off + kk * 32, 16, 1024);
#pragma unroll
                    for (int pc = 0; pc < PX; ++pc) {
                        const uint64_t adesc = make_desc(st + pc * PIECE_BYTES + kk * a_kstep, a_lbo, a_sbo);
                        mma_bf16(tmem, adesc, bdesc, tp.idesc, (s | kk | pc) != 0 ? 1u : 0u);
                    }
                }
                if (s + STAGES < nst) mma_commit(smem_u32(&empty_bar[slot]));
            }
            if (!ok) {
                abort_flag = 1;
                set_status(p.status, MTK_ETIMEOUT);
            }
            if (nst > 0) mma_commit(smem_u32(&done_bar));   // arrives once every issued MMA has completed
            else mbar_arrive(smem_u32(&done_bar));
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ converters
        // tensor loads: K-major -> thread owns rows r_j = (t>>4) + 16 j and the k-quad
        // 4*(t&15) of every stage; MN-major -> float4 f_j = t + 256 j of the
        // (rows/4 i-quads) x 64 k stage, i-quad fastest.
        const int kq = t & 15;
        const int nq = rows >> 2;                       // i-quads (MN-major; rows % 4 == 0)
        int64_t goff[8];                                // stage-invariant part of the address
        uint32_t soff[8];                               // offset in a piece
        int kloc[8];                                    // k within the stage (MN-major)
        bool rvalid[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (!tp.mn_major) {
                const int r = (t >> 4) + 16 * j;
                rvalid[j] = r < rows;
                goff[j] = L * (i0 + r);
                soff[j] = kmajor_off(r, 4 * kq);
                kloc[j] = 4 * kq;
            } else {
                const int f = t + CONV_THREADS * j;
                const int iq = nq > 0 ? f % nq : 0, kl = nq > 0 ? f / nq : TC_BK;
                rvalid[j] = nq > 0 && kl < TC_BK;
                goff[j] = i0 + 4 * iq + I * (int64_t)kl;
                soff[j] = rvalid[j] ? mnmajor_off(4 * iq, kl) : 0u;
                kloc[j] = kl;
            }
        }
        // X tracker: (l, r) of the k-quad of this thread at the next stage to load
        int64_t xl = 0, xr = 0;
        if (!tp.mn_major) {
            const int64_t k0 = kb + 4 * kq;
            xl = k0 % L;
            xr = k0 / L;
        }
        int64_t xks = kb;                               // first k of the next stage to load
        // W tracker: (d0, q) of the first k of the stage being produced
        int64_t wd = kb % W.rad0, wq = kb / W.rad0;
        int64_t qcached = -1;
        const int64_t qtot = K / W.rad0;

        float (*qs)[MAX_CB] = qs_all[warp];
        auto load_stage = [&](float4 (&v)[8]) {
            const int64_t ks = xks;
            if (!tp.mn_major) {
                const bool kval = ks + 4 * kq < ke;
                const float* base = p.X + xl + L * I * xr;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    v[j] = (kval && rvalid[j]) ? ldg_stream(base + goff[j]) : make_float4(0.f, 0.f, 0.f, 0.f);
                xl += TC_BK;
                while (xl >= L) { xl -= L; ++xr; }
            } else {
                const float* base = p.X + I * ks;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    v[j] = (rvalid[j] && ks + kloc[j] < ke) ? ldg_stream(base + goff[j])
                                                          : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            xks += TC_BK;
        };

        auto produce = [&](const float4 (&v)[8], int s) -> bool {
            const int slot = s % STAGES;
            if (s >= STAGES) {
                if (!mbar_wait(smem_u32(&empty_bar[slot]), (uint32_t)(((s / STAGES) - 1) & 1), &abort_flag,
                               kWaitNs)) {
                    abort_flag = 1;
                    set_status(p.status, MTK_ETIMEOUT);
                    return false;
                }
            }
            uint8_t* st = dsm + slot * tp.stage_bytes;
            // tensor pieces
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (!rvalid[j]) continue;
                uint2 pcs[PX];
                split4<PX>(v[j], pcs);
#pragma unroll
                for (int q = 0; q < PX; ++q)
                    *reinterpret_cast<uint2*>(st + q * PIECE_BYTES + soff[j]) = pcs[q];
            }
            // Q rows for this stage's q and q+1, refreshed by each warp for its own copy
            // (no cross-warp barrier, so a warp that stops early cannot strand others)
            if (W.ntail > 0 && wq != qcached) {
                __syncwarp();
                for (int e = lane; e < 2 * MAX_CB; e += 32) {
                    const int which = e / MAX_CB, c = e % MAX_CB;
                    qs[which][c] = (c < C && wq + which < qtot) ? tail_product(W, wq + which, c, C) : 0.0f;
                }
                qcached = wq;
                __syncwarp();
            }
            // W pieces: item (c, oct) -> 8 consecutive k of column c, three BF16 pieces
            const int64_t ks = kb + (int64_t)s * TC_BK;
            uint8_t* bst = st + tp.b_off;
            for (int it = t; it < C * 8; it += CONV_THREADS) {
                const int c = it >> 3, oct = it & 7;
                float w[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int kl = oct * 8 + j;
                    float val = 0.0f;
                    if (ks + kl < ke) {
                        int64_t d = wd + kl;
                        int which = 0;
                        if (W.ntail > 0 && d >= W.rad0) { d -= W.rad0; which = 1; }
                        val = __ldg(W.f0 + d * C + c);
                        if (W.ntail > 0) val *= qs[which][c];
                    }
                    w[j] = val;
                }
                uint2 lo4[3], hi4[3];
                split4<3>(make_float4(w[0], w[1], w[2], w[3]), lo4);
                split4<3>(make_float4(w[4], w[5], w[6], w[7]), hi4);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int n = q * CP + c;
                    const uint32_t off = (uint32_t)((n >> 3) * 1024 + (n & 7) * 128 + (((oct ^ (n & 7)) & 7) << 4));
                    *reinterpret_cast<uint4*>(bst + off) = make_uint4(lo4[q].x, lo4[q].y, hi4[q].x, hi4[q].y);
                }
            }
            wd += TC_BK;
            while (wd >= W.rad0) { wd -= W.rad0; ++wq; }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&full_bar[slot]));
            return true;
        };

        float4 va[8], vb[8];
        if (nst > 0) load_stage(va);
        for (int s = 0; s < nst; s += 2) {
            if (s + 1 < nst) load_stage(vb);
            if (!produce(va, s)) break;
            if (s + 1 >= nst) break;
            if (s + 2 < nst) load_stage(va);
            if (!produce(vb, s + 1)) break;
        }

        // ------------------------------------------------------------ epilogue
        const bool done = mbar_wait(smem_u32(&done_bar), 0u, &abort_flag, 8ull * kWaitNs);
        if (!done) set_status(p.status, MTK_ETIMEOUT);
        tc_fence_after();
        const int sub = warp & 3;                       // TMEM lanes 32*sub .. 32*sub+31
        const int row = sub * 32 + lane;
        const int64_t i = i0 + row;
        const bool live = done && row < rows && nst > 0;
        for (int cc = (warp >> 2) * 16; cc < CP; cc += 32) {
            float a0[16], a1[16], a2[16];
            const uint32_t ta = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)cc;
            tmem_ld16(ta, a0);
            tmem_ld16(ta + (uint32_t)CP, a1);
            tmem_ld16(ta + (uint32_t)(2 * CP), a2);
            tmem_ld_wait();
            if (live) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = cc + j;
                    if (c < C) {
                        const float v = (a0[j] + a1[j]) + a2[j];
                        if (p.S == 1) p.out[i * p.out_si + c * p.out_sc] = v;
                        else p.part[((int64_t)sp * I + i) * C + c] = v;
                    }
                }
            }
        }
        if (nst == 0 && row < rows) {
            for (int c = (warp >> 2); c < C; c += 2) {
                if (p.S == 1) p.out[i * p.out_si + c * p.out_sc] = 0.0f;
                else p.part[((int64_t)sp * I + i) * C + c] = 0.0f;
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

int pieces_for(int precision) { return precision == MTK_PREC_BF16X3 ? 3 : 2; }

TcParams make_tc_params(const ContractParams& p, int precision) {
    TcParams tp;
    memset(&tp, 0, sizeof(tp));
    tp.p = p;
    tp.BI = tile_rows(p.I);
    tp.CP = (p.C + 15) & ~15;
    tp.N = 3 * tp.CP;
    tp.px = pieces_for(precision);
    tp.mn_major = p.L == 1 ? 1 : 0;
    tp.b_off = tp.px * PIECE_BYTES;
    const int bbytes = ((tp.N * 128) + 1023) & ~1023;
    tp.stage_bytes = tp.b_off + bbytes;
    int cols = 32;
    while (cols < tp.N) cols <<= 1;
    tp.tmem_cols = cols;
    // kind::f16 instruction descriptor: D = F32 (bits 4-5), A = B = BF16 (bits 7-9,
    // 10-12), A major (bit 15), B K-major, N >> 3 (bits 17-22), M >> 4 (bits 24-28)
    tp.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)tp.mn_major << 15) |
               ((uint32_t)(tp.N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    return tp;
}

}  // namespace

int contract_tc_i_tile_rows(int64_t I) { return tile_rows(I); }

bool contract_tc_shape_ok(int64_t L, int64_t I, int C, int precision) {
    if (precision != MTK_PREC_BF16X2 && precision != MTK_PREC_BF16X3) return false;
    if (C < 1 || C > MAX_CB) return false;
    if (L == 1) return I % 4 == 0;     // 16-byte loads along i
    return L % 4 == 0;                 // 16-byte loads along k
}

bool contract_tc_supported(const ContractParams& p, int precision) {
    if (!contract_tc_shape_ok(p.L, p.I, p.C, precision)) return false;
    if ((reinterpret_cast<uintptr_t>(p.X) & 15) != 0) return false;
    if (p.W.ntail > 0 && p.W.rad0 < TC_BK) return false;
    if (p.kchunk <= 0 || p.kchunk % TC_BK != 0) return false;
    return true;
}

cudaError_t launch_contract_tc(const ContractParams& p, int precision, cudaStream_t s) {
    const TcParams tp = make_tc_params(p, precision);
    const size_t smem = (size_t)STAGES * tp.stage_bytes + 1024;
    const int64_t tiles = (p.I + tp.BI - 1) / tp.BI;
    dim3 grid((unsigned)tiles, (unsigned)p.S);
    cudaError_t e;
    if (tp.px == 3) {
        e = cudaFuncSetAttribute(contract_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        contract_tc_kernel<3><<<grid, NTHREADS, smem, s>>>(tp);
        note_launches(1);
    } else {
        e = cudaFuncSetAttribute(contract_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        contract_tc_kernel<2><<<grid, NTHREADS, smem, s>>>(tp);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace mtk
