// contract_tc_kernel.cuh -- the tcgen05 split-BF16 contraction kernel of contract_tc.cu.
//
// The kernel template has eight variants (tensor pieces PX = 2 or 3, a K-major or MN-major
// tensor operand, TMA or cp.async staging).  Each (PX, MN) pair is instantiated in a
// translation unit of its own (contract_tc_px*.cu) through tc_launch, so that the
// variants compile in parallel; contract_tc.cu holds the planning and the dispatch.
// The algorithm, the operand layouts and the warp roles are described in contract_tc.cu.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <string.h>

#include "mtk_internal.cuh"
#include "tc_ptx.cuh"

// pipeline shape (compile-time; the defaults are the tuned ones)
#ifndef MTK_TC_CONV_WARPS
#define MTK_TC_CONV_WARPS 8
#endif
#ifndef MTK_TC_AB_STAGES
#define MTK_TC_AB_STAGES 3
#endif

namespace mtk {
namespace tcd {   // shared by the planning code and the kernel variants

constexpr int TC_BK = 64;                    // k per stage
constexpr int TC_M = 128;                    // MMA M
constexpr int CONV_WARPS = MTK_TC_CONV_WARPS;
constexpr int CONV_THREADS = CONV_WARPS * 32;
constexpr int NTHREADS = CONV_THREADS + 64;  // + the MMA warp + the TMA producer warp
constexpr int QW = CONV_WARPS / 4;           // converter warps per TMEM sub-partition
constexpr int NCH = (64 + 16 * QW - 1) / (16 * QW);   // 16-column chunks per drain thread
constexpr int MAX_STAGES = 4;
constexpr int MAX_STAGING = 4;               // stages of tensor data in flight per thread
constexpr int GROUP = 2;                     // stages per accumulation chain
constexpr int PIECE_BYTES = TC_M * 128;      // one BF16 piece of the 128 x 64 tensor tile
constexpr int MAX_CB = 64;                   // columns per launch (one 16-column chunk per drain thread)
constexpr int RPT = 1024 / CONV_THREADS;     // tile rows (or row octets) per converter thread per stage
constexpr unsigned long long kWaitNs = 1000000000ull;

struct TcParams {
    ContractParams p;
    const uint8_t* bimg;    // B image: (rad0p / 64) slices of N x 128 bytes
    int ntail;
    const float* tail[MTK_MAXN];
    int64_t tail_rad[MTK_MAXN];
    int64_t rad0, rad0p, Kp, nruns;
    int BI, U, CP, N, stages, P, mn_major, linear, nslabs;
    int kwide;              // TMA, K-major: one 64-k box per row set (contiguous runs), else octet boxes
    int stage_bytes, b_off, b_bytes, stg_off, tmem_cols;
    uint32_t idesc;
    unsigned long long wait_ns;   // limit of every wait that an abort can end (kWaitNs by default)
    int stall;              // test hook: the MMA issuer first waits on a barrier that nothing completes
};

}  // namespace tcd

namespace {

using namespace tc;
using namespace tcd;

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

// PX: tensor pieces; MN: the tensor operand is i-contiguous (I^L == 1);
// TMA: the tensor is staged by TMA tile loads (tensor map `xmap`) issued by a producer
// warp, else by per-thread 16-byte cp.async copies.
template <int PX, bool MN, bool TMA>
__global__ void __launch_bounds__(NTHREADS, 1)
contract_tc_kernel(const __grid_constant__ TcParams tp, const __grid_constant__ CUtensorMap xmap) {
    extern __shared__ uint8_t dsm_raw[];
    __shared__ __align__(8) uint64_t full_bar[MAX_STAGES];
    __shared__ __align__(8) uint64_t empty_bar[MAX_STAGES];
    __shared__ __align__(8) uint64_t xfull_bar[MAX_STAGING];
    __shared__ __align__(8) uint64_t xempty_bar[MAX_STAGING];
    __shared__ __align__(8) uint64_t accf_bar[2];
    __shared__ __align__(8) uint64_t acce_bar[2];
    __shared__ __align__(8) uint64_t fin_bar, stall_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int b_issued;                 // stages whose B-image copy has been issued

    const ContractParams& p = tp.p;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = threadIdx.x;
    uint8_t* dsm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t dsm_s = smem_u32(dsm);
    const int ST = tp.stages;

    const int64_t I = p.I, L = p.L;
    const int C = p.C, CP = tp.CP, N = tp.N;
    const int BI = tp.BI, U = tp.U;
    const int64_t i0 = (int64_t)blockIdx.x * BI;
    const int rows = (int)((I - i0) < BI ? (I - i0) : BI);   // rows of i in each packed group
    const int sp = blockIdx.y;
    const int64_t kb = (int64_t)sp * p.kchunk;                 // padded index over run-groups
    const int64_t ke = (kb + p.kchunk < tp.Kp) ? kb + p.kchunk : tp.Kp;
    const int nst = (int)((ke - kb + TC_BK - 1) / TC_BK);
    const int64_t rad0 = tp.rad0, rad0p = tp.rad0p, nruns = tp.nruns;
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
        for (int x = 0; x < MAX_STAGING; ++x) {
            mbar_init(smem_u32(&xfull_bar[x]), 1);
            mbar_init(smem_u32(&xempty_bar[x]), CONV_WARPS);
        }
        mbar_init(smem_u32(&fin_bar), 1);
        mbar_init(smem_u32(&stall_bar), 1);
        abort_flag = 0;
        b_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zero the tensor pieces of every stage once: rows beyond the packed tile are never
    // written again and must read as zero
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
            if (tp.stall && !mbar_wait(smem_u32(&stall_bar), 0u, &abort_flag, tp.wait_ns)) ok = false;
            for (int s = 0; ok && s < nst; ++s) {
                const int slot = s % ST;
                if (!mbar_wait(smem_u32(&full_bar[slot]), (uint32_t)((s / ST) & 1), &abort_flag, tp.wait_ns)) {
                    ok = false;
                    break;
                }
                if (first) {
                    b = (uint32_t)(g & 1);
                    if (g >= 2 && !mbar_wait(smem_u32(&acce_bar[b]), (uint32_t)(((g >> 1) - 1) & 1), &abort_flag,
                                             tp.wait_ns)) {
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
            // every MMA issued by this thread (and the barrier arrivals of its commits) has
            // completed once fin_bar flips; this wait ignores the abort flag
            mma_commit(smem_u32(&fin_bar));
            volatile int never = 0;
            (void)mbar_wait(smem_u32(&fin_bar), 0u, &never, kWaitNs);
        }
        __syncwarp();
    } else if (warp == CONV_WARPS + 1) {
        // ------------------------------------------------------------ TMA producer
        if constexpr (TMA) {
            if (lane == 0) {
                const uint32_t stg0 = dsm_s + (uint32_t)tp.stg_off;
                const uint32_t stg_bytes = (uint32_t)(2 * RPT * CONV_THREADS * 16);
                // bytes every stage delivers (boxes include their out-of-range zeros)
                const uint32_t bytes = (uint32_t)(U * BI * TC_BK * 4);
                int64_t ld_qg = kb / rad0p, ld_d0 = kb % rad0p;
                int64_t xl = 0, xr = 0;                 // non-linear runs: (l, r) of the stage start
                if constexpr (!MN) {
                    if (!tp.linear) {
                        const int64_t k0 = ld_qg * rad0 + ld_d0;
                        xl = k0 % L;
                        xr = k0 / L;
                    }
                }
                int issued = 0;
                for (int s = 0; s < nst; ++s) {
                    const int slot = s % tp.P;
                    if (s >= tp.P &&
                        !mbar_wait(smem_u32(&xempty_bar[slot]), (uint32_t)(((s / tp.P) - 1) & 1), &abort_flag, tp.wait_ns)) {
                        abort_flag = 1;
                        set_status(p.status, MTK_ETIMEOUT);
                        break;
                    }
                    ++issued;
                    const uint32_t fb = smem_u32(&xfull_bar[slot]);
                    const uint32_t dst = stg0 + (uint32_t)slot * stg_bytes;
                    mbar_arrive_expect_tx(fb, bytes);
                    for (int u = 0; u < U; ++u) {
                        const int64_t q = ld_qg * U + u;
                        if constexpr (MN) {
                            // box (BI i, 64 k) of run q at d0; k = r for I^L == 1
                            const int64_t r0 = q * rad0 + ld_d0;
                            tma_load_2d(dst + (uint32_t)(u * BI * TC_BK * 4), &xmap, (int)(U > 1 ? 0 : i0),
                                        (int)(r0 < ((int64_t)1 << 31) - 1 ? r0 : ((int64_t)1 << 31) - 1), fb);
                        } else if (tp.kwide) {
                            // one box (64 k, BI rows) of the contiguous run q
                            const int64_t k0 = q * rad0;
                            int64_t r = k0 / L;
                            if (r > ((int64_t)1 << 31) - 1) r = ((int64_t)1 << 31) - 1;
                            tma_load_3d(dst + (uint32_t)(u * BI * TC_BK * 4), &xmap, (int)((k0 % L) + ld_d0),
                                        (int)(U > 1 ? 0 : i0), (int)r, fb);
                        } else {
                            // eight boxes (8 k, BI rows): one per k-octet plane
                            for (int o = 0; o < 8; ++o) {
                                int64_t l, r;
                                if (tp.linear) {
                                    const int64_t k0 = q * rad0;
                                    l = (k0 % L) + ld_d0 + 8 * o;
                                    r = k0 / L;
                                } else {
                                    l = xl + 8 * o;
                                    r = xr;
                                    while (l >= L) { l -= L; ++r; }
                                }
                                if (r > ((int64_t)1 << 31) - 1) r = ((int64_t)1 << 31) - 1;
                                tma_load_3d(dst + (uint32_t)(o * TC_M * 32 + u * BI * 32), &xmap, (int)l,
                                            (int)(U > 1 ? 0 : i0), (int)r, fb);
                            }
                        }
                    }
                    // next stage (skipping the padding at the end of a run)
                    if constexpr (!MN) {
                        if (!tp.linear) {
                            const int64_t delta = (ld_d0 + TC_BK == rad0p) ? (rad0 - ld_d0) : TC_BK;
                            xl += delta;
                            while (xl >= L) { xl -= L; ++xr; }
                        }
                    }
                    ld_d0 += TC_BK;
                    if (ld_d0 == rad0p) { ld_d0 = 0; ++ld_qg; }
                }
                // the loads of the last P stages may still be in flight when another role has
                // aborted: let them land before the CTA leaves (consumed phases return at once)
                for (int s = issued > tp.P ? issued - tp.P : 0; s < issued; ++s) {
                    volatile int never = 0;
                    (void)mbar_wait(smem_u32(&xfull_bar[s % tp.P]), (uint32_t)((s / tp.P) & 1), &never, kWaitNs);
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ converters
        // Tile row m (0..127) is (u, il) = (m / BI, m % BI): output row i0 + il of run
        // q = qg*U + u of the current run-group qg.  Each thread moves RPT rows x 8
        // values per stage as 2*RPT float4 (two adjacent 16-byte loads per row):
        //   K-major:  rows m_j = (t>>3) + (CONV_THREADS/8) j, values k = 8*(t&7) .. +7;
        //   MN-major: octet f_j = t + CONV_THREADS j of the (U*BI/8 row-octets) x 64 k stage,
        //             values i = 8*(f % nmo) .. +7 at k = f / nmo.
        // The 8 values become one 16-byte store per BF16 piece.
        const int ko = t & 7;
        const int nmo = (U * BI) >> 3;
        const int tile_rows_all = U * BI;
        int mrow[RPT];                                   // tile row (first of the octet, MN)
        int mkl[RPT];                                    // k within the stage
        uint32_t soff[RPT];
        uint32_t hvalid = 0;                             // bit 2j+h: half h of row j holds real rows
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            if constexpr (!MN) {
                const int m = (t >> 3) + (CONV_THREADS / 8) * j;
                const bool v = m < tile_rows_all && (m % BI) < rows;
                mrow[j] = m < tile_rows_all ? m : -1;
                mkl[j] = 8 * ko;
                soff[j] = (uint32_t)((m >> 3) * 1024 + (m & 7) * 128 + (((ko ^ (m & 7)) & 7) << 4));
                if (v) hvalid |= 3u << (2 * j);
            } else {
                const int f = t + CONV_THREADS * j;
                const int mo = nmo > 0 ? f % nmo : 0, kl = nmo > 0 ? f / nmo : TC_BK;
                const int m = 8 * mo;
                const bool inside = nmo > 0 && kl < TC_BK;
                mrow[j] = inside ? m : -1;
                mkl[j] = kl;
                soff[j] = inside ? mnmajor_off(m, kl) : 0u;
                if (inside && (m % BI) < rows) hvalid |= 1u << (2 * j);
                if (inside && (m % BI) + 4 < rows) hvalid |= 2u << (2 * j);
            }
        }
        // TMA staging layouts (filled by the producer warp):
        //   K-major, contiguous runs: rows of 64 floats; thread reads row (t>>4) + 16 j,
        //             quad t&15;
        //   K-major, other runs: eight planes (one per k-octet) of 128 rows x 8 floats; the
        //             warp w reads plane w, rows (lane>>1) + 16 j, half lane&1 (4 floats);
        //   MN-major: per packed run u, a (64 k) x (BI i) box; float4 f_j = t + 256 j is the
        //             i-quad f % nq at k = f / nq (nq = U*BI/4).
        uint32_t trd[8], tst[8];
        uint32_t tvalid = 0;
        if constexpr (TMA) {
            const int nq = (U * BI) >> 2;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if constexpr (!MN) {
                    if (tp.kwide) {                      // rows of 64 floats: row (t>>4) + 16 j, quad t&15
                        const int r = (t >> 4) + 16 * j, kq = t & 15;
                        trd[j] = (uint32_t)(r * TC_BK * 4 + kq * 16);
                        tst[j] = kmajor_off(r, 4 * kq);
                        if (r < tile_rows_all) tvalid |= 1u << j;
                    } else {
                        const int r = (lane >> 1) + 16 * j, h = lane & 1;
                        trd[j] = (uint32_t)(warp * TC_M * 32 + r * 32 + h * 16);
                        tst[j] = kmajor_off(r, 8 * warp + 4 * h);
                        if (r < tile_rows_all) tvalid |= 1u << j;
                    }
                } else {
                    const int f = t + CONV_THREADS * j;
                    const int mq = nq > 0 ? f % nq : 0, kl = nq > 0 ? f / nq : TC_BK;
                    const int m = 4 * mq, u = m / BI, il = m % BI;
                    trd[j] = (uint32_t)((u * BI * TC_BK + kl * BI + il) * 4);
                    tst[j] = kl < TC_BK ? mnmajor_off(m, kl) : 0u;
                    if (nq > 0 && kl < TC_BK) tvalid |= 1u << j;
                }
            }
        }
        // staging ring: thread-private 16-byte slots, P stages deep
        const uint32_t stg = dsm_s + (uint32_t)tp.stg_off + (uint32_t)(t * 16);
        // load tracker: next stage to issue (padded index ld_k; run-group ld_qg; offset ld_d0)
        int64_t ld_k = kb, ld_qg = kb / rad0p, ld_d0 = kb % rad0p;
        int64_t xl = 0, xr = 0;                          // non-linear runs (U == 1): (l, r) of the octet
        const float* rbase[RPT];                         // row base pointers (see set_bases)
        uint32_t rmask = 0;                              // bit 2j+h: load allowed for this run-group
        int64_t rbase_qg = -1;
        if constexpr (!MN) {
            if (!tp.linear) {
                const int64_t k0 = ld_qg * rad0 + ld_d0 + 8 * ko;
                xl = k0 % L;
                xr = k0 / L;
            }
        }
        // linear runs: rbase = address of (row, run q, d0 = 0) plus the thread's k offset;
        // non-linear: rbase = address of the row at (l, r) = (0, 0)
        auto set_bases = [&]() {
            rmask = 0;
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                rbase[j] = p.X;
                if (mrow[j] < 0) continue;
                const int u = mrow[j] / BI, il = mrow[j] % BI;
                if (!tp.linear) {
                    rbase[j] = p.X + L * (i0 + il);
                    rmask |= hvalid & (3u << (2 * j));
                    continue;
                }
                const int64_t q = ld_qg * U + u;
                if (q >= nruns) continue;
                const int64_t k0 = q * rad0;             // first real contraction index of run q
                if constexpr (MN) rbase[j] = p.X + (i0 + il) + I * (k0 + mkl[j]);
                else rbase[j] = p.X + (k0 % L) + L * I * (k0 / L) + L * (i0 + il) + 8 * ko;
                rmask |= hvalid & (3u << (2 * j));
            }
            rbase_qg = ld_qg;
        };
        auto issue = [&](int slot) {
            if (rbase_qg != ld_qg && (tp.linear || rbase_qg < 0)) set_bases();
            // values of the stage that exist: k < lim (run end and split end)
            int64_t lim64 = rad0 - ld_d0;
            if (ke - ld_k < lim64) lim64 = ke - ld_k;
            const int lim = lim64 > TC_BK ? TC_BK : (int)lim64;
            int64_t common0, common1;                    // offsets of the two halves
            if constexpr (MN) {
                common0 = I * ld_d0;
                common1 = common0 + 4;
            } else if (true) {
                if (tp.linear) {
                    common0 = ld_d0;
                    common1 = ld_d0 + 4;
                } else {
                    common0 = xl + L * I * xr;
                    common1 = (xl + 4 < L) ? common0 + 4 : (xl + 4 - L) + L * I * (xr + 1);
                }
            }
            const uint32_t sbase = stg + (uint32_t)(slot * 2 * RPT * CONV_THREADS * 16);
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const int kl0 = mkl[j], kl1 = MN ? mkl[j] : mkl[j] + 4;
                const bool v0 = ((rmask >> (2 * j)) & 1u) && kl0 < lim;
                const bool v1 = ((rmask >> (2 * j + 1)) & 1u) && kl1 < lim;
                const float* s0 = v0 ? rbase[j] + common0 : p.X;
                const float* s1 = v1 ? rbase[j] + common1 : p.X;
                const uint32_t d0 = sbase + (uint32_t)((2 * j) * CONV_THREADS * 16);
                const uint32_t d1 = d0 + (uint32_t)(CONV_THREADS * 16);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d0), "l"(s0), "r"(v0 ? 16 : 0) : "memory");
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d1), "l"(s1), "r"(v1 ? 16 : 0) : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            // advance to the next stage (skipping the padding at the end of a run)
            if constexpr (!MN) {
                if (!tp.linear) {
                    const int64_t delta = (ld_d0 + TC_BK == rad0p) ? (rad0 - ld_d0) : TC_BK;
                    xl += delta;
                    while (xl >= L) { xl -= L; ++xr; }
                }
            }
            ld_k += TC_BK;
            ld_d0 += TC_BK;
            if (ld_d0 == rad0p) { ld_d0 = 0; ++ld_qg; }
        };

        // production tracker (stage index within its run, run-group)
        int pr_sir = (int)((kb % rad0p) / TC_BK);
        int64_t pr_qg = kb / rad0p;

        auto produce = [&](int s) -> bool {
            const int slot = s % ST;
            const int pslot = s % tp.P;
            float4 v[2 * RPT];
            if constexpr (TMA) {
                // the producer's boxes for stage s have landed
                if (!mbar_wait(smem_u32(&xfull_bar[pslot]), (uint32_t)((s / tp.P) & 1), &abort_flag, tp.wait_ns)) {
                    abort_flag = 1;
                    set_status(p.status, MTK_ETIMEOUT);
                    return false;
                }
                const uint32_t sbase = dsm_s + (uint32_t)tp.stg_off + (uint32_t)(pslot * 2 * RPT * CONV_THREADS * 16);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    v[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if ((tvalid >> e) & 1u)
                        asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                                     : "=f"(v[e].x), "=f"(v[e].y), "=f"(v[e].z), "=f"(v[e].w)
                                     : "r"(sbase + trd[e]));
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&xempty_bar[pslot]));
            } else {
                // the thread's own copies of stage s are complete after this wait (P groups
                // are always committed ahead of the stage being read)
                switch (tp.P) {
                    case 2: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
                    case 3: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
                    default: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
                }
                const uint32_t sbase = stg + (uint32_t)(pslot * 2 * RPT * CONV_THREADS * 16);
#pragma unroll
                for (int e = 0; e < 2 * RPT; ++e) {
                    const uint32_t a = sbase + (uint32_t)(e * CONV_THREADS * 16);
                    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                                 : "=f"(v[e].x), "=f"(v[e].y), "=f"(v[e].z), "=f"(v[e].w)
                                 : "r"(a));
                }
            }
            if (s >= ST) {
                if (!mbar_wait(smem_u32(&empty_bar[slot]), (uint32_t)(((s / ST) - 1) & 1), &abort_flag, tp.wait_ns)) {
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
                *reinterpret_cast<volatile int*>(&b_issued) = s + 1;
            }
            if constexpr (TMA) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if (!((tvalid >> e) & 1u)) continue;
                    uint2 pcs[PX];
                    split4<PX>(v[e], pcs);
#pragma unroll
                    for (int q = 0; q < PX; ++q) *reinterpret_cast<uint2*>(st + q * PIECE_BYTES + tst[e]) = pcs[q];
                }
            } else {
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    if (mrow[j] < 0) continue;
                    uint2 lo[PX], hi[PX];
                    split4<PX>(v[2 * j], lo);
                    split4<PX>(v[2 * j + 1], hi);
#pragma unroll
                    for (int q = 0; q < PX; ++q)
                        *reinterpret_cast<uint4*>(st + q * PIECE_BYTES + soff[j]) =
                            make_uint4(lo[q].x, lo[q].y, hi[q].x, hi[q].y);
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&full_bar[slot]));
            if constexpr (!TMA) {
                // the staging slot is free again (its values were consumed above)
                if (s + tp.P < nst) issue(pslot);
                else asm volatile("cp.async.commit_group;" ::: "memory");
            }
            return true;
        };

        // accumulator drain state: this thread's tile row (its TMEM lane), its run offset,
        // and its 16-column chunks cc = 16 * (quarter + QW * m) of the CP columns
        const int sub = warp & 3, quarter = warp >> 2;
        const int myrow = sub * 32 + lane;
        const int myu = myrow / BI, myil = myrow % BI;
        const bool myvalid = myu < U && myil < rows;
        float acc[16 * NCH];
        float qc[16 * NCH];
#pragma unroll
        for (int e = 0; e < 16 * NCH; ++e) { acc[e] = 0.0f; qc[e] = 1.0f; }
        int64_t q_cached = -1;
        auto drain = [&](int g, int64_t qg) -> bool {
            const int b = g & 1;
            if (!mbar_wait(smem_u32(&accf_bar[b]), (uint32_t)((g >> 1) & 1), &abort_flag, tp.wait_ns)) {
                abort_flag = 1;
                set_status(p.status, MTK_ETIMEOUT);
                return false;
            }
            tc_fence_after();
            const int64_t q = qg * U + myu;
            const bool live = myvalid && q < nruns;
            const bool newq = tp.ntail > 0 && q != q_cached && live;
#pragma unroll
            for (int m = 0; m < NCH; ++m) {
                const int cc = 16 * (quarter + QW * m);
                if (cc >= CP) continue;                  // warp-uniform
                if (newq) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int c = cc + j;
                        qc[16 * m + j] = (c < C) ? tail_product(tp, q, c, C) : 0.0f;
                    }
                }
                float v0[16], v1[16], v2[16];
                const uint32_t ta = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(b * N + cc);
                tmem_ld16(ta, v0);
                tmem_ld16(ta + (uint32_t)CP, v1);
                tmem_ld16(ta + (uint32_t)(2 * CP), v2);
                tmem_ld_wait();
                if (live) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        acc[16 * m + j] = fmaf((v0[j] + v1[j]) + v2[j], qc[16 * m + j], acc[16 * m + j]);
                }
            }
            if (newq) q_cached = q;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce_bar[b]));
            return true;
        };

        int g = 0;
        bool pending = false, ok = true;
        int pend_g = 0;
        int64_t pend_qg = 0;
        if constexpr (!TMA) {
            for (int sl = 0; sl < tp.P; ++sl) {
                if (sl < nst) issue(sl);
                else asm volatile("cp.async.commit_group;" ::: "memory");
            }
        }
        int arrived = 0;                                 // stages this warp has arrived on
        for (int s = 0; s < nst; ++s) {
            if (!produce(s)) { ok = false; break; }
            ++arrived;
            const bool last = ((pr_sir + 1) % GROUP == 0) || (pr_sir + 1 == spr) || (s == nst - 1);
            const int64_t qg_s = pr_qg;
            if (++pr_sir == spr) { pr_sir = 0; ++pr_qg; }
            if (last) {
                if (pending && !drain(pend_g, pend_qg)) { ok = false; break; }
                pend_g = g;
                pend_qg = qg_s;
                pending = true;
                ++g;
            }
        }
        if (ok && pending) ok = drain(pend_g, pend_qg);
        asm volatile("cp.async.wait_all;" ::: "memory");
        // Abort: the B-image copies already issued must land before the CTA leaves.  Each
        // completes a full barrier that also counts one arrival per converter warp, so every
        // warp first arrives for the issued stages it has not reached (at most ST of them,
        // each the current phase of its slot: stage s was issued only after stage s - ST had
        // been consumed), then the issuing thread waits for those phases.
        asm volatile("bar.sync 1, %0;" ::"r"(CONV_THREADS) : "memory");
        if (*reinterpret_cast<volatile int*>(&abort_flag)) {
            const int nb = *reinterpret_cast<volatile int*>(&b_issued);
            if (lane == 0)
                for (int s = arrived; s < nb; ++s) mbar_arrive(smem_u32(&full_bar[s % ST]));
            if (warp == 0 && lane == 0) {
                for (int s = nb > ST ? nb - ST : 0; s < nb; ++s) {
                    volatile int never = 0;
                    (void)mbar_wait(smem_u32(&full_bar[s % ST]), (uint32_t)((s / ST) & 1), &never, kWaitNs);
                }
            }
        }

        // ------------------------------------------------------------ epilogue
        // packed run offsets become separate partial slabs: slab = sp * U + u
        if (ok && myvalid) {
            const int64_t i = i0 + myil;
            const int64_t slab = (int64_t)sp * U + myu;
#pragma unroll
            for (int m = 0; m < NCH; ++m) {
                const int cc = 16 * (quarter + QW * m);
                if (cc >= CP) continue;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = cc + j;
                    if (c < C) {
                        if (tp.nslabs == 1) p.out[i * p.out_si + c * p.out_sc] = acc[16 * m + j];
                        else p.part[(slab * I + i) * C + c] = acc[16 * m + j];
                    }
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

template <int PX, bool MN, bool TMA>
cudaError_t launch_variant(const TcParams& tp, const CUtensorMap& map, dim3 grid, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(contract_tc_kernel<PX, MN, TMA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    contract_tc_kernel<PX, MN, TMA><<<grid, NTHREADS, smem, s>>>(tp, map);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

// Launch of one kernel variant; instantiated explicitly in the translation unit of its
// (PX, MN) pair and declared extern where it is called.
template <int PX, bool MN, bool TMA>
cudaError_t tc_launch(const tcd::TcParams& tp, const CUtensorMap& map, dim3 grid, size_t smem, cudaStream_t s) {
    return launch_variant<PX, MN, TMA>(tp, map, grid, smem, s);
}

}  // namespace mtk
