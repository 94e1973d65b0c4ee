// contract_split.cu -- the MTTKRP contraction on a tensor stored as two BF16 planes.
//
// CP-ALS (Section 2.2) runs an MTTKRP for every mode of every sweep on the same
// tensor X.  Here X is split once into x = hi + lo, hi = bf16_rn(x), lo =
// bf16_rn(x - hi) (the two-piece split of Henry, Tang and Heinecke, ARITH 2019),
// and the two pieces are kept as two planes in the natural linearization (Section
// 2.1).  The planes take exactly the bytes of the FP32 tensor, so every MTTKRP still
// reads 4 bytes per entry, but the tensor-core operand is then a plain tile load:
// TMA brings each 64-k tile of both planes into shared memory in the 128-byte-swizzled
// layout that tcgen05.mma reads, and no thread touches tensor entries at all.
//
// The contraction is the one of contract_tc.cu (Algorithm 3's block structure on the
// 3-way view of Fig. 2):
//     M(i, c) = sum_q Q(q, c) * sum_h X3(h + H q, i) * Hd(h, c)
// where the head Hd is the KRP of the first factors of the mode (H rows, split into
// three BF16 pieces stacked along N = 3 * CP in an image of the B operand, one slice per
// 64-k stage) and Q(q, c) is the product of the remaining factors' rows, applied when
// the accumulator is drained from TMEM.  Drains happen at every run boundary and at
// least every two stages, which bounds each tensor-core accumulation chain.
//
// Tensor operand: K-major (h along the contiguous mode, modes n > 0) or MN-major (i
// contiguous, mode 0).  Rows of the 128-row MMA tile: one tile of BI <= 128 rows of i,
// or, for I_n <= 64, U runs of the head packed one above the other (each packed run is
// a separate partial slab).
//
// Warp roles (96 + 128 MT threads, one CTA per SM, MT = 128-row MMA tiles per CTA):
// warp 0 issues the tensor TMA loads into the A ring, warp 1 owns TMEM and one of its
// lanes issues the MMAs, warp 2 issues the image slices into the B ring, and 4 warps per
// MMA tile drain the accumulators (one TMEM lane, i.e. one row of M, per thread) and
// write the result or a partial slab.  The work is a list of units (a tile of rows and a
// slab of its stages); a CTA runs one unit, or, when the view has more units than SMs,
// several back to back, each role carrying its ring slots, phases and accumulator
// buffers over from one unit to the next.  Every mbarrier wait is bounded (1 s of
// %globaltimer by default, or the caller's limit); on expiry the kernel sets MTK_ETIMEOUT
// and every role stops.  The producers then wait for their last copies to land and the
// MMA issuer for its last MMAs (waits of 1 s that an abort does not shorten) before the
// CTA frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <string.h>

#include "mtk_internal.cuh"
#include "tc_ptx.cuh"

namespace mtk {
namespace {

using namespace tc;

constexpr int PS_BK = 64;                    // k per stage
constexpr int PS_M = 128;                    // MMA M
#ifndef MTK_PS_GROUP
#define MTK_PS_GROUP 2
#endif
#ifndef MTK_PS_LO_SEP
#define MTK_PS_LO_SEP 1
#endif
// head: the first prefix with at least 64 rows whose padding is at most 1/MTK_PS_HEAD_PAD
// of its padded rows; 1/MTK_PS_HEAD_PAD_NEAR when the K-major tile packs several runs and
// the prefix keeps consecutive runs in one box (see planes_plan)
#ifndef MTK_PS_HEAD_PAD
#define MTK_PS_HEAD_PAD 32
#endif
// K-major tiling when the fewest i-tiles are under 3/4 full: 1 the fewest stages (measured:
// 165^4 mode 1 from 0.70 to 0.81 of the roofline, the other modes unchanged or better);
// 0 the most rows per stage (ties: fewer tiles)
#ifndef MTK_PS_TILE_MODEL
#define MTK_PS_TILE_MODEL 1
#endif
#ifndef MTK_PS_HEAD_PAD_NEAR
#define MTK_PS_HEAD_PAD_NEAR 4
#endif
constexpr int PS_GROUP = MTK_PS_GROUP;       // stages per accumulation chain (at most)
// one MMA tile: the lo plane accumulates into accumulator columns of its own (1) or into
// the hi plane's first two pieces (0)
constexpr bool PS_LO_SEP = MTK_PS_LO_SEP != 0;
constexpr int PS_MAX_A = 8;
constexpr int PS_MAX_B = 6;
constexpr int PS_MAX_BUF = 4;
constexpr int PS_MAX_U = 32;                 // packed run groups per tile (256 rows / 8)
constexpr int PS_TILE = PS_M * 128;          // one plane of a 128 x 64 BF16 tile (16 KB)
constexpr int PS_MN_ATOM = 64 * 128;         // MN-major: 64 k rows x 64 i (8 KB)
constexpr unsigned long long kPsWaitNs = 1000000000ull;
// smallest B ring of a one-MMA-tile CTA (the A ring takes the rest of the budget)
#ifndef MTK_PS_SB_MIN1
#define MTK_PS_SB_MIN1 3
#endif

// L2 eviction hints: tensor tiles are read once (evict first), the head image is read by
// every stage of every CTA (evict last), so that the streaming tensor does not push the
// image out of L2.
#ifndef MTK_PS_L2_HINTS
#define MTK_PS_L2_HINTS 1
#endif
// L2 promotion of the tensor-map loads (0 none, 1 64 B, 2 128 B, 3 256 B), per operand
// orientation.  MN-major boxes read 128-byte pieces of rows I_n apart; promoting them to
// 256 B fetched sectors no stage used: 128 B took the 200x200x300x40 right partial from
// 335 to 311 us and mode 0 from 359 to 326 us.
#ifndef MTK_PS_KM_PROMO
#define MTK_PS_KM_PROMO 3
#endif
#ifndef MTK_PS_MN_PROMO
#define MTK_PS_MN_PROMO 2
#endif
CUtensorMapL2promotion promo(int code) {
    switch (code) {
        case 0: return CU_TENSOR_MAP_L2_PROMOTION_NONE;
        case 1: return CU_TENSOR_MAP_L2_PROMOTION_L2_64B;
        case 2: return CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
        default: return CU_TENSOR_MAP_L2_PROMOTION_L2_256B;
    }
}

struct PsParams {
    int64_t I;              // output rows (I_n)
    int64_t nruns;          // runs of the head along the contraction
    int64_t Lq;             // K-major: runs per r (I^L / H)
    int64_t gpr;            // box mode 2 with U not dividing Lq: packed groups per r (ceil(Lq / U));
                            // group sr holds runs lq = (sr mod gpr) U + u < Lq of r = sr / gpr.
                            // 0: group sr holds runs q = sr U + u
    int64_t stot;           // stages of one tile: (groups of runs) * spr
    int64_t H;              // head rows (the last chunk of a run holds H - 64 (spr - 1) of them)
    int spr;                // stages per run (H padded to a multiple of 64, / 64)
    int U, BI, MT;          // packed runs, rows per run group (tile rows), 128-row MMA tiles
    int box_mode;           // packed runs (U > 1): 0 one TMA box per run group; 1 one box for all U
                            // groups, runs along r (rows grouped by run); 2 one box, runs along lq
                            // (rows interleaved: tile row m = U i + u)
    int C, CP, N;           // N = 3 CP columns of the hi-plane accumulator
    int lo_sep;             // the lo plane accumulates into its own 2 CP columns (one MMA tile)
    int acc_cols;           // TMEM columns per accumulator buffer
    int sa, sb, nbuf, tmem_cols;
    uint32_t idesc_hi, idesc_lo;
    int a_stage, plane_bytes, b_bytes, b_stage, b_base;
    int ntiles, s_full, s_last, nslab;
    int sk;                 // stream-K: CTA c takes stages [c tot / G, (c + 1) tot / G) of the flattened
    int64_t sk_tot;         // (tile, stage) space (tot = ntiles * stot, G = gridDim.x); a tile split
                            // between CTAs leaves one partial slab per piece
    const uint8_t* bimg;
    const float* qtab;      // Q(q, c) as [nruns][CP], or null (products formed in the drain)
    int ntail;
    const float* tail[MTK_MAXN];
    int64_t tail_rad[MTK_MAXN];
    float* out;
    int64_t out_si, out_sc;
    int64_t opad, oreal;    // output rows: row j of the view is row (j mod opad) + oreal (j / opad) of
                            // the output, dropped when j mod opad >= oreal (planes with mode 0
                            // padded); opad = 0: row j
    float* part;            // partial slabs when nslab > 1: [slab][I][C], or [slab][C][I] (part_cm)
    int part_cm;            // slabs in the output's column-major layout (out_si == 1)
    uint32_t* status;
    unsigned long long wait_ns;   // limit of every wait that an abort can end
    int stall;              // test hook: the MMA issuer first waits on a barrier that nothing completes
};

// A unit of work: one tile of rows and one slab (a contiguous range of its stages).
// Units are numbered tile-major: the first ntiles - 1 tiles have s_full slabs each, the
// last one s_last.  A CTA takes units blockIdx.x, blockIdx.x + gridDim.x, ...; the grid
// is at most one CTA per SM, so a view with more units than that runs them back to back
// in each CTA with the rings, barriers and TMEM kept from one unit to the next.
struct PsUnit {
    int tile, sp, nst;
    int64_t t0, i0;         // first stage; first row of the tile
    bool direct;            // the unit is the whole tile: the result goes straight to the output
};

__device__ __forceinline__ int ps_units(const PsParams& p) { return (p.ntiles - 1) * p.s_full + p.s_last; }

// stream-K: the CTA that holds flattened stage s
__host__ __device__ __forceinline__ int64_t sk_cta(int64_t s, int64_t tot, int64_t G) { return ((s + 1) * G - 1) / tot; }

// The units of this CTA, in order: classic, units blockIdx.x, blockIdx.x + gridDim.x, ...;
// stream-K, the tiles its stage range touches.
struct PsIter {
    int64_t s0, s1;
    int tfirst, nk;
};
__device__ __forceinline__ PsIter ps_iter(const PsParams& p) {
    PsIter it;
    it.s0 = it.s1 = 0;
    it.tfirst = 0;
    const int64_t c = blockIdx.x, G = gridDim.x;
    if (!p.sk) {
        const int nu = ps_units(p);
        it.nk = c < nu ? (int)((nu - c + G - 1) / G) : 0;
    } else {
        it.s0 = c * p.sk_tot / G;
        it.s1 = (c + 1) * p.sk_tot / G;
        it.tfirst = (int)(it.s0 / p.stot);
        it.nk = it.s1 > it.s0 ? (int)((it.s1 - 1) / p.stot) - it.tfirst + 1 : 0;
    }
    return it;
}

__device__ __forceinline__ PsUnit ps_unit(const PsParams& p, int b) {
    PsUnit u;
    int S_t;
    if (b < (p.ntiles - 1) * p.s_full) {
        u.tile = b / p.s_full;
        u.sp = b - u.tile * p.s_full;
        S_t = p.s_full;
    } else {
        u.tile = p.ntiles - 1;
        u.sp = b - (p.ntiles - 1) * p.s_full;
        S_t = p.s_last;
    }
    u.t0 = p.stot * u.sp / S_t;
    u.nst = (int)(p.stot * (u.sp + 1) / S_t - u.t0);
    u.i0 = (int64_t)u.tile * p.BI;
    u.direct = p.nslab == 1;
    return u;
}

__device__ __forceinline__ PsUnit ps_unit_k(const PsParams& p, const PsIter& it, int k) {
    if (!p.sk) return ps_unit(p, (int)blockIdx.x + k * (int)gridDim.x);
    PsUnit u;
    u.tile = it.tfirst + k;
    const int64_t ts = (int64_t)u.tile * p.stot;
    const int64_t a = it.s0 > ts ? it.s0 : ts;
    const int64_t b = it.s1 < ts + p.stot ? it.s1 : ts + p.stot;
    u.t0 = a - ts;
    u.nst = (int)(b - a);
    u.direct = (a == ts && b == ts + p.stot) && p.U == 1;   // packed runs always leave slabs
    u.sp = (int)((int64_t)blockIdx.x - sk_cta(ts, p.sk_tot, gridDim.x));      // piece of the tile
    u.i0 = (int64_t)u.tile * p.BI;
    return u;
}

template <int NCH, bool MN, int MT>
__global__ void __launch_bounds__(96 + 128 * MT, 1)
contract_planes_kernel(const __grid_constant__ PsParams p, const __grid_constant__ CUtensorMap xmap) {
    extern __shared__ uint8_t dsm_raw[];
    __shared__ __align__(8) uint64_t afull[PS_MAX_A], aempty[PS_MAX_A];
    __shared__ __align__(8) uint64_t bfull[PS_MAX_B], bempty[PS_MAX_B];
    __shared__ __align__(8) uint64_t accf_bar[PS_MAX_BUF], acce_bar[PS_MAX_BUF];
    __shared__ __align__(8) uint64_t fin_bar, stall_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* dsm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t dsm_s = smem_u32(dsm);
    const int SA = p.sa, SB = p.sb, NB = p.nbuf;

    const PsIter pit = ps_iter(p);
    const int64_t I = p.I;
    const int U = p.U, BI = p.BI, spr = p.spr;
    const int64_t nruns = p.nruns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SA; ++s) {
            mbar_init(smem_u32(&afull[s]), 1);
            mbar_init(smem_u32(&aempty[s]), 1);
        }
        for (int s = 0; s < SB; ++s) {
            mbar_init(smem_u32(&bfull[s]), 1);
            mbar_init(smem_u32(&bempty[s]), 1);
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), 4 * MT);
        }
        mbar_init(smem_u32(&fin_bar), 1);
        mbar_init(smem_u32(&stall_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(p.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ tensor (A) producer
        if (lane == 0) {
            int issued = 0;                                  // stages issued by this CTA
            bool ok = true;
            // position of the next stage: super-run sr (the group of U packed runs that a
            // stage carries), chunk j of the head (no divisions
            // in the loop); per packed run g present, its (lq, r) coordinates
            int64_t sr = 0;
            int j = 0;
            int ng = 0;
            // K-major: group g of the super-run loads rows i0 + m of run q = (lq, r) as rows
            // y = i0 + m + I_n r of the (I^L, I_n I^R) row view, from column x = H lq + 64 j
            // (a multiple of 8: the planes keep every row 16-byte aligned)
            int gx[PS_MAX_U], gy[PS_MAX_U];
            int64_t i0 = 0;
            auto set_groups = [&]() {
                ng = 0;
                while (ng < U && sr * U + ng < nruns) ++ng;
                if (!MN) {
                    const uint32_t Lq = (uint32_t)p.Lq;
                    for (int g = 0; g < ng; ++g) {
                        const uint32_t q = (uint32_t)(sr * U + g);
                        const uint32_t r = q / Lq;
                        gx[g] = (int)(p.H * (int64_t)(q - r * Lq));
                        gy[g] = (int)(i0 + p.I * (int64_t)r);
                    }
                }
            };
            int slot = 0;
            uint32_t ph = 1;                                 // parity of the empty phase to wait for
            const uint64_t pol_a = MTK_PS_L2_HINTS ? policy_evict_first() : policy_evict_normal();
            for (int uk = 0; ok && uk < pit.nk; ++uk) {
                const PsUnit w = ps_unit_k(p, pit, uk);
                i0 = w.i0;
                sr = w.t0 / spr;
                j = (int)(w.t0 - sr * spr);
                set_groups();
                int nbox = 0;                                    // MN-major, U == 1: 64-row boxes present
                if (MN && U == 1)
                    while (nbox < 2 * MT && i0 + 64 * nbox < I) ++nbox;
                for (int s = 0; s < w.nst; ++s) {
                    if (issued >= SA && !mbar_wait(smem_u32(&aempty[slot]), ph, &abort_flag, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = dsm_s + (uint32_t)(slot * p.a_stage);
                    const uint32_t fb = smem_u32(&afull[slot]);
                    uint32_t bytes;
                    if (MN) bytes = (uint32_t)(2 * (U == 1 ? nbox : (p.box_mode ? U : ng)) * PS_MN_ATOM);
                    else bytes = (uint32_t)(2 * (p.box_mode ? U : ng) * BI * 128);
                    mbar_arrive_expect_tx(fb, bytes);
                    if (p.box_mode) {
                        // one box holds every packed run of the super-run (a run beyond the
                        // last reads the zero fill)
                        const int q0 = (int)(sr * U);
#pragma unroll
                        for (int pl = 0; pl < 2; ++pl) {
                            const uint32_t dst = st + (uint32_t)(pl * p.plane_bytes);
                            if (MN) {
                                tma_load_4d_hint(dst, &xmap, 0, 64 * j, q0, pl, fb, pol_a);
                            } else if (p.box_mode == 1) {
                                // one run per row (q = r)
                                tma_load_4d_hint(dst, &xmap, 64 * j, (int)i0, q0, pl, fb, pol_a);
                            } else if (p.gpr) {
                                // row-local groups: runs beyond the row's last read the zero fill
                                const int r = (int)(sr / p.gpr);
                                const int lq0 = (int)(sr - (int64_t)r * p.gpr) * U;
                                tma_load_5d_hint(dst, &xmap, 64 * j, lq0, (int)i0, r, pl, fb, pol_a);
                            } else {
                                const int r = q0 / (int)p.Lq;
                                tma_load_5d_hint(dst, &xmap, 64 * j, q0 - r * (int)p.Lq, (int)i0, r, pl, fb, pol_a);
                            }
                        }
                    }
                    for (int g = 0; !p.box_mode && g < ng; ++g) {
#pragma unroll
                        for (int pl = 0; pl < 2; ++pl) {
                            const uint32_t dst = st + (uint32_t)(pl * p.plane_bytes);
                            if (MN) {
                                const int q = (int)(sr * U + g);
                                if (U == 1) {
                                    for (int a = 0; a < nbox; ++a)
                                        tma_load_4d_hint(dst + (uint32_t)(a * PS_MN_ATOM), &xmap, (int)(i0 + 64 * a),
                                                         64 * j, q, pl, fb, pol_a);
                                } else {
                                    tma_load_4d_hint(dst + (uint32_t)(g * PS_MN_ATOM), &xmap, 0, 64 * j, q, pl, fb, pol_a);
                                }
                            } else {
                                tma_load_3d_hint(dst + (uint32_t)(g * BI * 128), &xmap, gx[g] + 64 * j, gy[g], pl, fb,
                                                 pol_a);
                            }
                        }
                    }
                    ++issued;
                    if (++slot == SA) {
                        slot = 0;
                        ph ^= 1u;
                    }
                    if (++j == spr) {
                        j = 0;
                        ++sr;
                        set_groups();
                    }
                }
            }
            if (!ok) {
                abort_flag = 1;
                set_status(p.status, MTK_ETIMEOUT);
            }
            // let the copies already issued land before the CTA leaves (also when another
            // role aborted after this one had issued its last stage; consumed phases return
            // at once)
            for (int s = issued > SA ? issued - SA : 0; s < issued; ++s) {
                volatile int never = 0;
                (void)mbar_wait(smem_u32(&afull[s % SA]), (uint32_t)((s / SA) & 1), &never, kPsWaitNs);
            }
        }
        __syncwarp();
    } else if (warp == 2) {
        // ------------------------------------------------------------ KRP image (B) producer
        if (lane == 0) {
            int issued = 0;                                  // slices issued by this CTA
            bool ok = true;
            int slot = 0;
            uint32_t ph = 1;
            const uint64_t pol_b = MTK_PS_L2_HINTS ? policy_evict_last() : policy_evict_normal();
            for (int uk = 0; ok && uk < pit.nk; ++uk) {
                const PsUnit w = ps_unit_k(p, pit, uk);
                int j = (int)(w.t0 % spr);
                for (int s = 0; s < w.nst; ++s) {
                    if (issued >= SB && !mbar_wait(smem_u32(&bempty[slot]), ph, &abort_flag, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&bfull[slot]);
                    mbar_arrive_expect_tx(fb, (uint32_t)p.b_bytes);
                    bulk_copy_g2s_hint(dsm_s + (uint32_t)(p.b_base + slot * p.b_stage),
                                       p.bimg + (int64_t)j * p.b_bytes, (uint32_t)p.b_bytes, fb, pol_b);
                    ++issued;
                    if (++slot == SB) {
                        slot = 0;
                        ph ^= 1u;
                    }
                    if (++j == spr) j = 0;
                }
            }
            if (!ok) {
                abort_flag = 1;
                set_status(p.status, MTK_ETIMEOUT);
            }
            for (int s = issued > SB ? issued - SB : 0; s < issued; ++s) {
                volatile int never = 0;
                (void)mbar_wait(smem_u32(&bfull[s % SB]), (uint32_t)((s / SB) & 1), &never, kPsWaitNs);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            // Descriptors are formed once and advanced by constant 16-byte-unit offsets; ring
            // slots and barrier phases are counters (no divisions in the loop): an MMA then
            // issues at its math rate.
            constexpr uint32_t a_lbo = MN ? (uint32_t)PS_MN_ATOM : 16u;
            constexpr uint32_t a_k16 = MN ? (2048u >> 4) : (32u >> 4);   // one K = 16 step
            const uint64_t adesc0 = make_desc(dsm_s, a_lbo, 1024u);
            const uint64_t bdesc0 = make_desc(dsm_s + (uint32_t)p.b_base, 16u, 1024u);
            const uint64_t plane16 = (uint64_t)(p.plane_bytes >> 4);
            const uint64_t a_st16 = (uint64_t)(p.a_stage >> 4), b_st16 = (uint64_t)(p.b_stage >> 4);
            const uint32_t idh = p.idesc_hi, idl = p.idesc_lo;
            const uint32_t ncol = (uint32_t)p.N;
            // k-steps of the last chunk of a run that hold head rows (the rest is padding)
            const int64_t tail_rows = p.H - (int64_t)PS_BK * (spr - 1);
            const int kk_last = (int)((tail_rows + 15) / 16);
            int g = 0, gs = 0;                               // accumulation groups (all units)
            int sa = 0, sb = 0, bi = 0;
            uint32_t pa = 0, pb = 0, pe = 1;
            uint64_t ad = adesc0, bd = bdesc0;
            bool ok = true;
            if (p.stall && !mbar_wait(smem_u32(&stall_bar), 0u, &abort_flag, p.wait_ns)) ok = false;
            uint32_t dcol = tmem;
            for (int uk = 0; ok && uk < pit.nk; ++uk) {
                const PsUnit w = ps_unit_k(p, pit, uk);
                const int nst = w.nst;
                int j = (int)(w.t0 % spr);
                for (int s = 0; s < nst; ++s) {
                    if (!mbar_wait(smem_u32(&afull[sa]), pa, &abort_flag, p.wait_ns) ||
                        !mbar_wait(smem_u32(&bfull[sb]), pb, &abort_flag, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    if (gs == 0) {
                        if (g >= NB && !mbar_wait(smem_u32(&acce_bar[bi]), pe, &abort_flag, p.wait_ns)) {
                            ok = false;
                            break;
                        }
                        dcol = tmem + (uint32_t)(bi * p.acc_cols);
                    }
                    tc_fence_after();
                    const int kk_n = (j == spr - 1) ? kk_last : PS_BK / 16;
                    // hi plane x all three KRP pieces; lo plane x the first two (the dropped
                    // lo * third-piece product is below 2^-24 of |x w|).  One MMA tile: the lo
                    // plane has its own accumulator (columns N .. N + 2 CP).
#pragma unroll
                    for (int kk = 0; kk < PS_BK / 16; ++kk) {
                        if (kk < kk_n) {
                            const uint64_t bk = bd + (uint64_t)(kk * 2);
                            const uint32_t acc = (kk == 0 && gs == 0) ? 0u : 1u;
                            if (MT == 1 && PS_LO_SEP) {
                                const uint64_t a0 = ad + (uint64_t)(kk * a_k16);
                                mma_bf16(dcol, a0, bk, idh, acc);
                                mma_bf16(dcol + ncol, a0 + plane16, bk, idl, acc);
                            } else {
#pragma unroll
                                for (int mt = 0; mt < MT; ++mt) {
                                    const uint64_t a0 = ad + (uint64_t)(kk * a_k16 + mt * (PS_TILE >> 4));
                                    mma_bf16(dcol + (uint32_t)mt * ncol, a0, bk, idh, acc);
                                }
#pragma unroll
                                for (int mt = 0; mt < MT; ++mt) {
                                    const uint64_t a0 = ad + (uint64_t)(kk * a_k16 + mt * (PS_TILE >> 4)) + plane16;
                                    mma_bf16(dcol + (uint32_t)mt * ncol, a0, bk, idl, 1u);
                                }
                            }
                        }
                    }
                    mma_commit(smem_u32(&aempty[sa]));
                    mma_commit(smem_u32(&bempty[sb]));
                    if (++sa == SA) {
                        sa = 0;
                        pa ^= 1u;
                        ad = adesc0;
                    } else {
                        ad += a_st16;
                    }
                    if (++sb == SB) {
                        sb = 0;
                        pb ^= 1u;
                        bd = bdesc0;
                    } else {
                        bd += b_st16;
                    }
                    ++gs;
                    const bool run_end = (++j == spr);
                    if (run_end) j = 0;
                    if (gs == PS_GROUP || run_end || s + 1 == nst) {
                        mma_commit(smem_u32(&accf_bar[bi]));
                        ++g;
                        gs = 0;
                        if (++bi == NB) {                // next round of the buffers: group g
                            bi = 0;                          // waits for drain #(g / NB - 1)
                            pe ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {
                abort_flag = 1;
                set_status(p.status, MTK_ETIMEOUT);
            }
            // every MMA issued by this thread has completed once fin_bar flips
            mma_commit(smem_u32(&fin_bar));
            volatile int never = 0;
            (void)mbar_wait(smem_u32(&fin_bar), 0u, &never, kPsWaitNs);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ drain + epilogue
        const int dw = warp - 3;
        const int sub = warp & 3;                    // TMEM sub-partition of this warp
        const int mt = dw >> 2;                      // MMA tile
        const int row = mt * 128 + sub * 32 + lane;  // row of the CTA tile = TMEM lane of tile mt
        const bool ilv = p.box_mode == 2;
        const int myg = U > 1 ? (ilv ? row % U : row / BI) : 0;
        const int myil = U > 1 ? (ilv ? row / U : row % BI) : row;
        const int C = p.C, CP = p.CP;
        float acc[16 * NCH], qc[16 * NCH];
        int g = 0, gs = 0;
        int db = 0;                                          // accumulator buffer of group g
        uint32_t dph = 0;                                    // and the parity of its next fill
        bool ok = true;
        for (int uk = 0; ok && uk < pit.nk; ++uk) {
            const PsUnit w = ps_unit_k(p, pit, uk);
            const int64_t i0 = w.i0;
            const int nst = w.nst;
            const int64_t rows_here = (I - i0) < BI ? (I - i0) : BI;
            const bool rowvalid = myg < U && myil < rows_here;
#pragma unroll
            for (int e = 0; e < 16 * NCH; ++e) {
                acc[e] = 0.0f;
                qc[e] = e < C ? 1.0f : 0.0f;
            }
            int64_t qcached = -1;
            int64_t sr = w.t0 / spr;                             // super-run of the next stage
            int j = (int)(w.t0 - sr * spr);
            for (int s = 0; s < nst; ++s) {
                const int64_t sr_s = sr;
                ++gs;
                const bool run_end = (++j == spr);
                if (run_end) {
                    j = 0;
                    ++sr;
                }
                if (!(gs == PS_GROUP || run_end || s + 1 == nst)) continue;
                gs = 0;
                const int b = db;
                int64_t q;
                bool qok;
                if (p.gpr) {
                    const int64_t r = sr_s / p.gpr;
                    const int64_t lq = (sr_s - r * p.gpr) * U + myg;
                    q = r * p.Lq + lq;
                    qok = lq < p.Lq;
                } else {
                    q = sr_s * U + myg;
                    qok = q < nruns;
                }
                const bool live = rowvalid && qok;
                if (live && p.ntail > 0 && q != qcached) {
                    // Q(q, c) = prod_z tail_z(digit_z(q), c): one row of the table, or the
                    // product formed here (digits once, then the columns)
                    if (p.qtab) {
                        const float4* qr = reinterpret_cast<const float4*>(p.qtab + q * CP);
#pragma unroll
                        for (int e4 = 0; e4 < 4 * NCH; ++e4) {
                            const float4 v = __ldg(qr + e4);
                            qc[4 * e4] = v.x;
                            qc[4 * e4 + 1] = v.y;
                            qc[4 * e4 + 2] = v.z;
                            qc[4 * e4 + 3] = v.w;
                        }
                    } else {
                        const float* rowp[MTK_MAXN];
                        int64_t rem = q;
                        for (int z = 0; z < p.ntail; ++z) {
                            const int64_t rad = p.tail_rad[z];
                            const int64_t nq = rem / rad;
                            rowp[z] = p.tail[z] + (rem - nq * rad) * C;
                            rem = nq;
                        }
#pragma unroll
                        for (int e = 0; e < 16 * NCH; ++e) qc[e] = e < C ? __ldg(rowp[0] + e) : 0.0f;
                        for (int z = 1; z < p.ntail; ++z) {
#pragma unroll
                            for (int e = 0; e < 16 * NCH; ++e)
                                if (e < C) qc[e] *= __ldg(rowp[z] + e);
                        }
                    }
                    qcached = q;
                }
                if (!mbar_wait(smem_u32(&accf_bar[b]), dph, &abort_flag, p.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ta = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(b * p.acc_cols + mt * p.N);
                if (MT == 1 && PS_LO_SEP) {
                    // hi accumulator (w0, w1, w2 at 0, CP, 2 CP) and lo accumulator (w0, w1 at
                    // N, N + CP); summed smallest first
#pragma unroll
                    for (int m = 0; m < NCH; ++m) {
                        float h0[16], h1[16], h2[16], l0[16], l1[16];
                        tmem_ld16(ta + 16 * m, h0);
                        tmem_ld16(ta + 16 * m + CP, h1);
                        tmem_ld16(ta + 16 * m + 2 * CP, h2);
                        tmem_ld16(ta + 16 * m + p.N, l0);
                        tmem_ld16(ta + 16 * m + p.N + CP, l1);
                        tmem_ld_wait();
                        if (live) {
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) {
                                const int e = 16 * m + jj;
                                const float v = ((h2[jj] + l1[jj]) + (h1[jj] + l0[jj])) + h0[jj];
                                acc[e] = fmaf(v, qc[e], acc[e]);
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < NCH; ++m) {
                        float v0[16], v1[16], v2[16];
                        tmem_ld16(ta + 16 * m, v0);
                        tmem_ld16(ta + 16 * m + CP, v1);
                        tmem_ld16(ta + 16 * m + 2 * CP, v2);
                        tmem_ld_wait();
                        if (live) {
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) {
                                const int e = 16 * m + jj;
                                acc[e] = fmaf((v2[jj] + v1[jj]) + v0[jj], qc[e], acc[e]);
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&acce_bar[b]));
                ++g;
                if (++db == NB) {
                    db = 0;
                    dph ^= 1u;
                }
            }
            if (ok && rowvalid) {
                const int64_t i = i0 + myil;
                if (w.direct) {
                    int64_t io = i;
                    if (p.opad) {
                        const int64_t q = i / p.opad, rr = i - q * p.opad;
                        io = rr < p.oreal ? rr + p.oreal * q : -1;
                    }
                    if (io >= 0) {
#pragma unroll
                        for (int e = 0; e < 16 * NCH; ++e)
                            if (e < C) p.out[io * p.out_si + e * p.out_sc] = acc[e];
                    }
                } else {
                    float* slab = p.part + ((int64_t)w.sp * U + myg) * I * C;
                    if (p.part_cm) {
#pragma unroll
                        for (int e = 0; e < 16 * NCH; ++e)
                            if (e < C) slab[(int64_t)e * I + i] = acc[e];
                    } else {
                        float* dst = slab + i * C;
#pragma unroll
                        for (int e = 0; e < 16 * NCH; ++e)
                            if (e < C) dst[e] = acc[e];
                    }
                }
            }
        }
        if (!ok) {
            abort_flag = 1;
            set_status(p.status, MTK_ETIMEOUT);
        }
        tc_fence_before();
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols));
    }
    // launched after a factorisation it may overlap: complete only after it (a no-op for
    // an ordinary launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---- per-call preparation: the B image of the head and the table of tail scales ----
// Image slice j (one 64-k stage) is the 128-byte-swizzled K-major shared-memory image of
// the N = 3 CP rows n = piece * CP + c, row n holding piece `piece` of Hd(64 j + d, c),
// d = 0..63 (zero outside the head's H rows and for c >= C).  Pieces: w0 = bf16_rn(w),
// w1 = bf16_rn(w - w0), w2 = bf16_rn(w - w0 - w1).  Q(q, c) = prod over the tail
// factors of their rows at the digits of q (first tail factor fastest), 0 for c >= C.
struct PrepArgs {
    int head, C, CP, N;
    const float* fac[MTK_MAXN];
    int64_t frad[MTK_MAXN];
    int64_t f0_rows;        // rows of the first factor that exist (the rest are taken as zero)
    int64_t H, Hp;
    uint8_t* img;
    int ntail;
    const float* tail[MTK_MAXN];
    int64_t tail_rad[MTK_MAXN];
    int64_t nruns;
    float* qtab;
};

__device__ __forceinline__ void split3(float w, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __float2bfloat16_rn(w);
    const float r1 = w - __bfloat162float(a);
    b = __float2bfloat16_rn(r1);
    c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

__global__ void __launch_bounds__(256) planes_prep_kernel(const __grid_constant__ PrepArgs a) {
    const int64_t n_img = a.Hp / 8 * a.CP;                 // octets of the image x columns
    // the table: one item per row q and 4 columns (one 16-byte store), q's digits formed
    // once per item in 32-bit arithmetic (runs and radices below 2^31)
    const int64_t n_q = a.qtab ? a.nruns * (a.CP / 4) : 0;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < n_img + n_q;
         it += (int64_t)gridDim.x * blockDim.x) {
        if (it < n_img) {
            const int c = (int)(it % a.CP);
            const int64_t k0 = it / a.CP * 8;                   // first head row of this octet
            int64_t dig[MTK_MAXN];
            int64_t rem = k0;
            for (int z = 0; z < a.head; ++z) {
                const int64_t nq = rem / a.frad[z];
                dig[z] = rem - nq * a.frad[z];
                rem = nq;
            }
            __nv_bfloat16 pc[3][8];
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const int64_t h = k0 + d;
                float w = 0.0f;
                if (h < a.H && c < a.C && dig[0] < a.f0_rows) {
                    w = 1.0f;
                    for (int z = 0; z < a.head; ++z) w *= __ldg(a.fac[z] + dig[z] * a.C + c);
                }
                split3(w, pc[0][d], pc[1][d], pc[2][d]);
                for (int z = 0; z < a.head; ++z) {           // next row: mixed-radix increment
                    if (++dig[z] < a.frad[z]) break;
                    dig[z] = 0;
                }
            }
            const int64_t slice = k0 / PS_BK;
            const int oct = (int)((k0 % PS_BK) / 8);
            uint8_t* base = a.img + slice * (int64_t)(a.N * 128);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int n = q * a.CP + c;
                const uint32_t off = (uint32_t)((n >> 3) * 1024 + (n & 7) * 128 + (((oct ^ (n & 7)) & 7) << 4));
                uint4 v;
                v.x = (uint32_t)__bfloat16_as_ushort(pc[q][0]) | ((uint32_t)__bfloat16_as_ushort(pc[q][1]) << 16);
                v.y = (uint32_t)__bfloat16_as_ushort(pc[q][2]) | ((uint32_t)__bfloat16_as_ushort(pc[q][3]) << 16);
                v.z = (uint32_t)__bfloat16_as_ushort(pc[q][4]) | ((uint32_t)__bfloat16_as_ushort(pc[q][5]) << 16);
                v.w = (uint32_t)__bfloat16_as_ushort(pc[q][6]) | ((uint32_t)__bfloat16_as_ushort(pc[q][7]) << 16);
                *reinterpret_cast<uint4*>(base + off) = v;
            }
        } else {
            const int64_t e = it - n_img;
            const int c4 = a.CP / 4;
            const uint32_t q = (uint32_t)(e / c4);
            const int c0 = 4 * (int)(e - (int64_t)q * c4);
            float prod[4] = {1.0f, 1.0f, 1.0f, 1.0f};
            uint32_t rem = q;
            for (int z = 0; z < a.ntail; ++z) {
                const uint32_t rad = (uint32_t)a.tail_rad[z];
                const uint32_t nq = rem / rad;
                const float* row = a.tail[z] + (int64_t)(rem - nq * rad) * a.C;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (c0 + j < a.C) prod[j] *= __ldg(row + c0 + j);
                rem = nq;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (c0 + j >= a.C) prod[j] = 0.0f;
            *reinterpret_cast<float4*>(a.qtab + (int64_t)q * a.CP + c0) = make_float4(prod[0], prod[1], prod[2], prod[3]);
        }
    }
}

// out = sum of the partial slabs of each output's tile.  The slabs have the output's
// layout (row-major [i][c] or column-major [c][i]; both dense), so one flat index f
// addresses an output and its entry in every slab.  A block of W warps takes 32 Q
// consecutive outputs, Q per lane (one float4 when Q = 4 and the 4 share their slab count
// and the buffers allow it); warp w adds slabs w, w + W, ... in order and the W warp sums
// are added in warp order, so the result does not depend on scheduling.  Many outputs
// and few slabs (a tall partial MTTKRP): Q = 4, W <= 8; few outputs and many slabs: Q = 1
// and up to 32 warps, so that enough loads are in flight.
struct ReduceShape {
    int64_t I;
    int C, BI, U, ntiles, s_full, s_last;
    int sk;                 // stream-K: slabs of a tile = its pieces (0: a whole-tile unit wrote it)
    int64_t stot, tot, G;
    int64_t opad, oreal, Iout;   // output row map (as in PsParams), output rows
};

// where output f of the slabs' layout goes in the output (-1: a padding row, dropped)
__device__ __forceinline__ int64_t reduce_out(const ReduceShape& rs, int64_t f, int colmajor) {
    if (!rs.opad) return f;
    const int64_t i = colmajor ? f % rs.I : f / rs.C;
    const int64_t c = colmajor ? f / rs.I : f - i * rs.C;
    const int64_t q = i / rs.opad, rr = i - q * rs.opad;
    if (rr >= rs.oreal) return -1;
    const int64_t io = rr + rs.oreal * q;
    return colmajor ? c * rs.Iout + io : io * rs.C + c;
}

// slabs that hold pieces of output f (0: its tile was written whole, nothing to add)
__device__ __forceinline__ int reduce_slabs(const ReduceShape& rs, int64_t f, int colmajor) {
    const int64_t i = colmajor ? f % rs.I : f / rs.C;
    const int64_t tile = i / rs.BI;
    if (rs.sk) {
        const int64_t np = sk_cta((tile + 1) * rs.stot - 1, rs.tot, rs.G) - sk_cta(tile * rs.stot, rs.tot, rs.G) + 1;
        return (np > 1 || rs.U > 1) ? (int)np * rs.U : 0;
    }
    return (tile < rs.ntiles - 1 ? rs.s_full : rs.s_last) * rs.U;
}

// Few slabs (<= 8) and many outputs: a thread takes 4 consecutive outputs (one 16-byte
// word), loads all of their slabs at once and adds them in slab order.
constexpr int kFewSlabs = 8;
__global__ void __launch_bounds__(256) planes_reduce_few_kernel(const float* __restrict__ part, const ReduceShape rs,
                                                               float* __restrict__ out, int colmajor, int vec,
                                                               const uint32_t* status) {
    allow_dependent_launch();
    if (status && (*reinterpret_cast<const volatile uint32_t*>(status) & (1u << MTK_ETIMEOUT))) return;
    const int64_t n = rs.I * rs.C;
    const int64_t ng = (n + 3) / 4;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f0 = 4 * g;
        int ns[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) ns[j] = f0 + j < n ? reduce_slabs(rs, f0 + j, colmajor) : 0;
        if (vec && f0 + 3 < n && ns[0] > 0 && ns[1] == ns[0] && ns[2] == ns[0] && ns[3] == ns[0]) {
            float4 x[kFewSlabs];
#pragma unroll
            for (int sl = 0; sl < kFewSlabs; ++sl)
                if (sl < ns[0]) x[sl] = __ldg(reinterpret_cast<const float4*>(part + (int64_t)sl * n + f0));
            float4 a = x[0];
#pragma unroll
            for (int sl = 1; sl < kFewSlabs; ++sl) {
                if (sl < ns[0]) {
                    a.x += x[sl].x;
                    a.y += x[sl].y;
                    a.z += x[sl].z;
                    a.w += x[sl].w;
                }
            }
            *reinterpret_cast<float4*>(out + f0) = a;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (ns[j] == 0) continue;
                float a = 0.0f;
                for (int sl = 0; sl < ns[j]; ++sl) a += __ldg(part + (int64_t)sl * n + f0 + j);
                const int64_t o = reduce_out(rs, f0 + j, colmajor);
                if (o >= 0) out[o] = a;
            }
        }
    }
}

template <int Q>
__global__ void __launch_bounds__(1024) planes_reduce_kernel(const float* __restrict__ part, const ReduceShape rs,
                                                             float* __restrict__ out, int colmajor, int vec,
                                                             const uint32_t* status) {
    const int64_t I = rs.I;
    const int C = rs.C;
    allow_dependent_launch();
    // a contraction that timed out left its slabs incomplete: the output stays as it was
    if (status && (*reinterpret_cast<const volatile uint32_t*>(status) & (1u << MTK_ETIMEOUT))) return;
    __shared__ float red[32][32 * Q];
    const int W = (int)(blockDim.x >> 5);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = I * C;
    const int64_t f0 = ((int64_t)blockIdx.x * 32 + lane) * Q;
    auto slabs = [&](int64_t f) -> int { return reduce_slabs(rs, f, colmajor); };
    float v[Q];
    int nsj[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        v[j] = 0.0f;
        nsj[j] = f0 + j < n ? slabs(f0 + j) : 0;
    }
    bool v4 = false;
    if (f0 < n) {
        const int ns = nsj[0];
        if (Q == 4) v4 = vec && f0 + 3 < n && ns > 0 && nsj[1 % Q] == ns && nsj[2 % Q] == ns && nsj[3 % Q] == ns;
        if (v4) {
            for (int sl = w; sl < ns; sl += W) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(part + (int64_t)sl * n + f0));
                v[0] += x.x;
                v[1 % Q] += x.y;
                v[2 % Q] += x.z;
                v[3 % Q] += x.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const int64_t f = f0 + j;
                if (f < n) {
                    const int nj = nsj[j];
                    float a = 0.0f;
                    for (int sl = w; sl < nj; sl += W) a += __ldg(part + (int64_t)sl * n + f);
                    v[j] = a;
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) red[w][lane * Q + j] = v[j];
    __syncthreads();
    if (w == 0 && f0 < n) {
        float t[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) t[j] = red[0][lane * Q + j];
        for (int k = 1; k < W; ++k)
#pragma unroll
            for (int j = 0; j < Q; ++j) t[j] += red[k][lane * Q + j];
        if (v4) {
            *reinterpret_cast<float4*>(out + f0) = make_float4(t[0], t[1 % Q], t[2 % Q], t[3 % Q]);
        } else {
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                if (f0 + j < n && nsj[j] > 0) {
                    const int64_t o = reduce_out(rs, f0 + j, colmajor);
                    if (o >= 0) out[o] = t[j];
                }
            }
        }
    }
}

// ---- the split into planes, with ||X||^2 --------------------------------------------
// (a, b) -> packed BF16 pairs hi = (bf16_rn(a), bf16_rn(b)) and lo = the BF16 rounding of
// the remainders (exact in FP32); the first value in the low half (lower address)
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hw, uint32_t& lw) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hw = *reinterpret_cast<const uint32_t*>(&h);
    lw = *reinterpret_cast<const uint32_t*>(&l);
}
__device__ __forceinline__ void split_one(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
}

#ifndef MTK_SPLIT_UNROLL
#define MTK_SPLIT_UNROLL 4
#endif
constexpr int SPLIT_UNROLL = MTK_SPLIT_UNROLL;   // 16-byte loads in flight per thread

__global__ void __launch_bounds__(256) split_planes_kernel(const float* __restrict__ X, int64_t NX, int64_t pitch,
                                                           int64_t chunk, __nv_bfloat16* __restrict__ Xs,
                                                           double* __restrict__ part) {
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = (b0 + chunk < NX) ? b0 + chunk : NX;
    __nv_bfloat16* hi = Xs;
    __nv_bfloat16* lo = Xs + pitch;
    // ||X||^2 (SquareSum: no FP64 arithmetic until the end)
    SquareSum sq;
    int cnt = 0;
    auto add_sq = [&](float x) { sq.add(x); };
    auto flush = [&]() { sq.flush(); };
    const bool vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && ((reinterpret_cast<uintptr_t>(Xs) & 15) == 0) &&
                     (pitch % 4 == 0) && (chunk % 4 == 0);
    if (vec) {
        // SPLIT_UNROLL loads of 16 bytes in flight per thread (one at a time left the copy at
        // about 0.57 of the HBM bandwidth); a thread still visits v = tid, tid + 256, ... in
        // order, so the sum of squares is the same for any unroll
        const int64_t n4 = (b1 - b0) / 4;
        for (int64_t v0 = threadIdx.x; v0 < n4; v0 += SPLIT_UNROLL * (int64_t)blockDim.x) {
            float4 xv[SPLIT_UNROLL];
#pragma unroll
            for (int u = 0; u < SPLIT_UNROLL; ++u) {
                const int64_t v = v0 + u * (int64_t)blockDim.x;
                xv[u] = v < n4 ? __ldcs(reinterpret_cast<const float4*>(X + b0 + 4 * v)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < SPLIT_UNROLL; ++u) {
                const int64_t v = v0 + u * (int64_t)blockDim.x;
                if (v >= n4) break;
                const int64_t e = b0 + 4 * v;
                const float4 x = xv[u];
                uint2 hw, lw;
                split_pair(x.x, x.y, hw.x, lw.x);
                split_pair(x.z, x.w, hw.y, lw.y);
                add_sq(x.x);
                add_sq(x.y);
                add_sq(x.z);
                add_sq(x.w);
                if (++cnt == 16) { flush(); cnt = 0; }
                *reinterpret_cast<uint2*>(hi + e) = hw;
                *reinterpret_cast<uint2*>(lo + e) = lw;
            }
        }
        for (int64_t e = b0 + 4 * n4 + threadIdx.x; e < b1; e += blockDim.x) {
            const float x = X[e];
            split_one(x, hi[e], lo[e]);
            add_sq(x);
        }
    } else {
        for (int64_t e = b0 + threadIdx.x; e < b1; e += blockDim.x) {
            const float x = X[e];
            split_one(x, hi[e], lo[e]);
            add_sq(x);
            if (++cnt == 64) { flush(); cnt = 0; }
        }
    }
    // fixed-order block reduction
    __shared__ double red[256];
    red[threadIdx.x] = sq.value();
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && part) part[blockIdx.x] = red[0];
}

// The split into planes whose mode 0 is padded from I0 to I0p (a multiple of 8) entries:
// output entries e = i0 + I0p r, four at a time (i0 a multiple of 4, the four in one row),
// x = X[i0 + I0 r] for i0 < I0 and 0 in the padding; ||X||^2 as in split_planes_kernel
__global__ void __launch_bounds__(256) split_planes_padded_kernel(const float* __restrict__ X, int64_t I0,
                                                                  int64_t I0p, int64_t NXp, int64_t pitch,
                                                                  int64_t chunk, __nv_bfloat16* __restrict__ Xs,
                                                                  double* __restrict__ part) {
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = (b0 + chunk < NXp) ? b0 + chunk : NXp;
    __nv_bfloat16* hi = Xs;
    __nv_bfloat16* lo = Xs + pitch;
    SquareSum sq;
    int cnt = 0;
    auto add_sq = [&](float x) { sq.add(x); };
    auto flush = [&]() { sq.flush(); };
    const int64_t n4 = (b1 - b0) / 4;                    // b0, b1: multiples of 4 (I0p % 8 == 0)
    for (int64_t v0 = threadIdx.x; v0 < n4; v0 += SPLIT_UNROLL * (int64_t)blockDim.x) {
        float xv[SPLIT_UNROLL][4];
#pragma unroll
        for (int u = 0; u < SPLIT_UNROLL; ++u) {
            const int64_t v = v0 + u * (int64_t)blockDim.x;
            const int64_t e = b0 + 4 * v;
            const int64_t r = e / I0p;
            const int64_t i0 = e - r * I0p;
            const float* src = X + i0 + I0 * r;
#pragma unroll
            for (int j = 0; j < 4; ++j) xv[u][j] = (v < n4 && i0 + j < I0) ? __ldcs(src + j) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < SPLIT_UNROLL; ++u) {
            const int64_t v = v0 + u * (int64_t)blockDim.x;
            if (v >= n4) break;
            const int64_t e = b0 + 4 * v;
            uint2 hw, lw;
            split_pair(xv[u][0], xv[u][1], hw.x, lw.x);
            split_pair(xv[u][2], xv[u][3], hw.y, lw.y);
#pragma unroll
            for (int j = 0; j < 4; ++j) add_sq(xv[u][j]);
            if (++cnt == 16) { flush(); cnt = 0; }
            *reinterpret_cast<uint2*>(hi + e) = hw;
            *reinterpret_cast<uint2*>(lo + e) = lw;
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = sq.value();
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && part) part[blockIdx.x] = red[0];
}

// one warp: lane l adds part[l], part[l + 32], ... in order, then a fixed shuffle tree
// (a chain of n dependent FP64 adds on one thread took ~40 us for n = 1216)
__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
    const int l = threadIdx.x;
    double s = 0.0;
    for (int k = l; k < n; k += 32) s += part[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (l == 0 && blockIdx.x == 0) *out = s;
}

// block: warp 0 tensor producer, warp 1 MMA issuer (TMEM owner), warp 2 image producer,
// then four drain warps per 128-row MMA tile
// pdl: launched with programmatic stream serialisation (it may start while the kernel
// before it, a factorisation, still runs)
template <int NCH, bool MN, int MT>
cudaError_t launch_planes_mt(const PsParams& p, const CUtensorMap& map, int grid, size_t smem, cudaStream_t s,
                             bool pdl) {
    cudaError_t e = cudaFuncSetAttribute(contract_planes_kernel<NCH, MN, MT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(96 + 128 * MT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, contract_planes_kernel<NCH, MN, MT>, p, map);
    note_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int NCH, bool MN>
cudaError_t launch_planes_variant(const PsParams& p, const CUtensorMap& map, int grid, size_t smem, cudaStream_t s,
                                  bool pdl) {
    return p.MT == 2 ? launch_planes_mt<NCH, MN, 2>(p, map, grid, smem, s, pdl)
                     : launch_planes_mt<NCH, MN, 1>(p, map, grid, smem, s, pdl);
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

int64_t planes_rows0(int64_t I0) { return round_up(I0, 8); }

void planes_dims(const int64_t* dims, int N, int64_t* pd) {
    for (int k = 0; k < N; ++k) pd[k] = dims[k];
    pd[0] = planes_rows0(dims[0]);
}

int64_t split_pitch(int64_t NXp) { return round_up(NXp, 64); }

int split_chunks(int64_t NXp) {
    int64_t nb = (NXp + 4095) / 4096;
    if (nb > 1216) nb = 1216;
    if (nb < 1) nb = 1;
    return (int)nb;
}

cudaError_t launch_split_planes(const float* X, int64_t I0, int64_t rest, void* Xs, double* part,
                                double* normX2, cudaStream_t s) {
    const int64_t I0p = planes_rows0(I0);
    const int64_t NX = I0p * rest;
    const int nb = split_chunks(NX);
    const int64_t chunk = round_up((NX + nb - 1) / nb, 1024);
    const int grid = (int)((NX + chunk - 1) / chunk);
    if (I0p == I0)
        split_planes_kernel<<<grid, 256, 0, s>>>(X, NX, split_pitch(NX), chunk, static_cast<__nv_bfloat16*>(Xs), part);
    else
        split_planes_padded_kernel<<<grid, 256, 0, s>>>(X, I0, I0p, NX, split_pitch(NX), chunk,
                                                        static_cast<__nv_bfloat16*>(Xs), part);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !normX2) return e;
    sum_partials_kernel<<<1, 32, 0, s>>>(part, grid, normX2);
    note_launches(1);
    return cudaGetLastError();
}

PlanesPlan planes_plan(int64_t L, int64_t I, const int64_t* frad, int nfac, int C, int n_left, int ctas) {
    PlanesPlan pl;
    memset(&pl, 0, sizeof(pl));
    if (C < 1 || C > 64 || nfac < 1) return pl;
    const int64_t lim = ((int64_t)1 << 31) - 1;
    const bool mn = (L == 1);
    // TMA loads start on 16-byte boundaries: MN-major boxes at i = multiples of 64 of rows
    // of I_n elements, K-major rows (i, r) at element I^L (i + I_n r) and runs at H lq
    // within them.  The planes keep mode 0 padded to a multiple of 8, so I^L (n >= 1) and
    // every head (a prefix of the factors, U_0 first) are multiples of 8.
    if (mn) {
        if (I % 8 != 0) return pl;
    } else {
        if (n_left < 1 || L % 8 != 0 || L > lim) return pl;
    }
    int64_t K = 1;
    for (int z = 0; z < nfac; ++z) K *= frad[z];
    pl.CP = (C + 15) & ~15;
    pl.N = 3 * pl.CP;
    // head: a prefix of the factor list (K-major: within the modes left of n, a multiple
    // of 8 rows or all of I^L, so that runs start on 16-byte boundaries).  The first prefix
    // with >= 64 rows and <= 1/32 padding, else the least padding, among those whose images
    // stay L2-resident.  A K-major mode with few rows (I_n <= 128) packs several runs per
    // tile, runs lq, lq + 1, ... of one row at a stride of H elements: a short head keeps
    // them within a few KB, so that each stage reads a few contiguous spans instead of one
    // 128-byte piece of every run, and that is worth up to 1/4 padding (measured on
    // 200x200x300x40, mode 3: 349 us with H = 200 against 444 us with H = 40,000).
    const int mmax = mn ? nfac : n_left;
    const bool near_runs = !mn && I <= PS_M;
    int best = -1;
    double best_waste = 2.0;
    int64_t prod = 1;
    for (int m = 1; m <= mmax; ++m) {
        prod *= frad[m - 1];
        if (!mn && prod % 8 != 0 && L / prod != 1) continue;
        const int64_t padded = round_up(prod, PS_BK);
        const size_t img = (size_t)(padded / PS_BK) * pl.N * 128;
        if (img > ((size_t)32 << 20)) break;
        const double waste = (double)(padded - prod) / (double)padded;
        const int64_t hp = (near_runs && L / prod > 1) ? MTK_PS_HEAD_PAD_NEAR : MTK_PS_HEAD_PAD;
        if (prod >= PS_BK && (padded - prod) * hp <= padded) { best = m; break; }
        if (waste < best_waste) { best_waste = waste; best = m; }
    }
    if (best < 0) return pl;
    int64_t H = 1;
    for (int z = 0; z < best; ++z) H *= frad[z];
    pl.head = best;
    pl.H = H;
    pl.Lq = mn ? 1 : L / H;
    pl.spr = (int)(round_up(H, PS_BK) / PS_BK);
    pl.nruns = K / H;
    if (H > lim || pl.nruns > lim || I > lim || (!mn && (K / L) > lim) || (!mn && I * (K / L) > lim)) return pl;
    pl.mn = mn ? 1 : 0;
    const int64_t maxU = pl.nruns;
    const int64_t Ic = I;
    // Rows of a CTA tile: up to 256 (two 128-row MMA tiles).  Each stage has a fixed cost
    // besides its bytes, so the tiling carries as many rows per stage as it can: BI rows of
    // i per run group and, when BI <= 128, U run groups of the head (different runs q,
    // the same rows) packed one above the other; each packed group is a partial slab of
    // its own.  K-major: the fewest i-tiles of at most 256 rows when they are at least 3/4
    // full; otherwise the number of i-tiles that maximises U * BI, preferring fewer tiles
    // (each packed group adds partial slabs) unless the rows grow by more than an eighth.
    // MN-major (i is the contiguous index, loaded in 64-row boxes): tiles of 256 rows, or
    // of 128 when I_n <= 128, and up to four packed 64-row groups when I_n <= 64.
    if (mn) {
        if (I <= 64) {
            pl.BI = 64;
            pl.U = (int)(pl.nruns < 4 ? pl.nruns : 4);
            pl.MT = pl.U > 2 ? 2 : 1;
            pl.ntiles = 1;
            pl.box_mode = pl.U > 1 ? 1 : 0;           // the runs' 64-row boxes in one load
        } else {
            pl.U = 1;
            pl.MT = I > PS_M ? 2 : 1;
            pl.BI = PS_M * pl.MT;
            pl.ntiles = (int)((I + pl.BI - 1) / pl.BI);
        }
    } else {
        const int64_t t0 = (Ic + 2 * PS_M - 1) / (2 * PS_M);
        int64_t best_bi = round_up((Ic + t0 - 1) / t0, 8), best_u = 1;
        if (best_bi <= PS_M) {
            best_u = (2 * PS_M) / best_bi;
            if (best_u > maxU) best_u = maxU;
        }
        int64_t best_rows = best_u * best_bi;
        if (MTK_PS_TILE_MODEL == 1 && best_rows * 4 < 3 * 2 * PS_M) {
            // the fewest stages: t i-tiles x ceil(runs / u) groups (ties: fewer tiles)
            int64_t best_st = t0 * ((pl.nruns + best_u - 1) / best_u);
            for (int64_t t = t0 + 1; t <= t0 + 64 && t <= (Ic + 7) / 8; ++t) {
                const int64_t bi = round_up((Ic + t - 1) / t, 8);
                int64_t u = 1;
                if (bi <= PS_M) {
                    u = (2 * PS_M) / bi;
                    if (u > maxU) u = maxU;
                }
                const int64_t st = t * ((pl.nruns + u - 1) / u);
                if (st < best_st) {
                    best_st = st;
                    best_rows = u * bi;
                    best_bi = bi;
                    best_u = u;
                }
            }
        } else if (best_rows * 4 < 3 * 2 * PS_M) {
            for (int64_t t = t0 + 1; t <= t0 + 64 && t <= (Ic + 7) / 8; ++t) {
                const int64_t bi = round_up((Ic + t - 1) / t, 8);
                int64_t u = 1;
                if (bi <= PS_M) {
                    u = (2 * PS_M) / bi;
                    if (u > maxU) u = maxU;
                }
                if (u * bi * 8 > best_rows * 9) {
                    best_rows = u * bi;
                    best_bi = bi;
                    best_u = u;
                }
            }
        }
        // packed runs in one TMA box when they lie at one stride: consecutive r (one run per
        // row) or consecutive lq of the same r (U dividing the runs per row; U is lowered to
        // a divisor when that keeps at least half of it)
        if (best_u > 1 && pl.Lq == 1) {
            pl.box_mode = 1;
        } else if (best_u > 1) {
            // U lowered to a divisor of Lq when that keeps at least 7/8 of it; otherwise the
            // groups are row-local (ceil(Lq / U) per r, the last one partly empty) when
            // that wastes under 1/8 of the rows
            int64_t u = best_u;
            while (u > 1 && pl.Lq % u != 0) --u;
            const int64_t gpr = (pl.Lq + best_u - 1) / best_u;
            if (8 * u >= 7 * best_u) {
                best_u = u;
                best_rows = u * best_bi;
                pl.box_mode = 2;
            } else if (8 * (gpr * best_u - pl.Lq) <= gpr * best_u) {
                pl.box_mode = 2;
                pl.gpr = gpr;
            } else if (2 * u >= best_u) {
                best_u = u;
                best_rows = u * best_bi;
                pl.box_mode = 2;
            }
        }
        pl.BI = (int)best_bi;
        pl.U = (int)best_u;
        if (pl.U > PS_MAX_U) return pl;
        pl.MT = best_rows > PS_M ? 2 : 1;
        pl.ntiles = (int)((Ic + pl.BI - 1) / pl.BI);
    }
    pl.stot = (pl.gpr ? (pl.nruns / pl.Lq) * pl.gpr : (pl.nruns + pl.U - 1) / pl.U) * pl.spr;
    // Work split.  A stage costs a fixed ~750 cycles besides its bytes, so a ragged last
    // tile (fewer rows, the same stages) costs nearly as much as a full one: the stages,
    // not the rows, are shared out.
    const int T = pl.ntiles;
    int64_t smax = pl.stot / 4;
    if (smax < 1) smax = 1;
    int64_t G = ctas;
    if (T >= 2) {
        // stream-K.  CTA c takes the stages [c tot / G, (c + 1) tot / G) of the flattened
        // (tile, stage) space (tot = T stot, G CTAs of at least 4 stages), so every CTA has
        // the same number of stages to within one; it runs the tiles its range touches back
        // to back with the rings and TMEM kept live.  A tile that one CTA covers whole goes
        // straight to the output; the pieces of a tile split between CTAs are partial slabs,
        // at most ceil(stot / (tot / G)) + 1 of them.
        const int64_t tot = (int64_t)T * pl.stot;
        if (G > tot / 4) G = tot / 4;
        if (G < 1) G = 1;
        const int64_t per = tot / G;
        const int64_t kmax = (pl.stot + per - 1) / per + 1;
        pl.sk = 1;
        pl.s_full = pl.s_last = (int)kmax;
    } else {
        // one tile: its stages split evenly, one slab per CTA
        pl.s_full = pl.s_last = (int)(ctas < smax ? ctas : smax);
    }
    pl.grid = pl.sk ? (int)G : pl.s_full;
    pl.nslab = (pl.s_full > pl.s_last ? pl.s_full : pl.s_last) * pl.U;
    pl.image_bytes = (size_t)pl.spr * pl.N * 128;
    // table of tail scales Q(q, c) when it is small
    const size_t qbytes = (size_t)pl.nruns * pl.CP * sizeof(float);
    pl.qtab_bytes = (nfac > best && qbytes <= ((size_t)32 << 20)) ? qbytes : 0;
    pl.part_bytes = pl.nslab > 1 ? (size_t)pl.nslab * I * C * sizeof(float) : 0;
    pl.ok = 1;
    return pl;
}

size_t planes_scratch_bytes(const PlanesPlan& pl) {
    return round_up((int64_t)pl.image_bytes, 256) + round_up((int64_t)pl.qtab_bytes, 256) +
           round_up((int64_t)pl.part_bytes, 256);
}

int planes_ctas(int splits) { return splits > 0 ? splits : num_sms(); }

cudaError_t launch_contract_planes(const void* Xs, int64_t pitch, int64_t L, int64_t I, int64_t R,
                                   const float* const* fac, const int64_t* frad, int nfac, int C,
                                   const PlanesPlan& pl, float* out, int64_t out_si, int64_t out_sc,
                                   void* scratch, uint32_t* status, cudaStream_t s,
                                   unsigned long long wait_ns, int stall, const FactorHook* hook,
                                   int64_t f0_rows, int64_t opad, int64_t oreal) {
    if (opad < 0 || (opad > 0 && (oreal < 1 || oreal > opad || I % opad != 0))) return cudaErrorInvalidValue;
    if (opad == oreal) opad = 0;
    const int64_t Iout = opad ? (I / opad) * oreal : I;
    char* sc = static_cast<char*>(scratch);
    uint8_t* image = reinterpret_cast<uint8_t*>(sc);
    float* qtab = pl.qtab_bytes ? reinterpret_cast<float*>(sc + round_up((int64_t)pl.image_bytes, 256)) : nullptr;
    float* part = reinterpret_cast<float*>(sc + round_up((int64_t)pl.image_bytes, 256) +
                                           round_up((int64_t)pl.qtab_bytes, 256));

    // 1) the B image of the head and the table of tail scales (one launch)
    PrepArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.head = pl.head;
    pa.C = C;
    pa.CP = pl.CP;
    pa.N = pl.N;
    for (int z = 0; z < pl.head; ++z) {
        pa.fac[z] = fac[z];
        pa.frad[z] = frad[z];
    }
    pa.f0_rows = f0_rows > 0 && f0_rows < frad[0] ? f0_rows : frad[0];
    pa.H = pl.H;
    pa.Hp = (int64_t)pl.spr * PS_BK;
    pa.img = image;
    pa.ntail = nfac - pl.head;
    for (int z = pl.head; z < nfac; ++z) {
        pa.tail[z - pl.head] = fac[z];
        pa.tail_rad[z - pl.head] = frad[z];
    }
    pa.nruns = pl.nruns;
    pa.qtab = qtab;
    {
        const int64_t items = (pa.Hp / 8) * pl.CP + (qtab ? pl.nruns * (pl.CP / 4) : 0);
        int64_t blocks = (items + 255) / 256;
        if (blocks > num_sms() * 8) blocks = num_sms() * 8;
        planes_prep_kernel<<<(int)blocks, 256, 0, s>>>(pa);
        note_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (hook) {
        const cudaError_t e = launch_als_factor(hook->G, hook->N, hook->C, hook->n, hook->hinv, hook->status, s);
        if (e != cudaSuccess) return e;
    }

    // 2) the tensor map over both planes
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    CUresult r;
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    if (pl.mn) {
        const cuuint64_t dims[4] = {(cuuint64_t)I, (cuuint64_t)pl.H, (cuuint64_t)pl.nruns, 2};
        const cuuint64_t strides[3] = {(cuuint64_t)I * 2, (cuuint64_t)I * pl.H * 2, (cuuint64_t)pitch * 2};
        const cuuint32_t box[4] = {64, 64, (cuuint32_t)(pl.box_mode ? pl.U : 1), 1};
        r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(Xs), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, promo(MTK_PS_MN_PROMO),
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else if (pl.box_mode == 1) {
        // packed runs along r (one run per row): (l, i, r, plane), box (64, BI, U)
        const cuuint64_t dims[4] = {(cuuint64_t)L, (cuuint64_t)I, (cuuint64_t)R, 2};
        const cuuint64_t strides[3] = {(cuuint64_t)L * 2, (cuuint64_t)L * I * 2, (cuuint64_t)pitch * 2};
        const cuuint32_t box[4] = {64, (cuuint32_t)pl.BI, (cuuint32_t)pl.U, 1};
        r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(Xs), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, promo(MTK_PS_KM_PROMO),
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else if (pl.box_mode == 2) {
        // packed runs along lq: (h, lq, i, r, plane), box (64, U, BI)
        const cuuint64_t dims[5] = {(cuuint64_t)pl.H, (cuuint64_t)pl.Lq, (cuuint64_t)I, (cuuint64_t)R, 2};
        const cuuint64_t strides[4] = {(cuuint64_t)pl.H * 2, (cuuint64_t)L * 2, (cuuint64_t)L * I * 2,
                                       (cuuint64_t)pitch * 2};
        const cuuint32_t box[5] = {64, (cuuint32_t)pl.U, (cuuint32_t)pl.BI, 1, 1};
        r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(Xs), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, promo(MTK_PS_KM_PROMO),
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        // K-major: rows (i, r) of I^L elements (a multiple of 8); both planes
        const cuuint64_t dims[3] = {(cuuint64_t)L, (cuuint64_t)(I * R), 2};
        const cuuint64_t strides[2] = {(cuuint64_t)L * 2, (cuuint64_t)pitch * 2};
        const cuuint32_t box[3] = {64, (cuuint32_t)pl.BI, 1};
        r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(Xs), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, promo(MTK_PS_KM_PROMO),
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;

    // 3) the contraction
    PsParams p;
    memset(&p, 0, sizeof(p));
    p.I = I;
    p.nruns = pl.nruns;
    p.Lq = pl.Lq;
    p.gpr = pl.gpr;
    p.stot = pl.stot;
    p.H = pl.H;
    p.spr = pl.spr;
    p.U = pl.U;
    p.BI = pl.BI;
    p.MT = pl.MT;
    p.box_mode = pl.box_mode;
    p.C = C;
    p.CP = pl.CP;
    p.N = pl.N;
    // A stage: both planes of the tile.  K-major planes hold only the rows they load
    // (U * BI, a multiple of 8: whole 1024-byte swizzle atoms); the MMAs still read
    // MT x 128 rows from each plane base, and the rows beyond the tile (the next plane or
    // stage, or the B ring after the last stage) only feed accumulator rows that are never
    // drained.
    const int tile_rows = pl.U > 1 ? pl.U * pl.BI : pl.BI;
    p.plane_bytes = !pl.mn ? (int)round_up(tile_rows, 8) * 128 : pl.MT * PS_TILE;
    p.a_stage = 2 * p.plane_bytes;
    p.b_bytes = pl.N * 128;
    p.b_stage = (int)round_up(p.b_bytes, 1024);
    // shared memory: the A ring (tensor tiles, HBM latency) as deep as fits next to the
    // shallowest useful B ring (image slices, L2 latency), then the rest to the B ring
    const int budget = 225 * 1024;
    const int sb_min = pl.MT == 1 ? MTK_PS_SB_MIN1 : 2;
    p.sa = (budget - sb_min * p.b_stage) / p.a_stage;
    if (p.sa > PS_MAX_A) p.sa = PS_MAX_A;
    p.sb = (budget - p.sa * p.a_stage) / p.b_stage;
    if (p.sb > PS_MAX_B) p.sb = PS_MAX_B;
    if (p.sa < 2 || p.sb < 2) return cudaErrorInvalidConfiguration;
    // the over-read of the last stage's lo plane (MT x 128 rows from its base) stays
    // inside the B ring
    if (pl.MT * PS_TILE - p.plane_bytes > p.sb * p.b_stage) return cudaErrorInvalidConfiguration;
    p.b_base = p.sa * p.a_stage;
    p.lo_sep = (pl.MT == 1 && PS_LO_SEP) ? 1 : 0;
    p.acc_cols = p.lo_sep ? pl.N + 2 * pl.CP : pl.MT * pl.N;
    p.nbuf = 512 / p.acc_cols;
    if (p.nbuf > PS_MAX_BUF) p.nbuf = PS_MAX_BUF;
    if (p.nbuf < 1) return cudaErrorInvalidConfiguration;
    int cols = 32;
    while (cols < p.nbuf * p.acc_cols) cols <<= 1;
    p.tmem_cols = cols;
    p.idesc_hi = idesc_bf16(PS_M, pl.N, pl.mn != 0);
    p.idesc_lo = idesc_bf16(PS_M, 2 * pl.CP, pl.mn != 0);
    p.ntiles = pl.ntiles;
    p.s_full = pl.s_full;
    p.s_last = pl.s_last;
    p.nslab = pl.nslab;
    p.sk = pl.sk;
    p.sk_tot = (int64_t)pl.ntiles * pl.stot;
    p.bimg = image;
    p.qtab = qtab;
    p.ntail = nfac - pl.head;
    for (int z = pl.head; z < nfac; ++z) {
        p.tail[z - pl.head] = fac[z];
        p.tail_rad[z - pl.head] = frad[z];
    }
    p.out = out;
    p.out_si = out_si;
    p.out_sc = out_sc;
    p.opad = opad;
    p.oreal = oreal;
    p.part = part;
    // slabs in the output's layout (over the view's rows); the output is row-major
    // (si = C, sc = 1) or column-major (si = 1, sc = its rows)
    if (!((out_si == C && out_sc == 1) || (out_si == 1 && out_sc == Iout))) return cudaErrorInvalidValue;
    p.part_cm = (out_si == 1 && C > 1) ? 1 : 0;
    p.status = status;
    p.wait_ns = wait_ns ? wait_ns : kPsWaitNs;
    p.stall = stall;
    const size_t smem = (size_t)p.sa * p.a_stage + (size_t)p.sb * p.b_stage + 1024;
    const int nch = pl.CP / 16;
    cudaError_t e;
    if (pl.mn) {
        switch (nch) {
            case 1: e = launch_planes_variant<1, true>(p, map, pl.grid, smem, s, hook != nullptr); break;
            case 2: e = launch_planes_variant<2, true>(p, map, pl.grid, smem, s, hook != nullptr); break;
            case 3: e = launch_planes_variant<3, true>(p, map, pl.grid, smem, s, hook != nullptr); break;
            default: e = launch_planes_variant<4, true>(p, map, pl.grid, smem, s, hook != nullptr); break;
        }
    } else {
        switch (nch) {
            case 1: e = launch_planes_variant<1, false>(p, map, pl.grid, smem, s, hook != nullptr); break;
            case 2: e = launch_planes_variant<2, false>(p, map, pl.grid, smem, s, hook != nullptr); break;
            case 3: e = launch_planes_variant<3, false>(p, map, pl.grid, smem, s, hook != nullptr); break;
            default: e = launch_planes_variant<4, false>(p, map, pl.grid, smem, s, hook != nullptr); break;
        }
    }
    if (e != cudaSuccess) return e;
    if (pl.nslab > 1) {
        const int64_t n = I * C;
        ReduceShape rs;
        rs.I = I;
        rs.C = C;
        rs.BI = pl.BI;
        rs.U = pl.U;
        rs.ntiles = pl.ntiles;
        rs.s_full = pl.s_full;
        rs.s_last = pl.s_last;
        rs.sk = pl.sk;
        rs.stot = pl.stot;
        rs.tot = (int64_t)pl.ntiles * pl.stot;
        rs.G = pl.grid;
        rs.opad = opad;
        rs.oreal = oreal;
        rs.Iout = Iout;
        const int vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0) &&
                        ((reinterpret_cast<uintptr_t>(part) & 15) == 0) && opad == 0;
        if (n >= 65536 && pl.nslab <= kFewSlabs) {
            const int64_t ng = (n + 3) / 4;
            int64_t blocks = (ng + 255) / 256;
            if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
            planes_reduce_few_kernel<<<(unsigned)blocks, 256, 0, s>>>(part, rs, out, p.part_cm, vec, status);
        } else if (n >= 65536) {
            const int W = pl.nslab < 8 ? pl.nslab : 8;
            planes_reduce_kernel<4><<<(unsigned)((n + 127) / 128), 32 * W, 0, s>>>(part, rs, out, p.part_cm, vec, status);
        } else {
            const int W = pl.nslab < 32 ? pl.nslab : 32;
            planes_reduce_kernel<1><<<(unsigned)((n + 31) / 32), 32 * W, 0, s>>>(part, rs, out, p.part_cm, 0, status);
        }
        note_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace mtk
