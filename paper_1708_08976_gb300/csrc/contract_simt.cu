// contract_simt.cu -- FP32 CUDA-core contraction D(i,c) = sum_k X3(k, i) W(k, c).
//
// This is the plain-FP32 form of the 1-step MTTKRP (Algorithms 2/3): the mode-n
// matricization is consumed in place as R row-major I x L blocks (Fig. 2), and
// the KRP rows W(k, :) are generated on chip from the factor rows (Algorithm 3
// forms K_R(j,:) kr K_L per block; here a block of 64 consecutive k is formed in
// shared memory and never written to HBM).  With a single materialised factor
// the same kernel is the GEMM of the materialised-KRP path and of the 2-step
// partial MTTKRP (Algorithm 4).
//
// Decomposition: grid = (i-tiles of 64, contraction splits S, column blocks of 2 TC).
// Each CTA owns a contiguous k-range (the private partial result of Algorithm 3), stages
// X tiles of 64 k through a 4-deep cp.async ring (16-byte copies when the rows allow it,
// else 4-byte ones; zero-filled outside the tensor) and generates the matching 64 x 2 TC
// block of W in shared memory.  Its 256 threads are 8 k-groups (one per warp, eight k of
// every 64-k stage each) x 16 row groups x 2 column groups: a thread accumulates the rows
// ig + 16 a (a = 0..3) x TC columns, so a row group past the end of a ragged tile is
// skipped by a whole warp.  Per stage a thread issues 8 x 4 x TC FMAs against 8 (K-major)
// or 32 (MN-major) shared loads of X and 8 x ceil(TC / 4) of W.  The eight k-groups are
// summed in shared memory in a fixed tree order; partials of the S splits are summed in
// split order by split_reduce_kernel (the parallel reduction of Algorithm 3), so results
// are deterministic.
//
// Layouts of an X stage: rows of i with k contiguous ([i][k]) when the view has I^L > 1
// (consecutive k are consecutive l in the tensor), columns of i ([k][i]) when I^L = 1
// (consecutive i are contiguous).
//
// 64-k stages (32 before) halve the per-FMA share of the per-stage work (copies, the W
// block, the barrier); with the row groups ig + 16 a the ragged last tile of a mode with
// few rows costs at most 15 extra rows instead of up to 63.
#include "mtk_internal.cuh"

namespace mtk {
namespace {

constexpr int BK = 64;        // k per stage (the planner's split quantum and minimum head)
constexpr int CB = 32;        // W stage slots per row: two groups of 16, the first TC of each used
constexpr int NKG = 8;        // k-groups per CTA (one warp each)
constexpr int KPG = BK / NKG; // k per group per stage
constexpr int THREADS = 256;
#ifndef MTK_SIMT_STAGES
#define MTK_SIMT_STAGES 4
#endif
constexpr int STAGES = MTK_SIMT_STAGES;   // X ring depth (3 stages, 52 KB, in flight per CTA)
constexpr int XPK = BK + 4;   // [i][k] stage: row pitch (floats)
constexpr int WP = CB + 4;    // W stage row pitch
constexpr int RP = CB + 4;    // reduction row pitch
constexpr int WROWS = BK * CB / THREADS;        // W values per thread per stage (8)

// RA rows per thread (rows ig + 16 a, a < RA): a CTA tile of BI = 16 RA rows
template <int RA>
struct SimtTile {
    static constexpr int BI = 16 * RA;
    static constexpr int XPM = BI + 4;          // [k][i] stage: row pitch
    static constexpr int XSTAGE = (BI * XPK > BK * XPM) ? BI * XPK : BK * XPM;
    static constexpr int XWORDS = BK * BI / 4 / THREADS;   // 16-byte copies per thread per stage
    static constexpr int MN_WPR = BI / 4;                  // MN: 16-byte words per k row
};

template <int RA>
struct __align__(16) SimtSmem {
    union {
        struct {
            float xs[STAGES][SimtTile<RA>::XSTAGE];
            float ws[2][BK][WP];
        } pipe;
        float red[NKG / 2][SimtTile<RA>::BI][RP];
    };
};

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
    unsigned saddr = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    int sz = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(saddr), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async16(float* smem, const float* gmem, bool valid) {
    unsigned saddr = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    int sz = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// KM: X stage [i][k] (I^L > 1); else [k][i] (I^L = 1).  VEC: 16-byte copies (KM: I^L a
// multiple of 4; else I_n a multiple of 4; the tensor 16-byte aligned, split starts at
// multiples of BK).
// TC: columns per thread (8, 13 or 16), so a CTA covers 2 TC columns of M: the fewest
// that hold C (C = 25 in 26 instead of 32).  RA: rows per thread (4: 64-row tiles, two
// CTAs per SM; 8 would give 128-row tiles, one CTA per SM, twice the FMAs per shared load
// of W, and measured slower).
template <bool KM, bool VEC, int TC, int RA>
__global__ void __launch_bounds__(THREADS, RA == 4 ? 2 : 1)
contract_simt_kernel(const __grid_constant__ ContractParams p) {
    constexpr int BI = SimtTile<RA>::BI;
    constexpr int XPM = SimtTile<RA>::XPM;
    constexpr int XWORDS = SimtTile<RA>::XWORDS;
    constexpr int WPR = SimtTile<RA>::MN_WPR;
    extern __shared__ __align__(16) uint8_t simt_smem_raw[];
    SimtSmem<RA>& sm = *reinterpret_cast<SimtSmem<RA>*>(simt_smem_raw);
    const int t = threadIdx.x;
    const int cg = t & 1, ig = (t >> 1) & 15, kg = t >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * BI;
    const int sp = blockIdx.y;
    const int c0 = blockIdx.z * 2 * TC;
    const int C = p.C;
    const int64_t L = p.L, I = p.I;
    const int64_t kb = (int64_t)sp * p.kchunk;
    const int64_t ke = (kb + p.kchunk < p.K) ? kb + p.kchunk : p.K;
    const int nst = (int)((ke - kb + BK - 1) / BK);
    const KrpOperand& W = p.W;
    const int rows_left = (I - i0) < BI ? (int)(I - i0) : BI;      // valid rows of this tile

    // uniform trackers of the stage start: (l, r) for X, (d0, q) for W
    int64_t xl = kb % L, xr = kb / L;            // X issue tracker (scalar copies)
    int64_t wd = kb % W.rad0, wq = kb / W.rad0;  // W generation tracker
    int64_t qcached = -1;
    const int64_t qtot = p.K / W.rad0;           // number of q values (rows of Q)

    // 16-byte copies: each thread issues XWORDS words of four floats per stage at fixed
    // positions of the stage tile and keeps the first word's tensor offset, advancing it by
    // constants from one stage to the next (no 64-bit products in the loop).
    //  KM: words (vi + 16 m, vk), vi = t / 16, vk = 4 (t % 16): four k of one row of the
    //      tensor (I^L % 4 == 0); offset l + I^L i + I^L I_n r, l = xl + vk.
    //  MN: words (vk + (256 / WPR) m, vi), vk = t / WPR, vi = 4 (t % WPR): four consecutive
    //      i of one k (WPR = BI / 4 words per k row); offset k I_n + i.
    constexpr int MN_KSTEP = THREADS / WPR;               // MN: k between a thread's words
    const int vk = KM ? 4 * (t & 15) : (t / WPR);         // k of the word within the stage
    const int vi = KM ? (t >> 4) : 4 * (t % WPR);         // row of the word within the tile
    int64_t vl = 0, voff = 0;                             // KM: the word's l; its tensor offset
    if (VEC) {
        if (KM) {
            vl = xl + vk;
            int64_t r = xr;
            while (vl >= L) { vl -= L; ++r; }
            voff = vl + L * (i0 + vi) + L * I * r;
        } else {
            voff = (kb + vk) * I + i0 + vi;
        }
    }
    const int64_t vstep = KM ? 16 * L : MN_KSTEP * I;     // offset between a thread's words
    const int64_t vwrap = L * (I - 1);                    // KM: end of row (i, r) -> (i, r + 1)

    auto issue_x = [&](int s, int slot) {
        float* dst = sm.pipe.xs[slot];
        const int64_t ks = kb + (int64_t)s * BK;
        const int kvalid = (ke - ks) < BK ? (int)(ke - ks) : BK;   // k of this stage in the range
        if (VEC) {
            if (KM) {
                const bool kval = vk < kvalid;
#pragma unroll
                for (int m = 0; m < XWORDS; ++m) {
                    const bool v = kval && vi + 16 * m < rows_left;
                    cp_async16(dst + (vi + 16 * m) * XPK + vk, p.X + (v ? voff + m * vstep : 0), v);
                }
                voff += BK;
                vl += BK;
                while (vl >= L) { vl -= L; voff += vwrap; }
            } else {
                const bool ival = vi < rows_left;
#pragma unroll
                for (int m = 0; m < XWORDS; ++m) {
                    const bool v = ival && vk + MN_KSTEP * m < kvalid;
                    cp_async16(dst + (vk + MN_KSTEP * m) * XPM + vi, p.X + (v ? voff + m * vstep : 0), v);
                }
                voff += (int64_t)BK * I;
            }
        } else {
            for (int e = t; e < BK * BI; e += THREADS) {
                int kk, ii;
                if (KM) { kk = e % BK; ii = e / BK; } else { ii = e % BI; kk = e / BI; }
                const int64_t i = i0 + ii;
                const bool valid = (kk < kvalid) && (ii < rows_left);
                int64_t off = 0;
                if (valid) {
                    if (L == 1) {
                        off = (ks + kk) * I;
                    } else {
                        int64_t l = xl + kk, r = xr;
                        while (l >= L) { l -= L; ++r; }
                        off = l + L * I * r;
                    }
                    off += L * i;
                }
                cp_async4(KM ? dst + ii * XPK + kk : dst + kk * XPM + ii, p.X + off, valid);
            }
        }
        cp_async_commit();
        if (!VEC && L > 1) { xl += BK; while (xl >= L) { xl -= L; ++xr; } }
    };

    // W stage s into ws[s & 1].  Thread t forms slot wcc = t % 32 (column group wcc / 16,
    // column wcc % 16 of it when below TC, else a zero pad) of rows kk = t / 32 + 8 m
    // (m = 0..7).  The factor entries of the next stage are loaded into registers before
    // the current stage's FMAs and multiplied by the tail scale Q(q, cc) and stored after
    // them, so their L2 latency is hidden.  The head has >= BK rows whenever there is a
    // tail, so a stage spans at most two q: rows kk < wlim of the stage have the stage's
    // first q, the others the next; the thread keeps Q(q, cc) for both in registers, formed
    // again only when q moves.
    const int wcc = t & (CB - 1), wk0 = t / CB;
    const int wsj = wcc & 15;
    const int wc = wsj < TC ? c0 + (wcc >> 4) * TC + wsj : C;     // C: a pad slot (zero)
    float wraw[WROWS];
    float q0 = 1.0f, q1 = 1.0f;
    int wlim = BK, wkval = BK;                   // rows before the q step; rows in the range
    // digits of q = wq over the tail factors (first fastest), kept by +1 steps: wq moves by
    // at most one per stage (the head has >= BK rows), so no division in the loop
    int qd[MTK_MAXN];
    if (W.ntail > 0) {
        int64_t rem = wq;
        for (int z = 0; z < W.ntail; ++z) {
            qd[z] = (int)(rem % W.tail_rad[z]);
            rem /= W.tail_rad[z];
        }
    }
    // Q(q, wc) from the digits of wq, or (next) of wq + 1: the digits below the first that
    // does not wrap are 0, that one is one more, the rest are wq's
    auto q_from = [&](bool next) -> float {
        float prod = 1.0f;
        bool carry = next;
        for (int z = 0; z < W.ntail; ++z) {
            int d = qd[z];
            if (carry) {
                if (++d < W.tail_rad[z]) carry = false;
                else d = 0;
            }
            prod *= __ldg(W.tail[z] + (int64_t)d * C + wc);
        }
        return prod;
    };
    // the factor entry of the thread's first row kk = wk0 of the stage, advanced with wd
    const float* wp0 = W.f0 + (wd + wk0) * C + (wc < C ? wc : 0);
    const int64_t wwrap = W.rad0 * C;
    auto load_w = [&](int s) {
        const int64_t ks = kb + (int64_t)s * BK;
        wkval = (ke - ks) < BK ? (int)(ke - ks) : BK;
        wlim = (W.ntail > 0 && W.rad0 - wd < BK) ? (int)(W.rad0 - wd) : BK;
        if (W.ntail > 0 && wq != qcached) {
            q0 = (wc < C && wq < qtot) ? q_from(false) : 0.0f;
            q1 = (wc < C && wq + 1 < qtot) ? q_from(true) : 0.0f;
            qcached = wq;
        }
#pragma unroll
        for (int m = 0; m < WROWS; ++m) {
            const int kk = wk0 + (THREADS / CB) * m;
            float w = 0.0f;
            if (kk < wkval && wc < C) {
                const float* ptr = wp0 + (THREADS / CB) * m * C;
                if (kk >= wlim) ptr -= wwrap;
                w = __ldg(ptr);
            }
            wraw[m] = w;
        }
    };
    auto store_w = [&](int s) {
        float* dst = &sm.pipe.ws[s & 1][0][0];
#pragma unroll
        for (int m = 0; m < WROWS; ++m) {
            const int kk = wk0 + (THREADS / CB) * m;
            float w = wraw[m];
            if (W.ntail > 0) w *= kk >= wlim ? q1 : q0;
            dst[kk * WP + wcc] = w;
        }
    };
    auto advance_w = [&]() {
        wd += BK;
        wp0 += BK * C;
        while (wd >= W.rad0) {
            wd -= W.rad0;
            ++wq;
            wp0 -= wwrap;
            for (int z = 0; z < W.ntail; ++z) {             // the digits of wq, +1
                if (++qd[z] < W.tail_rad[z]) break;
                qd[z] = 0;
            }
        }
    };

    float acc[RA][TC];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < TC; ++b) acc[a][b] = 0.0f;
    bool arow[RA];                       // row group a (rows ig + 16 a) has a row of the tensor
#pragma unroll
    for (int a = 0; a < RA; ++a) arow[a] = 16 * a < rows_left;

    int islot = 0;                       // ring slot of the next stage to issue
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nst) issue_x(s, islot); else cp_async_commit();
        islot = islot + 1 == STAGES ? 0 : islot + 1;
    }
    if (nst > 0) {
        load_w(0);
        store_w(0);
    }

    int cslot = 0;                       // ring slot of the stage being consumed
    for (int s = 0; s < nst; ++s) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        if (s + STAGES - 1 < nst) issue_x(s + STAGES - 1, islot); else cp_async_commit();
        islot = islot + 1 == STAGES ? 0 : islot + 1;
        // the next stage's factor entries, in flight during this stage's FMAs
        const bool more = s + 1 < nst;
        if (more) {
            advance_w();
            load_w(s + 1);
        }

        const float* xs = sm.pipe.xs[cslot];
        const float* ws = &sm.pipe.ws[s & 1][0][0];
        cslot = cslot + 1 == STAGES ? 0 : cslot + 1;
#pragma unroll
        for (int h = 0; h < KPG / 4; ++h) {
            float xv[RA][4];             // [row group a][k j of this half]
            if (KM) {
#pragma unroll
                for (int a = 0; a < RA; ++a) {
                    const float4 v = *reinterpret_cast<const float4*>(xs + (ig + 16 * a) * XPK + KPG * kg + 4 * h);
                    xv[a][0] = v.x; xv[a][1] = v.y; xv[a][2] = v.z; xv[a][3] = v.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int a = 0; a < RA; ++a) xv[a][j] = xs[(KPG * kg + 4 * h + j) * XPM + ig + 16 * a];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float* wr = ws + (KPG * kg + 4 * h + j) * WP + 16 * cg;
                float w[TC];
#pragma unroll
                for (int q = 0; q < TC / 4; ++q) {
                    const float4 w4 = *reinterpret_cast<const float4*>(wr + 4 * q);
                    w[4 * q] = w4.x; w[4 * q + 1] = w4.y; w[4 * q + 2] = w4.z; w[4 * q + 3] = w4.w;
                }
#pragma unroll
                for (int e = (TC / 4) * 4; e < TC; ++e) w[e] = wr[e];
#pragma unroll
                for (int a = 0; a < RA; ++a) {
                    // a row group past the last row of a ragged tile is skipped by the whole warp
                    if (!arow[a]) continue;
#pragma unroll
                    for (int b = 0; b < TC; ++b) acc[a][b] = fmaf(xv[a][j], w[b], acc[a][b]);
                }
            }
        }
        if (more) store_w(s + 1);
    }
    cp_async_wait<0>();
    __syncthreads();

    // fixed-order reduction over the k-groups: (g, g + 4), then (g, g + 2), then (0, 1)
    for (int half = NKG / 2; half >= 1; half >>= 1) {
        if (kg >= half && kg < 2 * half) {
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < TC; ++b) sm.red[kg - half][ig + 16 * a][16 * cg + b] = acc[a][b];
        }
        __syncthreads();
        if (kg < half) {
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < TC; ++b) acc[a][b] += sm.red[kg][ig + 16 * a][16 * cg + b];
        }
        __syncthreads();
    }
    if (kg == 0) {
#pragma unroll
        for (int a = 0; a < RA; ++a) {
            const int64_t i = i0 + ig + 16 * a;
            if (i >= I) continue;
#pragma unroll
            for (int b = 0; b < TC; ++b) {
                const int c = c0 + TC * cg + b;
                if (c >= C) continue;
                if (p.S == 1) p.out[i * p.out_si + c * p.out_sc] = acc[a][b];
                else p.part[((int64_t)sp * I + i) * C + c] = acc[a][b];
            }
        }
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

int simt_cta_cols(int C) { return 2 * (C <= 16 ? 8 : C <= 26 ? 13 : 16); }
// 64-row tiles, two CTAs per SM, for every I: 128-row tiles (RA = 8, one CTA per SM) were
// measured 1.03-1.24x slower on 200x200x300x40 and 512^3
int simt_tile_rows(int64_t) { return 64; }
int simt_ctas_per_sm(int64_t) { return 2; }

template <int TC, int RA>
cudaError_t launch_simt_ra(const ContractParams& p, dim3 grid, cudaStream_t s) {
    const bool km = p.L > 1;
    const bool xa = (reinterpret_cast<uintptr_t>(p.X) & 15) == 0 && p.kchunk % BK == 0;
    const size_t smem = sizeof(SimtSmem<RA>);
    auto go = [&](auto kernel) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kernel<<<grid, THREADS, smem, s>>>(p);
        return cudaSuccess;
    };
    if (km)
        return (xa && p.L % 4 == 0) ? go(contract_simt_kernel<true, true, TC, RA>)
                                    : go(contract_simt_kernel<true, false, TC, RA>);
    return (xa && p.I % 4 == 0) ? go(contract_simt_kernel<false, true, TC, RA>)
                                : go(contract_simt_kernel<false, false, TC, RA>);
}

template <int TC>
cudaError_t launch_simt_tc(const ContractParams& p, dim3 grid, cudaStream_t s) {
    return launch_simt_ra<TC, 4>(p, grid, s);
}

cudaError_t launch_contract_simt(const ContractParams& p, int c_blocks, int i_tiles,
                                 cudaStream_t s) {
    dim3 grid(i_tiles, p.S, c_blocks);
    const int cols = simt_cta_cols(p.C);
    if (c_blocks * cols < p.C) return cudaErrorInvalidValue;
    cudaError_t e = cols == 16 ? launch_simt_tc<8>(p, grid, s)
                  : cols == 26 ? launch_simt_tc<13>(p, grid, s)
                               : launch_simt_tc<16>(p, grid, s);
    note_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
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
