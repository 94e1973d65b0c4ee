// mtk_internal.cuh -- declarations shared by the libmttkrp translation units.
//
// Notation (Section 2.1 of the paper): for mode n of an N-way tensor,
// I^L = prod_{k<n} I_k, I^R = prod_{k>n} I_k.  Every contraction in this library
// is expressed on the 3-way view X3(l, i, r) = X[l + L*i + L*I*r] (L = I^L,
// I = I_n, R = I^R), which is exactly the natural layout (Section 2.1): the
// mode-n matricization is R contiguous row-major I x L blocks (Fig. 2).  The
// contraction index is k = l + L*r in [0, L*R), and the Khatri-Rao weight of
// k is W(k, c) = prod_z F_z(d_z(k), c), where d_z are the mixed-radix digits of
// k over the factor list (first factor fastest).  For mode n of a tensor the
// list is U_0..U_{n-1}, U_{n+1}..U_{N-1}, i.e. the rows of
// U_{N-1} kr ... kr U_{n+1} kr U_{n-1} kr ... kr U_0 (Section 2.2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "mttkrp.h"

#define MTK_MAXN 16
#define MTK_MAXC 256

namespace mtk {

// status word at the head of every workspace (first 256 bytes reserved)
constexpr size_t kStatusBytes = 256;

__device__ __forceinline__ void set_status(uint32_t* st, int code) {
    if (st) atomicOr(st, 1u << code);
}

// Khatri-Rao operand of a contraction, split as W(k,c) = F0(k % rad0, c) * Q(k / rad0, c)
// with Q(q, c) = prod_t tail[t](digit_t(q), c).  The host guarantees that either
// rad0 >= 32 or there is no tail (ntail == 0), so a block of 32 consecutive k
// meets at most two values of q.
struct KrpOperand {
    const float* f0;
    int64_t rad0;
    int ntail;
    const float* tail[MTK_MAXN];
    int64_t tail_rad[MTK_MAXN];
};

struct ContractParams {
    const float* X;
    int64_t L, I, R, K;    // view and contraction length K = L*R
    int C;                 // columns of W and of the output
    KrpOperand W;          // the operand as the FP32 kernel consumes it
    int nfac;              // the raw factor list (first factor = fastest digit of k)
    const float* fac[MTK_MAXN];
    int64_t frad[MTK_MAXN];
    int S;                 // number of contraction splits
    int64_t kchunk;        // split sp covers k in [sp*kchunk, min((sp+1)*kchunk, K))
    float* out;            // final output, element (i, c) at out[i*out_si + c*out_sc]
    int64_t out_si, out_sc;
    float* part;           // S x I x C partials when S > 1
    uint32_t* status;
    unsigned long long wait_ns;   // limit of the tensor-core kernels' abortable waits (0: 1 s)
    int stall;             // test hook: one wait that nothing completes (the kernel times out)
};

// host-side count of kernel launches issued by the library (monotonic, atomic)
void note_launches(int n);
// streaming multiprocessors of the current device (queried once per process)
int num_sms();

// ---- launchers (host side), defined in the .cu files -------------------------
cudaError_t launch_contract_simt(const ContractParams& p, int c_blocks, int i_tiles,
                                 cudaStream_t s);
int simt_cta_cols(int C);              // columns of M per CTA of the FP32 kernel (16, 26 or 32)
int simt_tile_rows(int64_t I);         // rows of M per CTA of the FP32 kernel (64 or 128)
int simt_ctas_per_sm(int64_t I);       // resident CTAs per SM of that kernel (2 or 1)
cudaError_t launch_split_reduce(const float* part, int S, int64_t I, int C, float* out,
                                int64_t si, int64_t sc, cudaStream_t s);
// Tensor-core contraction plan.  The factor list is split into a head (the first
// `head` factors, rad0 rows of their KRP, padded to rad0p = a multiple of 64) whose
// split BF16 image is the B operand, and a tail applied as a per-run column scale.
// The contraction runs over the padded index k' = q*rad0p + d0, Kp = (K/rad0)*rad0p.
// For small I (<= 64) with contiguous runs, U runs share the 128 MMA rows; each packed
// run offset writes its own partial slab (S * U slabs in all).
struct TcPlan {
    int head;
    int64_t rad0, rad0p, Kp, nruns;
    int BI, U, linear, CP, N;
    size_t image_bytes;
};
bool contract_tc_shape_ok(int64_t L, int64_t I, int C, int precision);
TcPlan contract_tc_plan(const int64_t* frad, int nfac, int64_t L, int64_t I, int C);
bool contract_tc_supported(const ContractParams& p, int precision);
// image: device scratch of plan.image_bytes (256-byte aligned)
cudaError_t launch_contract_tc(const ContractParams& p, int precision, void* image, cudaStream_t s);
// The B image alone: the KRP of the first `head` factors (rad0 rows, padded to rad0p, a
// multiple of 64) split into three BF16 pieces stacked along N = 3*CP, written as
// rad0p/64 slices, each the 128-byte-swizzled K-major shared-memory image of one 64-k
// stage (N rows x 128 bytes).
cudaError_t launch_tc_image(const float* const* fac, const int64_t* frad, int head, int C, int CP,
                            int64_t rad0, int64_t rad0p, void* image, cudaStream_t s);

// ---- tensor stored as two BF16 planes (contract_split.cu) --------------------------
// The planes hold the tensor with mode 0 padded to I0p = planes_rows0(I0), a multiple of 8
// (entries with i0 >= I0 are zero), so that every row of every mode-n view is 16-byte
// aligned: entry (i0, rest) at i0 + I0p rest.  NXp = I0p * (the other dims' product);
// hi = bf16_rn(x) at [0, NXp), lo = bf16_rn(x - hi) at [pitch, pitch + NXp),
// pitch = split_pitch(NXp) (a multiple of 64 entries).
int64_t planes_rows0(int64_t I0);
void planes_dims(const int64_t* dims, int N, int64_t* pd);   // dims with mode 0 padded
int64_t split_pitch(int64_t NXp);
int split_chunks(int64_t NXp);          // FP64 partials of ||X||^2 written by the split
// X: I0 x rest FP32 (natural order); part: split_chunks(NXp) doubles; normX2 (may be
// NULL): receives ||X||^2
cudaError_t launch_split_planes(const float* X, int64_t I0, int64_t rest, void* Xs, double* part,
                                double* normX2, cudaStream_t s);
// Plan of the planes contraction for view (L, I, R) and the mode's factor list; ok = 0
// when the shape is not taken (C > 64; MN-major: I_n not a multiple of 8; K-major: I^L
// not a multiple of 8 (the padded planes always have it); a head image above 32 MB, ...).
struct PlanesPlan {
    int ok, mn, head, spr, U, BI, MT, CP, N, ntiles, s_full, s_last, nslab, grid;
    int box_mode;             // packed runs: one TMA box per group (0) or for all (1: along r, 2: along lq)
    int sk;                   // stream-K over the (tile, stage) space (tall views)
    int64_t H, nruns, Lq, stot;
    int64_t gpr;              // box mode 2: packed groups per r when U does not divide Lq (else 0)
    size_t image_bytes, qtab_bytes, part_bytes;
};
PlanesPlan planes_plan(int64_t L, int64_t I, const int64_t* frad, int nfac, int C, int n_left, int ctas);
size_t planes_scratch_bytes(const PlanesPlan& pl);   // image + Q table + partials
int planes_ctas(int splits);           // CTAs of one launch (0 = one per SM)
// scratch: planes_scratch_bytes(pl) bytes, 256-byte aligned
// A factorisation to overlap with a planes contraction: H_n^{-1} of a CP-ALS update
// (launch_als_factor), launched between the contraction's prep and the contraction, which
// then starts at once (programmatic stream serialisation) on the SMs the plan left free and
// completes only after the factorisation has.
struct FactorHook {
    const double* const* G;
    int N, C, n;
    void* hinv;
    uint32_t* status;
};
// wait_ns: limit of the kernel's abortable waits (0: 1 s); stall: the timeout test hook.
// f0_rows: rows of fac[0] that exist (a padded mode 0 has frad[0] > f0_rows; the head
// image takes the rest as zero).  opad, oreal: row j of the view (I rows) is output row
// (j mod opad) + oreal (j / opad), dropped when j mod opad >= oreal (opad = 0: row j);
// the output has Iout = (I / opad) oreal rows.
cudaError_t launch_contract_planes(const void* Xs, int64_t pitch, int64_t L, int64_t I, int64_t R,
                                   const float* const* fac, const int64_t* frad, int nfac, int C,
                                   const PlanesPlan& pl, float* out, int64_t out_si, int64_t out_sc,
                                   void* scratch, uint32_t* status, cudaStream_t s,
                                   unsigned long long wait_ns, int stall, const FactorHook* hook,
                                   int64_t f0_rows, int64_t opad, int64_t oreal);

// ---- batched MTTKRPs in one persistent launch (batched.cu) --------------------------
typedef mtk_batch_problem BatchedProblem;
int batched_max_problems();
bool batched_plan_item(const int64_t* dims, int N, int n, int C, int64_t kchunk_target, int ctas,
                       int* ntiles, int* nchunks, int* kchunk, int* CB);
size_t batched_scratch_floats(const BatchedProblem* probs, int P, int64_t kchunk_target, int ctas);
// scratch: batched_scratch_floats(...) floats, 256-byte aligned
cudaError_t launch_batched(const BatchedProblem* probs, int P, int64_t kchunk_target, int ctas, float* scratch,
                           cudaStream_t s);

// ---- FP32 FMA throughput probe (probe.cu) ---------------------------------------------
cudaError_t launch_ffma_probe(int blocks, int iters, float* out, cudaStream_t s);
int ffma_probe_threads();

// ---- tensors symmetric in modes 0 and 1, packed (symmetric.cu) ----------------------
// diag = 1: the n0 (n0 + 1) / 2 entries a >= b; 0: the n0 (n0 - 1) / 2 entries a > b
int64_t sym_packed_rows(int64_t n0, int diag);      // rounded up to a multiple of 8
cudaError_t launch_sym_pack(const float* X, int64_t n0, int diag, int64_t rest, float* Xp, cudaStream_t s);
cudaError_t launch_sym_pair(const float* U0, const float* U1, int64_t n0, int diag, int C, float* W, cudaStream_t s);
cudaError_t launch_sym_ttv(const float* V, const float* U, int64_t n0, int diag, int C, float* M, cudaStream_t s);

cudaError_t launch_krp(const float* const* U, const int64_t* rows, int Z, int C, float* K,
                       int reuse, cudaStream_t s);
cudaError_t launch_multi_ttv(const float* T, int64_t L, int64_t I, int64_t R, const float* Ko,
                             int C, int right, float* M, cudaStream_t s);
// out(a, b, c) = sum_j T(a, j, b, c) K(j, c), c slowest (out_rowmajor: out[(a + A b) C + c])
cudaError_t launch_ttv_mode(const float* T, int64_t A, int64_t J, int64_t B, const float* K, int C, float* out,
                            int out_rowmajor, cudaStream_t s);
cudaError_t launch_gram(const float* U, int64_t I, int C, double* G, double* part,
                        int nchunks, cudaStream_t s);
int gram_chunks(int64_t I);
size_t solve_scratch_doubles(int C);   // Hbuf of launch_chol_solve
cudaError_t launch_chol_solve(const double* const* G, int N, int C, int n, const float* M,
                              int64_t In, float* Un, double* Hbuf, int* flag,
                              uint32_t* status, cudaStream_t s);
cudaError_t launch_norm2(const float* X, int64_t I, double* part, int nchunks, double* out,
                         cudaStream_t s);
int norm2_chunks(int64_t I);
// loss (may be NULL): 0.5 r2 as FP32
cudaError_t launch_residual(const double* normX2, const float* M, const float* U, int64_t I,
                            const double* const* G, int N, int C, double* r2, double* fit,
                            cudaStream_t s, float* loss = nullptr);
// factor update of a CP-ALS step in one launch (als_update.cu), C <= 64: U_n = M H^{-1}
// with H = Hadamard_{k != n} G_k (FP64 L D L^T and H^{-1}, formed before the kernel waits
// for M), and with Gn given the Gram of the new U_n, reduced in a fixed order and written
// to Gn, then with normX2 (and fit / r2) the fit.  Tickets: als_ticket_bytes() of zeros,
// left at zero.  programmatic: launched with programmatic stream serialisation (H and its
// inverse are formed while the previous kernel of the stream runs; M is read after that
// kernel completed).
struct AlsUpdateArgs {
    const double* const* G;
    int N, C, n;
    const float* M;
    int64_t In;
    float* Un;
    double* Gn;
    void* scratch;
    int Pmax;
    unsigned int* tickets;
    const double* normX2;
    double* fit;
    double* r2;
    uint32_t* status;
    bool programmatic;
    const void* hinv;          // H^{-1} from launch_als_factor (null: factored in the update)
    bool normalize;            // scale U_n (and G_n) to unit columns; not with the fit
};
bool als_update_supported(int C);
// H_n^{-1} (and its not-positive-definite flag) for a later update, in one CTA that
// triggers the next kernel of the stream at once (so a long kernel launched after it with
// programmatic stream serialisation can run meanwhile).  hinv: als_hinv_bytes(C) bytes.
size_t als_hinv_bytes(int C);
cudaError_t launch_als_factor(const double* const* G, int N, int C, int n, void* hinv, uint32_t* status,
                              cudaStream_t s);
size_t als_ticket_bytes();
int als_update_ctas(int64_t In, int64_t* rows);
int als_update_max_ctas(const int64_t* dims, int N);
size_t als_update_scratch_bytes(int Pmax, int C);
cudaError_t launch_als_update(const AlsUpdateArgs& a, cudaStream_t s);
// G_k = U_k^T U_k for k = 0..N-1 in one launch (C <= 64; same tickets)
size_t gram_all_scratch_bytes(const int64_t* I, int N, int C);
cudaError_t launch_gram_all(const float* const* U, const int64_t* I, int N, int C, double* const* G,
                            void* scratch, unsigned int* tickets, cudaStream_t s);
// Sum of squares of FP32 numbers with no FP64 arithmetic in the loop (an FP64 conversion
// and add every 16 entries kept this part's FP64 pipe 83% busy and made an HBM-bound pass
// 1.6x slower).  Each square is exact as p + e (p = x*x, e = fma(x, x, -p)); the p are
// summed with two-sum compensation in FP32 over at most 64 entries (flush()), and those
// partial sums go into a double-FP32 total by Dekker's addition (two-sum, then a fast
// two-sum renormalisation), about 2^-44 relative.  value() rounds the total to FP64 once.
struct SquareSum {
    float S = 0.0f, cmp = 0.0f, hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float pp = __fmul_rn(x, x);
        const float ee = fmaf(x, x, -pp);
        const float t = __fadd_rn(S, pp);
        const float z = __fsub_rn(t, S);
        cmp = __fadd_rn(cmp, __fadd_rn(__fadd_rn(__fsub_rn(S, __fsub_rn(t, z)), __fsub_rn(pp, z)), ee));
        S = t;
    }
    __device__ __forceinline__ void flush() {
        const float s = __fadd_rn(hi, S);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(S, bb));
        const float t = __fadd_rn(__fadd_rn(e, lo), cmp);
        hi = __fadd_rn(s, t);                       // |s| >= |t|: every term is >= 0 or tiny
        lo = __fsub_rn(t, __fsub_rn(hi, s));
        S = 0.0f;
        cmp = 0.0f;
    }
    __device__ __forceinline__ double value() {
        flush();
        return (double)hi + (double)lo;
    }
};

// a kernel that the next kernel of its stream may overlap (programmatic dependent launch)
__device__ __forceinline__ void allow_dependent_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
cudaError_t launch_gradient(const float* U, const float* M, const double* const* G, int N, int C,
                            int n, int64_t In, const float* scale, float* grad, cudaStream_t s);

}  // namespace mtk
