/*
 * mttkrp.h -- C ABI of libmttkrp, dense MTTKRP and CP-ALS on one GB300 GPU.
 *
 * Follows "Shared-Memory Parallelization of MTTKRP for Dense Tensors"
 * (Hayashi, Ballard, Jiang, Tobia, 2017).  Conventions used by every call:
 *
 *  - Indices are 0-based (Section 2.1).  A tensor with dims I_0..I_{N-1} is a
 *    dense FP32 array in the natural linearization l = sum_k i_k prod_{j<k} I_j,
 *    mode 0 fastest (Section 2.1).  It is never reordered in memory.
 *  - Factor matrices U_k are I_k x C FP32, row-major (C contiguous).  MTTKRP
 *    outputs M are I_n x C FP32 row-major.  (The paper leaves the factor layout
 *    open; this library fixes it.)
 *  - Every float / double pointer argument is a DEVICE pointer unless stated.
 *    Arrays of pointers (U, G) are HOST arrays whose elements are device
 *    pointers.  dims / rows arrays are HOST arrays.
 *  - The caller owns all memory, including the workspace `ws`; the library
 *    allocates no device memory.  Workspace sizes come from the *_workspace
 *    queries.  The first 256 bytes of every workspace hold the device status
 *    word; zero them once (mtk_clear_status) before first use.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL
 *    is the legacy default stream).  Host-detectable errors return at once with
 *    no launch.  Errors found on the device (a non-positive-definite normal
 *    matrix, an expired wait) are OR-ed into the status word and read back by
 *    mtk_read_status.
 *  - N <= 16, 1 <= C <= 256, every dim >= 1, every product of dims < 2^62.
 *    Device pointers must be 4-byte aligned; 16-byte alignment enables the
 *    vectorised and tensor-core paths.
 *  - Functions are reentrant; the only global state is a monotonic, atomic
 *    count of the kernel launches issued (mtk_launch_count).
 */
#ifndef MTTKRP_H
#define MTTKRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (return values and bits of the device status word) */
typedef enum {
    MTK_OK = 0,
    MTK_EINVAL = 1,        /* bad argument (null pointer, bad size, misalignment) */
    MTK_ECUDA = 3,         /* a CUDA launch or copy failed */
    MTK_ENOTPD = 4,        /* normal-equation matrix not positive definite */
    MTK_ETIMEOUT = 5,      /* a bounded device-side wait expired */
    MTK_EUNSUPPORTED = 6,  /* option not available for this shape */
    MTK_EWORKSPACE = 7     /* workspace too small */
} mtk_status;

/* MTTKRP algorithm (Section 4) */
enum {
    MTK_ALGO_AUTO = 0,          /* per-mode choice made by the library */
    MTK_ALGO_FUSED = 1,         /* 1-step, KRP rows generated on chip, never stored */
    MTK_ALGO_MATERIALIZED = 2,  /* 1-step with the full KRP written to the workspace
                                   (Algorithm 2) */
    MTK_ALGO_TWO_STEP = 3       /* partial MTTKRP + multi-TTV (Algorithm 4); at the
                                   external modes it is the 1-step algorithm */
};

/* arithmetic of the tensor contraction */
enum {
    MTK_PREC_AUTO = 0,          /* currently MTK_PREC_FP32 */
    MTK_PREC_FP32 = 1,          /* FP32 fused multiply-adds on the CUDA cores */
    MTK_PREC_BF16X2 = 2,        /* tensor entries as 2 BF16 pieces, KRP entries as 3,
                                   all 6 cross products on tcgen05, FP32 accumulate */
    MTK_PREC_BF16X3 = 3         /* tensor entries as 3 BF16 pieces (9 products) */
};

typedef struct {
    int algo;          /* MTK_ALGO_* */
    int precision;     /* MTK_PREC_* */
    int splits;        /* contraction splits across CTAs; 0 = automatic */
    int wait_us;       /* limit of each device-side wait of the tensor-core contraction
                          kernels, in microseconds; 0 = 1 second.  A wait that runs out
                          sets MTK_ETIMEOUT in the status word; the kernel then lets the
                          copies and MMAs it has started finish and returns. */
    int test_stall;    /* 0 in normal use.  1 (a test of the timeout path): the tensor-core
                          contraction kernel first waits on a barrier that nothing
                          completes, so that this wait runs out after wait_us and the call
                          reports MTK_ETIMEOUT (the output is not valid then). */
    int normalize;     /* CP-ALS sweeps only.  1: after its update, every factor but the
                          last is scaled to unit 2-norm columns (its Gram with it); the
                          last factor then carries the weights, so [[U_0, ..., U_{N-1}]]
                          is the model without a separate lambda, and the sweep's result
                          is the same model as without the scaling (ALS is equivariant
                          under column scaling).  Needs C <= 64 (else MTK_EUNSUPPORTED).
                          0: no scaling (the paper's sweep). */
    int reserved[2];   /* set to 0 */
} mtk_opts;            /* NULL = all defaults */

/* status helpers --------------------------------------------------------- */
const char* mtk_status_string(int status);
int mtk_version(void);

/* Number of CUDA kernel launches this library has issued in this process
 * (all threads, all devices).  Differences around a region count its launches. */
uint64_t mtk_launch_count(void);

/* Zero the status word at the head of a workspace (async on stream). */
int mtk_clear_status(void* ws, void* stream);

/* Synchronise `stream`, then return the status word of `ws` (MTK_OK if
   nothing was recorded).  *bits_out (host, may be NULL) gets the raw bits. */
int mtk_read_status(const void* ws, void* stream, uint32_t* bits_out);

/* Khatri-Rao product (Section 4.1, Algorithm 1) ---------------------------
 * K = U_0 kr U_1 kr ... kr U_{Z-1}: the row of K for row indices
 * (a_0, ..., a_{Z-1}) is U_0(a_0,:) * ... * U_{Z-1}(a_{Z-1},:), with the LAST
 * operand's index fastest (Section 2.1 row rule).  U: host array of Z device
 * pointers to rows[z] x C row-major matrices.  K: device, (prod rows) x C
 * row-major, overwritten.  reuse = 1 shares each prefix product across the
 * rows that follow it (Algorithm 1); reuse = 0 forms every row from scratch
 * (the naive comparator of Section 5.2).  Z in [1, 16]. */
int mtk_khatri_rao(const float* const* U, const int64_t* rows, int Z, int C,
                   float* K, int reuse, void* stream);

/* MTTKRP (Section 2.2; Algorithms 2-4) ----------------------------------
 *   M(i_n, c) = sum_{all i_k, k != n} X(i_0..i_{N-1}) prod_{k != n} U_k(i_k, c)
 * i.e. M = X_(n) (U_{N-1} kr ... kr U_{n+1} kr U_{n-1} kr ... kr U_0).
 * X: device tensor (natural order).  dims: host, N entries.  U: host array of
 * N device pointers (U[n] is not read, may be NULL).  M: device I_n x C,
 * overwritten.  ws/ws_bytes: device workspace of at least
 * mtk_mttkrp_workspace(...) bytes.  The result does not depend on the launch
 * order of CTAs (fixed-order reduction). */
size_t mtk_mttkrp_workspace(const int64_t* dims, int N, int C, int n, const mtk_opts* opts);
int mtk_mttkrp(const float* X, const int64_t* dims, int N, const float* const* U, int C,
               int n, float* M, void* ws, size_t ws_bytes, const mtk_opts* opts,
               void* stream);

/* MTTKRP that allocates nothing (the paper has no counterpart: an interface for
 * callers that cannot allocate device memory).  Same operation, arguments and
 * results as mtk_mttkrp, but the workspace is a fixed device array of
 * MTK_NOALLOC_SCRATCH_BYTES bytes inside the library; no cudaMalloc, cudaFree
 * or allocating library routine is called.
 *  - The first call on a device (the current device) looks up that device's
 *    copy of the array; make that first call before any stream capture.  The
 *    lookup is repeated when the device's context has changed since (after
 *    cudaDeviceReset the module, and so the array, is loaded again).
 *  - Every call on a device shares the one array, which keeps the previous
 *    call's contents (the status word is cleared at the start of each call).
 *    Calls whose work overlaps on the GPU (other streams, other host threads)
 *    race on it: order them on one stream or serialise them.
 *  - Returns MTK_EWORKSPACE, before any launch and with M untouched, when the
 *    shape and options need more than MTK_NOALLOC_SCRATCH_BYTES of workspace
 *    (mtk_mttkrp_workspace(...) tells).
 *  - status_bits (host, may be NULL): if given, the call synchronises the
 *    stream, stores the device status bits there and returns the lowest
 *    recorded code, as mtk_read_status does; if NULL nothing is synchronised. */
#define MTK_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int mtk_mttkrp_noalloc(const float* X, const int64_t* dims, int N, const float* const* U,
                       int C, int n, float* M, const mtk_opts* opts, uint32_t* status_bits,
                       void* stream);

/* Tensor stored as two BF16 planes (Section 2.2: CP-ALS runs an MTTKRP for every mode
 * of every sweep on the same tensor, so the tensor can be prepared once) ----------
 * The split: hi = bf16_rn(x), lo = bf16_rn(x - hi) for every entry x (two-piece split
 * of Henry, Tang and Heinecke, ARITH 2019; |x - hi - lo| <= 2^-16 |x|).  The planes keep
 * the natural linearization with mode 0 padded to I0p = mtk_split_rows0(dims[0]), the
 * next multiple of 8: entry (i0, i1, ..., i_{N-1}) sits at i0 + I0p (i1 + I1 (i2 + ...)),
 * and the entries with i0 >= I0 are zero.  Every row of every mode's matricization then
 * starts on a 16-byte boundary, which the tensor-core loads need.  Xs holds hi at entries
 * [0, NXp) and lo at [pitch, pitch + NXp), NXp = I0p prod(dims[1..N-1]),
 * pitch = mtk_split_pitch(dims, N) (NXp rounded up to 64), as 16-bit BF16 words:
 * mtk_split_bytes(dims, N) bytes in all, the size of the FP32 tensor when I0 is a
 * multiple of 8.  Xs: device, 16-byte aligned, caller-owned.  normX2 (device double, may
 * be NULL) receives ||X||^2 from the same pass (exact squares, compensated FP32 sums of 64
 * entries added in FP64, fixed order).  ws: at least mtk_split_workspace(dims, N) bytes.
 * X: device memory, or pinned (page-locked) host memory, which the split reads in place
 * through its mapping into the device address space: the transfer from the host and the
 * split are then one pass, and the FP32 tensor never occupies device memory.  Pageable
 * host memory: MTK_EINVAL.
 * Bad dims (N outside 1..8, a dim < 1, more than 2^46 padded entries): the size queries
 * return 0 and the split MTK_EINVAL. */
int64_t mtk_split_rows0(int64_t I0);
int64_t mtk_split_pitch(const int64_t* dims, int N);
size_t mtk_split_bytes(const int64_t* dims, int N);
size_t mtk_split_workspace(const int64_t* dims, int N);
int mtk_split_tensor(const float* X, const int64_t* dims, int N, void* Xs, double* normX2, void* ws,
                     size_t ws_bytes, void* stream);

/* MTTKRP on the planes (the same operation as mtk_mttkrp, tensor entries carried as
 * hi + lo, KRP entries as three BF16 pieces, all six cross products on tcgen05 with
 * FP32 accumulation: the accuracy of MTK_PREC_BF16X2).  The tensor is read through TMA
 * straight into the tensor-core operand, 4 bytes per entry.  Xs: from
 * mtk_split_tensor for a tensor with these dims.  X (device, may be NULL): the FP32
 * tensor, used only for shapes the planes kernel does not take (C > 64, a head KRP
 * image above 32 MB, index ranges above 2^31), which then run mtk_mttkrp with
 * MTK_PREC_BF16X2; with X NULL such shapes return MTK_EUNSUPPORTED.  opts: algo AUTO or FUSED, precision AUTO or
 * BF16X2, splits = CTAs of the launch (0: one per SM); else MTK_EINVAL.  ws: at least
 * mtk_mttkrp_split_workspace(...) bytes. */
size_t mtk_mttkrp_split_workspace(const int64_t* dims, int N, int C, int n, const mtk_opts* opts);
int mtk_mttkrp_split(const void* Xs, const float* X, const int64_t* dims, int N, const float* const* U,
                     int C, int n, float* M, void* ws, size_t ws_bytes, const mtk_opts* opts,
                     void* stream);

/* Every mode's MTTKRP with the same factors, on the planes (the gradient of the CP loss,
 * Section 2.2, needs all N of them).  M[n] (device, I_n x C row-major) receives the
 * mode-n MTTKRP for n = 0..N-1.  With opts->algo AUTO or TWO_STEP this runs the dimension
 * tree of Algorithm 4: the partial contraction over modes >= 2 (one pass over the tensor)
 * and multi-TTVs give M[0] and M[1]; the contraction over modes 0, 1 (N >= 4; for N >= 5
 * while 4 C <= I_0 I_1) or the mode-2 MTTKRP (N = 3) gives the rest, through multi-TTVs
 * or one-mode contractions of that partial, so the tensor is read twice instead of N
 * times.  FUSED, or shapes outside those: N planes MTTKRPs.  Xs: from mtk_split_tensor; every mode must
 * be one the planes kernel takes (else MTK_EUNSUPPORTED and a workspace query of 0).
 * opts: precision AUTO or BF16X2; algo AUTO, FUSED or TWO_STEP.  ws: at least
 * mtk_mttkrp_all_split_workspace(...) bytes. */
size_t mtk_mttkrp_all_split_workspace(const int64_t* dims, int N, int C, const mtk_opts* opts);
int mtk_mttkrp_all_split(const void* Xs, const int64_t* dims, int N, const float* const* U, int C,
                         float* const* M, void* ws, size_t ws_bytes, const mtk_opts* opts, void* stream);

/* FP32 FMA throughput probe: the ceiling of the plain-FP32 contraction ------------------
 * mtk_ffma_probe launches ctas_per_sm CTAs per SM of 256 threads, each thread running 8
 * independent FMA chains of `iters` steps, and stores one float per thread into `out`
 * (device, mtk_ffma_probe_out_floats(ctas_per_sm) floats).  *flops (host, may be null)
 * receives the floating-point operations it performs (2 per FMA).  The caller times the
 * launch (CUDA events on `stream`): flops / time is the device's FP32 FMA throughput.
 * ctas_per_sm in [1, 64], iters in [1, 2^24], else MTK_EINVAL. */
int64_t mtk_ffma_probe_out_floats(int ctas_per_sm);
int mtk_ffma_probe(int ctas_per_sm, int iters, float* out, double* flops, void* stream);

/* Tensors symmetric in modes 0 and 1, stored packed (Section 5.3.3: the fMRI tensor's
 * pair of region modes kept as one mode of the entries of one triangle) ----------------
 * dims[0] = dims[1] = n0; r is the flat index of modes 2..N-1 (natural order).
 * diag = 1: the entry X(a, b, r) with a >= b is kept at Xp[p + Pp r], p = a (a + 1) / 2 + b
 * (n0 (n0 + 1) / 2 rows).  diag = 0 (the paper's layout: 200 regions -> 19,900 rows): only
 * a > b, p = a (a - 1) / 2 + b (n0 (n0 - 1) / 2 rows), and the tensor is taken to be zero
 * on its diagonal a = b.  Pp = mtk_sym_packed_rows(n0, diag) is the row count rounded up to
 * a multiple of 8, or of 64 from 2048 rows on; the padding rows hold zeros.  The packed tensor has about half the
 * entries of the full one.
 * mtk_pack_symmetric: Xp (device, Pp * prod(dims[2..N-1]) floats) from the full tensor X
 * (device, natural order); only the entries with a >= b (a > b) are read: the tensor is
 * taken to be symmetric in modes 0, 1.  N >= 3, dims[0] == dims[1], diag 0 or 1, else
 * MTK_EINVAL.
 * mtk_mttkrp_sym_split: the mode-n MTTKRP of the full tensor (the same M as mtk_mttkrp on it,
 * with its diagonal zeroed for diag = 0) from the BF16 planes of its packed form
 * (mtk_split_tensor of Xp, mtk_split_bytes of Pp * prod(dims[2..]) entries).  Modes n >= 2
 * run the planes MTTKRP of the packed tensor with a first factor
 * W(p(a, b), c) = U_0(a, c) U_1(b, c) + U_0(b, c) U_1(a, c) (a > b), U_0(a, c) U_1(a, c)
 * (a = b); modes 0 and 1 run its mode-0 MTTKRP V and then
 * M(a, c) = sum_b V(p(max(a, b), min(a, b)), c) U_other(b, c) (b != a for diag = 0).
 * dims: the full tensor's; U as for mtk_mttkrp (U[n] may be null); opts as for
 * mtk_mttkrp_split; shapes the planes kernel does not take give MTK_EUNSUPPORTED (the
 * workspace query then returns 0).  ws: at least mtk_mttkrp_sym_split_workspace(...) bytes. */
int64_t mtk_sym_packed_rows(int64_t n0, int diag);
int mtk_pack_symmetric(const float* X, const int64_t* dims, int N, int diag, float* Xp, void* stream);
size_t mtk_mttkrp_sym_split_workspace(const int64_t* dims, int N, int diag, int C, int n, const mtk_opts* opts);
int mtk_mttkrp_sym_split(const void* Xps, const int64_t* dims, int N, int diag, const float* const* U, int C, int n,
                         float* M, void* ws, size_t ws_bytes, const mtk_opts* opts, void* stream);

/* Batched MTTKRPs (Section 2.2) in one persistent launch ---------------------
 * P independent problems, each one mode-n MTTKRP of its own tensor, all computed by one
 * persistent kernel (plus one reduce launch), so that a batch of many small, uneven
 * tensors costs two launches and can be captured in a CUDA graph.  FP32 fused
 * multiply-adds on the CUDA cores, FP32 accumulation, fixed-order reductions (the
 * result does not depend on scheduling).  Any dims (no alignment needed).
 * Limits: P <= MTK_BATCH_MAXP, N in [2, MTK_BATCH_MAXN], C in [1, 32], and the
 * contraction length prod_{k != n} dims[k] < 2^31; otherwise MTK_EINVAL.
 * opts->splits: contraction indices per work unit (0 = automatic; the autotuner of the
 * Python binding picks it by timing); algo and precision are ignored.
 * ws: device, at least mtk_mttkrp_batched_workspace(...) bytes (first 256: status). */
#define MTK_BATCH_MAXN 4
#define MTK_BATCH_MAXP 192
typedef struct {
    const float* X;                    /* device tensor, natural order */
    const float* U[MTK_BATCH_MAXN];    /* device factors, U[k] is dims[k] x C (U[n] not read) */
    int64_t dims[MTK_BATCH_MAXN];
    int N;                             /* order of this tensor */
    int n;                             /* mode */
    int C;                             /* rank */
    float* M;                          /* device output, dims[n] x C, overwritten */
} mtk_batch_problem;
size_t mtk_mttkrp_batched_workspace(const mtk_batch_problem* probs, int P, const mtk_opts* opts);
int mtk_mttkrp_batched(const mtk_batch_problem* probs, int P, void* ws, size_t ws_bytes, const mtk_opts* opts,
                       void* stream);

/* 2-step pieces (Section 4.3, Algorithm 4) -------------------------------
 * Partial MTTKRP.  right = 1: T = X_(0:n) K_R, K_R = U_{N-1} kr ... kr U_{n+1}
 * (R = prod_{k>n} I_k rows); T is the (I^L x I_n x C) tensor R of the paper in
 * natural order, T[l + I^L i + I^L I_n c].  right = 0: T = X_(0:n-1)^T K_L,
 * K_L = U_{n-1} kr ... kr U_0 (I^L rows); T[i + I_n r + I_n I^R c].
 * Kp: device, the materialised partial KRP (row-major, C columns), e.g. from
 * mtk_khatri_rao.  T: device, overwritten. */
size_t mtk_partial_mttkrp_workspace(const int64_t* dims, int N, int C, int n, int right,
                                    const mtk_opts* opts);
int mtk_partial_mttkrp(const float* X, const int64_t* dims, int N, const float* Kp, int C,
                       int n, int right, float* T, void* ws, size_t ws_bytes,
                       const mtk_opts* opts, void* stream);

/* The same partial MTTKRP on the tensor's BF16 planes (Section 4.3, Algorithm 4, first
 * step; the accuracy of mtk_mttkrp_split).  The partial KRP is not materialised: U is a
 * host array of N device pointers to the factors (row-major dims[k] x C; only the
 * factors on the contracted side are read: k > n for right = 1, k < n for right = 0),
 * and the contraction forms it on chip.  T has the layout of mtk_partial_mttkrp.  This
 * is the contraction that the dimension tree of mtk_cp_als_sweep_split runs (n = 1
 * right, n = 2 left).  Requirements: right = 1 needs n < N-1, right = 0 needs n > 0
 * (else MTK_EINVAL); C <= 64 and the shapes the planes kernel takes (right: I^L I_n a
 * multiple of 8; left: I^L a multiple of 8), else MTK_EUNSUPPORTED (the workspace query
 * then returns 0).  Xs: from mtk_split_tensor, 16-byte aligned.  opts: as for
 * mtk_mttkrp_split.  ws: at least mtk_partial_mttkrp_split_workspace(...) bytes. */
size_t mtk_partial_mttkrp_split_workspace(const int64_t* dims, int N, int C, int n, int right,
                                          const mtk_opts* opts);
int mtk_partial_mttkrp_split(const void* Xs, const int64_t* dims, int N, const float* const* U,
                             int C, int n, int right, float* T, void* ws, size_t ws_bytes,
                             const mtk_opts* opts, void* stream);

/* Multi-TTV, the second step.  right = 1: M(i,c) = sum_l T[l + I^L i + I^L I_n c] K_L(l,c);
 * right = 0: M(i,c) = sum_r T[i + I_n r + I_n I^R c] K_R(r,c).  Ko: device, the other
 * partial KRP (K_L for right, K_R for left), row-major.  M: device I_n x C. */
int mtk_multi_ttv(const float* T, const int64_t* dims, int N, const float* Ko, int C, int n,
                  int right, float* M, void* stream);

/* Gram matrices and the normal-equation solve (Section 2.2) -------------
 * G = U^T U for an I x C FP32 matrix, accumulated in FP64; G: device C x C
 * FP64 row-major.  ws: at least mtk_gram_workspace(I, C) bytes. */
size_t mtk_gram_workspace(int64_t I, int C);
int mtk_gram(const float* U, int64_t I, int C, double* G, void* ws, size_t ws_bytes,
             void* stream);

/* U_n = M H^{-1} with H = Hadamard_{k != n} G_k (FP64 Cholesky).  G: host array of
 * N device pointers to C x C FP64 Grams (G[n] not read).  M: device In x C FP32.
 * Un: device In x C FP32, written only if H is positive definite; otherwise
 * left unchanged and MTK_ENOTPD is OR-ed into the status word.  Gn (device,
 * may be NULL): receives Un^T Un of the result (FP64).  ws: at least
 * mtk_solve_workspace(In, C) bytes. */
size_t mtk_solve_workspace(int64_t In, int C);
int mtk_gram_hadamard_solve(const double* const* G, int N, int C, int n, const float* M,
                            int64_t In, float* Un, double* Gn, void* ws, size_t ws_bytes,
                            void* stream);

/* ||X||^2 in FP64 (fixed-order reduction).  out: device double. */
size_t mtk_norm2_workspace(int64_t I);
int mtk_norm2(const float* X, int64_t I, double* out, void* ws, size_t ws_bytes, void* stream);

/* One CP-ALS sweep (Section 2.2): for n = 0..N-1, M = MTTKRP(X, n),
 * H = Hadamard_{k != n} U_k^T U_k, U_n = M H^{-1}, the other factors fixed at
 * their latest values.  U: host array of N device pointers, updated in place.
 * normX2 (device, may be NULL): ||X||^2 from mtk_norm2; if given with fit
 * (device, may be NULL), *fit = 1 - sqrt(max(0, ||X||^2 - 2<M_{N-1}, U_{N-1}> +
 * sum(Hadamard_k G_k))) / ||X||.  No host synchronisation inside. */
size_t mtk_cp_als_workspace(const int64_t* dims, int N, int C, const mtk_opts* opts);
int mtk_cp_als_sweep(const float* X, const int64_t* dims, int N, float* const* U, int C,
                     const double* normX2, double* fit, void* ws, size_t ws_bytes,
                     const mtk_opts* opts, void* stream);

/* The same sweep with every MTTKRP on the tensor's BF16 planes (mtk_mttkrp_split).
 * Xs: from mtk_split_tensor.  X: the FP32 tensor or NULL (see mtk_mttkrp_split); device
 * or pinned host memory (read in place, for the modes the planes do not take).  opts
 * as for mtk_mttkrp_split, and algo MTK_ALGO_TWO_STEP selects the dimension tree for
 * N = 3 or 4 (Section 6 of the paper, reuse of partial MTTKRPs across modes): the partial
 * contraction over modes >= 2 serves the updates of U_0 and U_1, the one over modes 0 and
 * 1 (with the updated U_0, U_1) those of U_2 and U_3; each per-mode MTTKRP then follows by
 * a multi-TTV (Algorithm 4).  The tensor is read twice per sweep instead of N times; the
 * updates are the same Gauss-Seidel sequence.  Shapes the tree does not take run the
 * per-mode sweep.  ws: mtk_cp_als_workspace(...) bytes (it covers every form). */
int mtk_cp_als_sweep_split(const void* Xs, const float* X, const int64_t* dims, int N, float* const* U,
                           int C, const double* normX2, double* fit, void* ws, size_t ws_bytes,
                           const mtk_opts* opts, void* stream);

/* CP loss pieces (Section 2.2; the paper names the residual as a cost but gives
 * no formula, this is the standard expansion of the squared norm):
 *   r2 = ||X||^2 - 2 <M_m, U_m> + sum_{a,b} prod_k G_k(a,b),   G_k = U_k^T U_k,
 * which equals ||X - [[U_0..U_{N-1}]]||^2 when M_m is the mode-m MTTKRP of X.
 * normX2: device double (mtk_norm2).  M, Um: device Im x C.  G: host array of N
 * device pointers to FP64 Grams.  r2, fit: device doubles, either may be NULL;
 * fit = 1 - sqrt(max(0, r2)) / ||X||. */
int mtk_cp_residual(const double* normX2, const float* M, const float* Um, int64_t Im,
                    const double* const* G, int N, int C, double* r2, double* fit, void* stream);

/* The CP least-squares loss f = 0.5 ||X - [[U_0..U_{N-1}]]||^2 (Section 2.2's model),
 * from the same identity as mtk_cp_residual: f = 0.5 r2.  loss: device float (the FP64
 * value rounded once).  Other arguments as for mtk_cp_residual. */
int mtk_cp_loss(const double* normX2, const float* M, const float* Um, int64_t Im,
                const double* const* G, int N, int C, float* loss, void* stream);

/* Gradient of f = 0.5 ||X - [[U]]||^2 with respect to U_n (MTTKRP is part of the
 * gradient, Section 2.2):  grad = scale * (U_n H_n - M_n), H_n = Hadamard_{k != n} G_k.
 * Un, Mn: device In x C FP32 (Mn = mode-n MTTKRP).  G: host array of N device
 * pointers (G[n] not read).  scale: device float, may be NULL (= 1).  grad: device
 * In x C FP32, may alias neither input. */
int mtk_cp_gradient(const float* Un, const float* Mn, const double* const* G, int N, int C, int n,
                    int64_t In, const float* scale, float* grad, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MTTKRP_H */
