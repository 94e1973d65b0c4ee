// api.cu -- the extern "C" entry points declared in include/mttkrp.h: argument
// checks, workspace layout and the choice of kernels.  No device memory is
// allocated here; every buffer comes from the caller.
#include <cuda.h>
#include <string.h>

#include "mtk_internal.cuh"

#include <atomic>
#include <mutex>

// Device scratch of mtk_mttkrp_noalloc: one fixed array per device, part of the
// module, so that entry point needs no allocation.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MTK_NOALLOC_SCRATCH_BYTES];

using namespace mtk;

namespace mtk {
static std::atomic<unsigned long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

// With no device to ask (a workspace query on a host without a GPU) the count of the
// GB300 the library is built for stands in, so that host-side sizes match that GPU's.
int num_sms() {
    constexpr int kGb300Sms = 152;
    static int n = []() {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return kGb300Sms;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return kGb300Sms;
        return v;
    }();
    return n;
}
}  // namespace mtk

namespace {

constexpr int kBK = 64;           // the W operand needs rad0 >= kBK (or no tail factors)
constexpr int kTcBK = 64;         // k per tensor-core stage; tensor-core splits are multiples
constexpr int kNoAllocMaxDevices = 64;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Identity of the CUDA context current on this thread (0 if none or unavailable):
// cuCtxGetCurrent + cuCtxGetId, reached through the runtime.  Context ids are never
// reused within a process, so an id that changes means the module (and its static
// device arrays) was loaded again, e.g. after cudaDeviceReset.
unsigned long long current_context_id() {
    typedef CUresult (*GetCurrentFn)(CUcontext*);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
    static GetCurrentFn get_current = []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (GetCurrentFn) nullptr;
        return reinterpret_cast<GetCurrentFn>(p);
    }();
    static GetIdFn get_id = []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (GetIdFn) nullptr;
        return reinterpret_cast<GetIdFn>(p);
    }();
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

struct Carve {                    // bump allocator over a caller workspace
    char* base;
    size_t off, cap;
    void* take(size_t bytes) {
        off = align256(off);
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

mtk_opts defaults(const mtk_opts* o) {
    mtk_opts d;
    memset(&d, 0, sizeof(d));
    if (o) d = *o;
    if (d.algo < MTK_ALGO_AUTO || d.algo > MTK_ALGO_TWO_STEP) d.algo = -1;
    if (d.precision == MTK_PREC_AUTO) d.precision = MTK_PREC_FP32;
    return d;
}

bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }

// The tensor as the kernels address it: device memory as it is; pinned host memory through
// its mapping into the device address space, so that a kernel reads it over the host link
// in the same pass that uses it; pageable host memory is refused (MTK_EINVAL)
int device_view(const float* X, const float** out) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, X) != cudaSuccess) {
        cudaGetLastError();
        return MTK_ECUDA;
    }
    if (a.type == cudaMemoryTypeUnregistered) return MTK_EINVAL;
    if (a.type == cudaMemoryTypeHost) {
        if (!a.devicePointer) return MTK_EINVAL;
        *out = static_cast<const float*>(a.devicePointer);
        return MTK_OK;
    }
    *out = X;
    return MTK_OK;
}

// limit of the contraction kernels' abortable device waits (0: the kernels' 1 s default)
unsigned long long wait_limit_ns(const mtk_opts& o) {
    return o.wait_us > 0 ? (unsigned long long)o.wait_us * 1000ull : 0ull;
}

int check_shape(const int64_t* dims, int N, int C, int n) {
    if (!dims || N < 2 || N > MTK_MAXN || C < 1 || C > MTK_MAXC || n < 0 || n >= N)
        return MTK_EINVAL;
    int64_t p = 1;
    for (int k = 0; k < N; ++k) {
        if (dims[k] < 1) return MTK_EINVAL;
        if (p > ((int64_t)1 << 62) / dims[k]) return MTK_EINVAL;
        p *= dims[k];
    }
    if (p > ((int64_t)1 << 62) / C) return MTK_EINVAL;
    return MTK_OK;
}

struct View { int64_t L, I, R; };

View mode_view(const int64_t* dims, int N, int n) {
    View v{1, dims[n], 1};
    for (int k = 0; k < n; ++k) v.L *= dims[k];
    for (int k = n + 1; k < N; ++k) v.R *= dims[k];
    return v;
}

// --- contraction planning --------------------------------------------------
struct ContractPlan {
    int tc;                 // use the tensor-core kernel
    int S, i_tiles, c_blocks;
    int slabs;              // partial slabs summed by the split reduce (S * packed runs)
    int64_t kchunk;         // contraction indices per split (padded space for tc)
    size_t part_bytes;
    size_t image_bytes;     // B-operand image of the tensor-core path
};

// Work decomposition of one contraction.  `tc_ok` says whether the tensor-core
// kernel accepts the shape; otherwise the FP32 kernel runs (it handles every shape).
ContractPlan plan_contract(int64_t I, int64_t K, int C, int precision, int splits, bool tc_ok,
                           int BI_tc) {
    ContractPlan pl;
    pl.image_bytes = 0;
    pl.tc = ((precision == MTK_PREC_BF16X2 || precision == MTK_PREC_BF16X3) && tc_ok) ? 1 : 0;
    const int BI = pl.tc ? BI_tc : simt_tile_rows(I);
    pl.i_tiles = (int)((I + BI - 1) / BI);
    pl.c_blocks = pl.tc ? 1 : (C + simt_cta_cols(C) - 1) / simt_cta_cols(C);
    const int64_t quantum = pl.tc ? kTcBK : kBK;            // split boundaries: whole stages
    int64_t S = splits;
    if (S <= 0) {
        const int64_t target = (int64_t)num_sms() * (pl.tc ? 2 : simt_ctas_per_sm(I));   // CTAs per wave
        const int64_t tiles = (int64_t)pl.i_tiles * pl.c_blocks;
        S = target / tiles;
        const int64_t maxS = (K + 4 * kTcBK - 1) / (4 * kTcBK);   // >= 4 stages per split
        if (S > maxS) S = maxS;
    }
    if (S < 1) S = 1;
    if (S > 4096) S = 4096;
    int64_t chunk = (K + S - 1) / S;
    chunk = (chunk + quantum - 1) / quantum * quantum;
    if (chunk < 1) chunk = 1;
    pl.kchunk = chunk;
    pl.S = (int)((K + chunk - 1) / chunk);
    pl.slabs = pl.S;
    pl.part_bytes = pl.slabs > 1 ? (size_t)pl.slabs * I * C * sizeof(float) : 0;
    return pl;
}

// plan for the contraction on view (L, I, *) against the factor list (radices frad,
// first fastest; their product is the contraction length); x_aligned16 says whether
// the tensor pointer allows 16-byte loads
ContractPlan plan_for(int64_t L, int64_t I, const int64_t* frad, int nfac, int C, const mtk_opts& o,
                      bool x_aligned16) {
    int64_t K = 1;
    for (int z = 0; z < nfac; ++z) K *= frad[z];
    const bool tc_ok = x_aligned16 && nfac >= 1 && contract_tc_shape_ok(L, I, C, o.precision);
    if (tc_ok) {
        const TcPlan tp = contract_tc_plan(frad, nfac, L, I, C);
        ContractPlan pl = plan_contract(I, tp.Kp, C, o.precision, o.splits, true, tp.BI);
        pl.image_bytes = tp.image_bytes;
        pl.slabs = pl.S * tp.U;
        pl.part_bytes = pl.slabs > 1 ? (size_t)pl.slabs * I * C * sizeof(float) : 0;
        return pl;
    }
    return plan_contract(I, K, C, o.precision, o.splits, false, 0);
}

// the plan used for workspace sizing: the larger scratch of the two alignments
ContractPlan plan_both(int64_t L, int64_t I, const int64_t* frad, int nfac, int C, const mtk_opts& o) {
    ContractPlan a = plan_for(L, I, frad, nfac, C, o, true);
    const ContractPlan b = plan_for(L, I, frad, nfac, C, o, false);
    if (b.part_bytes > a.part_bytes) a.part_bytes = b.part_bytes;
    if (b.image_bytes > a.image_bytes) a.image_bytes = b.image_bytes;
    return a;
}

size_t plan_scratch(const ContractPlan& pl) { return align256(pl.image_bytes) + align256(pl.part_bytes); }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// factor list of mode n: U_0..U_{n-1}, U_{n+1}..U_{N-1} (first fastest)
struct FactorList {
    int Z;
    const float* f[MTK_MAXN];
    int64_t rad[MTK_MAXN];
};

FactorList mode_factors(const float* const* U, const int64_t* dims, int N, int n) {
    FactorList fl;
    fl.Z = 0;
    for (int k = 0; k < N; ++k) {
        if (k == n) continue;
        fl.f[fl.Z] = U ? U[k] : nullptr;
        fl.rad[fl.Z] = dims[k];
        ++fl.Z;
    }
    return fl;
}

// leading factors merged into one materialised head when the first radix is < 32
int head_merge_count(const FactorList& fl) {
    if (fl.Z <= 1 || fl.rad[0] >= kBK) return 0;
    int m = 0;
    int64_t p = 1;
    while (m < fl.Z && p < kBK) { p *= fl.rad[m]; ++m; }
    return m;
}

size_t head_bytes(const FactorList& fl, int C) {
    const int m = head_merge_count(fl);
    if (m == 0) return 0;
    int64_t rows = 1;
    for (int z = 0; z < m; ++z) rows *= fl.rad[z];
    return (size_t)rows * C * sizeof(float);
}

// Build the KRP operand from a factor list; materialises a merged head into `head`
// (device scratch of head_bytes) with the KRP kernel when needed.
cudaError_t make_operand(const FactorList& fl, int C, float* head, KrpOperand* W, cudaStream_t s) {
    memset(W, 0, sizeof(*W));
    const int m = head_merge_count(fl);
    if (m == 0) {
        W->f0 = fl.f[0];
        W->rad0 = fl.rad[0];
        W->ntail = fl.Z - 1;
        for (int z = 1; z < fl.Z; ++z) { W->tail[z - 1] = fl.f[z]; W->tail_rad[z - 1] = fl.rad[z]; }
        return cudaSuccess;
    }
    // head = U_{m-1} kr ... kr U_0 (first factor fastest)
    const float* ops[MTK_MAXN];
    int64_t rows[MTK_MAXN];
    int64_t hr = 1;
    for (int z = 0; z < m; ++z) { ops[z] = fl.f[m - 1 - z]; rows[z] = fl.rad[m - 1 - z]; hr *= fl.rad[z]; }
    cudaError_t e = launch_krp(ops, rows, m, C, head, 1, s);
    W->f0 = head;
    W->rad0 = hr;
    W->ntail = fl.Z - m;
    for (int z = m; z < fl.Z; ++z) { W->tail[z - m] = fl.f[z]; W->tail_rad[z - m] = fl.rad[z]; }
    return e;
}

// scratch: device memory of plan_scratch(sized plan) bytes (image, then partials)
int run_contract(ContractParams& p, const ContractPlan& pl, int precision, void* scratch,
                 cudaStream_t s) {
    cudaError_t e;
    char* sc = static_cast<char*>(scratch);
    p.S = pl.S;
    p.kchunk = pl.kchunk;
    p.part = reinterpret_cast<float*>(sc + align256(pl.image_bytes));
    if (pl.tc) {
        if (!contract_tc_supported(p, precision)) return MTK_EUNSUPPORTED;
        e = launch_contract_tc(p, precision, sc, s);
    } else {
        e = launch_contract_simt(p, pl.c_blocks, pl.i_tiles, s);
    }
    if (e != cudaSuccess) return MTK_ECUDA;
    if (pl.slabs > 1) {
        e = launch_split_reduce(p.part, pl.slabs, p.I, p.C, p.out, p.out_si, p.out_sc, s);
        if (e != cudaSuccess) return MTK_ECUDA;
    }
    return MTK_OK;
}

// --- MTTKRP workspace layout --------------------------------------------------
struct MttkrpLayout {
    int algo;               // resolved algorithm
    int right;              // two-step ordering
    ContractPlan plan;
    size_t head, krp_full, kl, kr, tmat, total;
};

int resolve_algo(int algo, int N, int n) {
    if (algo == MTK_ALGO_AUTO) return MTK_ALGO_FUSED;
    if (algo == MTK_ALGO_TWO_STEP && (n == 0 || n == N - 1)) return MTK_ALGO_FUSED;  // degenerates
    return algo;
}

MttkrpLayout mttkrp_layout(const int64_t* dims, int N, int C, int n, const mtk_opts& o) {
    MttkrpLayout ly;
    memset(&ly, 0, sizeof(ly));
    const View v = mode_view(dims, N, n);
    ly.algo = resolve_algo(o.algo, N, n);
    Carve cv{nullptr, kStatusBytes, 0};
    if (ly.algo == MTK_ALGO_FUSED) {
        FactorList fl = mode_factors(nullptr, dims, N, n);
        ly.head = head_bytes(fl, C);
        cv.take(ly.head);
        ly.plan = plan_both(v.L, v.I, fl.rad, fl.Z, C, o);
    } else if (ly.algo == MTK_ALGO_MATERIALIZED) {
        ly.krp_full = (size_t)v.L * v.R * C * sizeof(float);
        cv.take(ly.krp_full);
        const int64_t rad = v.L * v.R;
        ly.plan = plan_both(v.L, v.I, &rad, 1, C, o);
    } else {  // two-step, internal mode
        ly.right = (v.L > v.R) ? 0 : 1;       // left first iff I^L > I^R (Algorithm 4)
        ly.kl = (size_t)v.L * C * sizeof(float);
        ly.kr = (size_t)v.R * C * sizeof(float);
        ly.tmat = (size_t)(ly.right ? v.L * v.I : v.I * v.R) * C * sizeof(float);
        cv.take(ly.kl);
        cv.take(ly.kr);
        cv.take(ly.tmat);
        const int64_t Ip = ly.right ? v.L * v.I : v.I * v.R;
        const int64_t Kp = ly.right ? v.R : v.L;
        ly.plan = plan_both(ly.right ? 1 : v.L, Ip, &Kp, 1, C, o);
    }
    cv.take(plan_scratch(ly.plan));
    ly.total = align256(cv.off);
    return ly;
}

void set_factors(ContractParams& p, const float* const* f, const int64_t* rad, int nfac) {
    p.nfac = nfac;
    for (int z = 0; z < nfac; ++z) { p.fac[z] = f[z]; p.frad[z] = rad[z]; }
}

// ws: workspace laid out by mttkrp_layout (its first kStatusBytes are not used here);
// status: the device status word the kernels report into.
int do_mttkrp(const float* X, const int64_t* dims, int N, const float* const* U, int C, int n,
              float* M, void* ws, size_t ws_bytes, uint32_t* status, const mtk_opts& o,
              cudaStream_t s) {
    const MttkrpLayout ly = mttkrp_layout(dims, N, C, n, o);
    if (ws_bytes < ly.total) return MTK_EWORKSPACE;
    const View v = mode_view(dims, N, n);
    Carve cv{static_cast<char*>(ws), kStatusBytes, ws_bytes};
    ContractParams p;
    memset(&p, 0, sizeof(p));
    p.X = X;
    p.C = C;
    p.status = status;
    p.wait_ns = wait_limit_ns(o);
    p.stall = o.test_stall;
    if (ly.algo == MTK_ALGO_FUSED || ly.algo == MTK_ALGO_MATERIALIZED) {
        p.L = v.L; p.I = v.I; p.R = v.R; p.K = v.L * v.R;
        FactorList fl = mode_factors(U, dims, N, n);
        if (ly.algo == MTK_ALGO_FUSED) {
            float* head = static_cast<float*>(cv.take(ly.head));
            set_factors(p, fl.f, fl.rad, fl.Z);
            const ContractPlan pl = plan_for(v.L, v.I, p.frad, p.nfac, C, o, aligned16(X));
            if (!pl.tc && make_operand(fl, C, head, &p.W, s) != cudaSuccess) return MTK_ECUDA;
        } else {
            float* K = static_cast<float*>(cv.take(ly.krp_full));
            const float* ops[MTK_MAXN];
            int64_t rows[MTK_MAXN];
            for (int z = 0; z < fl.Z; ++z) { ops[z] = fl.f[fl.Z - 1 - z]; rows[z] = fl.rad[fl.Z - 1 - z]; }
            if (launch_krp(ops, rows, fl.Z, C, K, 1, s) != cudaSuccess) return MTK_ECUDA;
            p.W.f0 = K; p.W.rad0 = p.K; p.W.ntail = 0;
            const float* kf = K;
            set_factors(p, &kf, &p.K, 1);
        }
        p.out = M; p.out_si = C; p.out_sc = 1;
        const ContractPlan pl = plan_for(v.L, v.I, p.frad, p.nfac, C, o, aligned16(X));
        return run_contract(p, pl, o.precision, cv.take(plan_scratch(ly.plan)), s);
    }
    // two-step (Algorithm 4)
    float* KL = static_cast<float*>(cv.take(ly.kl));
    float* KR = static_cast<float*>(cv.take(ly.kr));
    float* T = static_cast<float*>(cv.take(ly.tmat));
    {
        const float* ops[MTK_MAXN];
        int64_t rows[MTK_MAXN];
        int Z = 0;
        for (int k = n - 1; k >= 0; --k) { ops[Z] = U[k]; rows[Z] = dims[k]; ++Z; }
        if (launch_krp(ops, rows, Z, C, KL, 1, s) != cudaSuccess) return MTK_ECUDA;
        Z = 0;
        for (int k = N - 1; k > n; --k) { ops[Z] = U[k]; rows[Z] = dims[k]; ++Z; }
        if (launch_krp(ops, rows, Z, C, KR, 1, s) != cudaSuccess) return MTK_ECUDA;
    }
    if (ly.right) {
        p.L = 1; p.I = v.L * v.I; p.R = v.R; p.K = v.R;
        p.W.f0 = KR; p.W.rad0 = v.R;
        p.out = T; p.out_si = 1; p.out_sc = v.L * v.I;
        const float* kf = KR;
        set_factors(p, &kf, &p.K, 1);
    } else {
        p.L = v.L; p.I = v.I * v.R; p.R = 1; p.K = v.L;
        p.W.f0 = KL; p.W.rad0 = v.L;
        p.out = T; p.out_si = 1; p.out_sc = v.I * v.R;
        const float* kf = KL;
        set_factors(p, &kf, &p.K, 1);
    }
    const ContractPlan pl = plan_for(p.L, p.I, p.frad, p.nfac, C, o, aligned16(X));
    int st = run_contract(p, pl, o.precision, cv.take(plan_scratch(ly.plan)), s);
    if (st) return st;
    if (launch_multi_ttv(T, v.L, v.I, v.R, ly.right ? KL : KR, C, ly.right, M, s) != cudaSuccess)
        return MTK_ECUDA;
    return MTK_OK;
}

// --- MTTKRP on a tensor split into BF16 planes ------------------------------------
// CTAs of a planes contraction: the caller's count, else one per SM less `reserve` (a CP-ALS
// sweep leaves one SM to the factorisation it overlaps with the contraction)
int planes_ctas_for(const mtk_opts& o, int reserve) {
    const int c = planes_ctas(o.splits);
    return (o.splits > 0 || c - reserve < 1) ? c : c - reserve;
}

// The planes keep mode 0 padded to a multiple of 8 (planes_dims): every view below is of
// the padded tensor.  Its first factor U_0 has only I_0 rows (the head image takes the
// padding rows as zero), and mode 0's output keeps only rows i_0 < I_0.
PlanesPlan planes_for(const int64_t* dims, int N, int C, int n, const mtk_opts& o, int reserve = 0) {
    int64_t pd[MTK_MAXN];
    planes_dims(dims, N, pd);
    const View v = mode_view(pd, N, n);
    const FactorList fl = mode_factors(nullptr, pd, N, n);
    return planes_plan(v.L, v.I, fl.rad, fl.Z, C, n, planes_ctas_for(o, reserve));
}

int64_t planes_entries(const int64_t* dims, int N) {
    int64_t e = planes_rows0(dims[0]);
    for (int k = 1; k < N; ++k) e *= dims[k];
    return e;
}

mtk_opts fallback_opts(const mtk_opts& o) {
    mtk_opts f = o;
    f.algo = MTK_ALGO_FUSED;
    f.precision = MTK_PREC_BF16X2;
    return f;
}

PlanesPlan partial_plan(const int64_t* dims, int N, int C, int n, int right, const mtk_opts& o, int reserve = 0);
int run_partial_split(const void* Xs, const int64_t* dims, int N, const float* const* U, int C, int n,
                      int right, float* T, void* ws, uint32_t* status, const mtk_opts& o, cudaStream_t s,
                      const FactorHook* hook = nullptr, int reserve = 0);

// Modes 0 and 1 whose stages would be poorly filled are taken as Algorithm 4's two steps:
// the contraction over the modes >= 2 on the view (1, I_0 I_1, I^R) (mode-0-like tiles over
// I_0 I_1 rows, whose head is a prefix of U_2, U_3, ...) and a multi-TTV with U_1 (mode
// 0) or U_0 (mode 1).  The tensor is read once either way; the partial is I_0 I_1 C floats.
//  - mode 0 with I_0 <= 32 (after padding): its 64-row boxes would be half empty;
//  - mode 1 whose head (U_0 alone) uses under 3/5 of its 64-k stages (I_0 = 30: 32 rows in
//    64).  A stage costs a fixed ~750 cycles besides its bytes.
bool two_step_right(const int64_t* dims, int N, int C, int n, const mtk_opts& o, int reserve) {
    if (n > 1 || N < 3) return false;
    if (n == 0) {
        if (planes_rows0(dims[0]) > 32) return false;
    } else {
        const PlanesPlan pl = planes_for(dims, N, C, n, o, reserve);
        if (!pl.ok || pl.H * 5 >= (int64_t)pl.spr * 64 * 3) return false;
    }
    return partial_plan(dims, N, C, 1, 1, o, reserve).ok;
}

// workspace of one MTTKRP on the planes: the planes kernel's scratch when it takes the
// shape, else that of the FP32-tensor path it falls back to
size_t split_mttkrp_bytes(const int64_t* dims, int N, int C, int n, const mtk_opts& o, int reserve = 0) {
    const PlanesPlan pl = planes_for(dims, N, C, n, o, reserve);
    if (!pl.ok) return mttkrp_layout(dims, N, C, n, fallback_opts(o)).total;
    if (two_step_right(dims, N, C, n, o, reserve))
        return align256(align256(kStatusBytes) + align256((size_t)dims[0] * dims[1] * C * sizeof(float)) +
                        planes_scratch_bytes(partial_plan(dims, N, C, 1, 1, o, reserve)));
    return align256(align256(kStatusBytes) + planes_scratch_bytes(pl));
}

// hook (may be null): a factorisation to run alongside the planes contraction; *hooked
// (may be null) tells whether it ran (not when the shape falls back to the FP32 tensor)
int do_mttkrp_split(const void* Xs, const float* X, const int64_t* dims, int N, const float* const* U,
                    int C, int n, float* M, void* ws, size_t ws_bytes, uint32_t* status,
                    const mtk_opts& o, cudaStream_t s, const FactorHook* hook = nullptr, int reserve = 0,
                    bool* hooked = nullptr) {
    if (hooked) *hooked = false;
    const PlanesPlan pl = planes_for(dims, N, C, n, o, reserve);
    if (!pl.ok) {
        if (!X) return MTK_EUNSUPPORTED;
        return do_mttkrp(X, dims, N, U, C, n, M, ws, ws_bytes, status, fallback_opts(o), s);
    }
    if (ws_bytes < split_mttkrp_bytes(dims, N, C, n, o, reserve)) return MTK_EWORKSPACE;
    if (two_step_right(dims, N, C, n, o, reserve)) {
        // T(i0, i1, c) over modes >= 2, then M_0(i0, c) = sum_i1 T(i0, i1, c) U_1(i1, c) or
        // M_1(i1, c) = sum_i0 T(i0, i1, c) U_0(i0, c)
        Carve cv{static_cast<char*>(ws), kStatusBytes, ws_bytes};
        float* T = static_cast<float*>(cv.take((size_t)dims[0] * dims[1] * C * sizeof(float)));
        char* inner = static_cast<char*>(cv.take(0)) - kStatusBytes;     // scratch follows T
        const int st = run_partial_split(Xs, dims, N, U, C, 1, 1, T, inner, status, o, s, hook, reserve);
        if (st) return st;
        if (hooked) *hooked = hook != nullptr;
        const cudaError_t e = n == 0 ? launch_multi_ttv(T, 1, dims[0], dims[1], U[1], C, 0, M, s)
                                     : launch_multi_ttv(T, dims[0], dims[1], 1, U[0], C, 1, M, s);
        if (e != cudaSuccess) return MTK_ECUDA;
        return MTK_OK;
    }
    int64_t pd[MTK_MAXN];
    planes_dims(dims, N, pd);
    const View v = mode_view(pd, N, n);
    const FactorList fl = mode_factors(U, pd, N, n);
    Carve cv{static_cast<char*>(ws), kStatusBytes, ws_bytes};
    void* scratch = cv.take(planes_scratch_bytes(pl));
    // the factor list starts with U_0 for n >= 1; mode 0's rows beyond I_0 are padding
    const int64_t f0_rows = n >= 1 ? dims[0] : fl.rad[0];
    const int64_t opad = n == 0 ? pd[0] : 0;
    if (launch_contract_planes(Xs, split_pitch(planes_entries(dims, N)), v.L, v.I, v.R, fl.f, fl.rad, fl.Z, C,
                               pl, M, C, 1, scratch, status, s, wait_limit_ns(o), o.test_stall, hook, f0_rows,
                               opad, dims[0]) != cudaSuccess)
        return MTK_ECUDA;
    if (hooked) *hooked = hook != nullptr;
    return MTK_OK;
}

// the planes hold two BF16 pieces: precision AUTO or BF16X2, the fused algorithm (a
// sweep also takes MTK_ALGO_TWO_STEP: the dimension tree below)
int check_split_opts(const mtk_opts* raw, bool sweep = false) {
    if (!raw) return MTK_OK;
    if (raw->algo != MTK_ALGO_AUTO && raw->algo != MTK_ALGO_FUSED && !(sweep && raw->algo == MTK_ALGO_TWO_STEP))
        return MTK_EINVAL;
    if (raw->precision != MTK_PREC_AUTO && raw->precision != MTK_PREC_BF16X2) return MTK_EINVAL;
    return MTK_OK;
}

// --- dimension tree of a CP-ALS sweep on the planes (N = 3 or 4) ---------------------
// The modes split into a left pair {0, 1} and the rest.  The right partial
// T_R(i0, i1, c) = sum over the modes >= 2 of X * prod U_k is shared by the updates of
// U_0 and U_1 (the factors it uses do not change in between), the left partial
// T_L(i2, i3, c) = sum over modes 0, 1 by those of U_2 and U_3 (N = 4; for N = 3 the
// mode-2 MTTKRP is run as it is).  Each partial is one planes contraction on another
// 3-way view of the same planes; the per-mode MTTKRPs follow from it by multi-TTVs
// (Section 4.3, Algorithm 4's second step).  The tensor is read twice per sweep.
bool tree_shape(const int64_t* dims, int N, int C) { return (N == 3 || N == 4) && C <= 64 && dims; }

// First step of Algorithm 4 on the planes.  right = 1: the contraction over the modes
// > n on the 3-way view (1, I^L I_n, I^R), T[l + I^L i + I^L I_n c]; right = 0: over the
// modes < n on the view (I^L, I_n I^R, 1), T[i + I_n r + I_n I^R c].  The partial KRP
// is formed on chip from the factors, as in a per-mode MTTKRP.
bool partial_sides_ok(int N, int n, int right) { return right ? n < N - 1 : n > 0; }

PlanesPlan partial_plan(const int64_t* dims, int N, int C, int n, int right, const mtk_opts& o, int reserve) {
    int64_t pd[MTK_MAXN];
    planes_dims(dims, N, pd);
    const View v = mode_view(pd, N, n);
    const int ctas = planes_ctas_for(o, reserve);
    if (right) return planes_plan(1, v.L * v.I, pd + n + 1, N - n - 1, C, 0, ctas);
    return planes_plan(v.L, v.I * v.R, pd, n, C, n, ctas);
}

// the dimension tree's partials: right = modes >= 2 (n = 1), left = modes 0, 1 (n = 2)
PlanesPlan tree_plan(const int64_t* dims, int N, int C, int right, const mtk_opts& o, int reserve = 0) {
    return partial_plan(dims, N, C, right ? 1 : 2, right, o, reserve);
}

bool tree_ok(const int64_t* dims, int N, int C, const mtk_opts& o, int reserve = 0) {
    if (!tree_shape(dims, N, C)) return false;
    if (!tree_plan(dims, N, C, 1, o, reserve).ok) return false;
    return N == 3 || tree_plan(dims, N, C, 0, o, reserve).ok;
}

size_t tree_scratch(const int64_t* dims, int N, int C, const mtk_opts& o, int reserve = 0) {
    size_t a = planes_scratch_bytes(tree_plan(dims, N, C, 1, o, reserve));
    if (N == 4) {
        const size_t b = planes_scratch_bytes(tree_plan(dims, N, C, 0, o, reserve));
        if (b > a) a = b;
    }
    return align256(align256(kStatusBytes) + a);
}

// ws: status (unused) then the planes scratch; T: rows x C, C slowest
int run_partial_split(const void* Xs, const int64_t* dims, int N, const float* const* U, int C, int n,
                      int right, float* T, void* ws, uint32_t* status, const mtk_opts& o, cudaStream_t s,
                      const FactorHook* hook, int reserve) {
    const PlanesPlan pl = partial_plan(dims, N, C, n, right, o, reserve);
    if (!pl.ok) return MTK_EUNSUPPORTED;
    int64_t pd[MTK_MAXN];
    planes_dims(dims, N, pd);
    const View v = mode_view(pd, N, n);
    const float* fac[MTK_MAXN];
    int64_t frad[MTK_MAXN];
    int nf = 0;
    for (int k = right ? n + 1 : 0; k < (right ? N : n); ++k) {
        fac[nf] = U[k];
        frad[nf] = pd[k];
        ++nf;
    }
    Carve cv{static_cast<char*>(ws), kStatusBytes, 0};
    void* scratch = cv.take(planes_scratch_bytes(pl));
    const int64_t pitch = split_pitch(planes_entries(dims, N));
    cudaError_t e;
    if (right) {
        // rows (i_0 .. i_n) of the padded view; the output drops the padding rows of mode 0
        const int64_t rows = v.L * v.I;
        const int64_t out_rows = rows / pd[0] * dims[0];
        e = launch_contract_planes(Xs, pitch, 1, rows, v.R, fac, frad, nf, C, pl, T, 1, out_rows, scratch, status,
                                   s, wait_limit_ns(o), o.test_stall, hook, frad[0], pd[0], dims[0]);
    } else {
        // the factors start with U_0, whose padding rows the head image takes as zero
        const int64_t rows = v.I * v.R;
        e = launch_contract_planes(Xs, pitch, v.L, rows, 1, fac, frad, nf, C, pl, T, 1, rows, scratch, status, s,
                                   wait_limit_ns(o), o.test_stall, hook, dims[0], 0, 0);
    }
    return e == cudaSuccess ? MTK_OK : MTK_ECUDA;
}

size_t partial_split_bytes(const PlanesPlan& pl) {
    return align256(align256(kStatusBytes) + planes_scratch_bytes(pl));
}

int run_tree_partial(const void* Xs, const int64_t* dims, int N, const float* const* U, int C, int right, float* T,
                     void* ws, uint32_t* status, const mtk_opts& o, cudaStream_t s, const FactorHook* hook,
                     int reserve) {
    return run_partial_split(Xs, dims, N, U, C, right ? 1 : 2, right, T, ws, status, o, s, hook, reserve);
}

int check_mttkrp_ptrs(const float* X, const float* const* U, int N, int n, const float* M,
                      const void* ws) {
    if (!X || !U || !M || !ws) return MTK_EINVAL;
    if (!aligned4(X) || !aligned4(M)) return MTK_EINVAL;
    for (int k = 0; k < N; ++k) {
        if (k == n) continue;
        if (!U[k] || !aligned4(U[k])) return MTK_EINVAL;
    }
    return MTK_OK;
}

}  // namespace

extern "C" {

const char* mtk_status_string(int st) {
    switch (st) {
        case MTK_OK: return "ok";
        case MTK_EINVAL: return "invalid argument";
        case MTK_ECUDA: return "CUDA error";
        case MTK_ENOTPD: return "normal-equation matrix not positive definite";
        case MTK_ETIMEOUT: return "device wait expired";
        case MTK_EUNSUPPORTED: return "unsupported option for this shape";
        case MTK_EWORKSPACE: return "workspace too small";
        default: return "unknown status";
    }
}

int mtk_version(void) { return 100; }

uint64_t mtk_launch_count(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

int mtk_clear_status(void* ws, void* stream) {
    if (!ws) return MTK_EINVAL;
    if (cudaMemsetAsync(ws, 0, kStatusBytes, (cudaStream_t)stream) != cudaSuccess) return MTK_ECUDA;
    return MTK_OK;
}

int mtk_read_status(const void* ws, void* stream, uint32_t* bits_out) {
    if (!ws) return MTK_EINVAL;
    uint32_t bits = 0;
    if (cudaMemcpyAsync(&bits, ws, sizeof(bits), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
        cudaSuccess)
        return MTK_ECUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return MTK_ECUDA;
    if (bits_out) *bits_out = bits;
    for (int code = 1; code < 32; ++code)
        if (bits & (1u << code)) return code;
    return MTK_OK;
}

int mtk_khatri_rao(const float* const* U, const int64_t* rows, int Z, int C, float* K, int reuse,
                   void* stream) {
    if (!U || !rows || !K || Z < 1 || Z > MTK_MAXN || C < 1 || C > MTK_MAXC) return MTK_EINVAL;
    int64_t J = 1;
    for (int z = 0; z < Z; ++z) {
        if (!U[z] || rows[z] < 1 || !aligned4(U[z])) return MTK_EINVAL;
        if (J > ((int64_t)1 << 62) / rows[z]) return MTK_EINVAL;
        J *= rows[z];
    }
    if (!aligned4(K)) return MTK_EINVAL;
    if (launch_krp(U, rows, Z, C, K, reuse, (cudaStream_t)stream) != cudaSuccess) return MTK_ECUDA;
    return MTK_OK;
}

size_t mtk_mttkrp_workspace(const int64_t* dims, int N, int C, int n, const mtk_opts* opts) {
    if (check_shape(dims, N, C, n) != MTK_OK) return 0;
    mtk_opts o = defaults(opts);
    if (o.algo < 0) return 0;
    return mttkrp_layout(dims, N, C, n, o).total;
}

int mtk_mttkrp(const float* X, const int64_t* dims, int N, const float* const* U, int C, int n,
               float* M, void* ws, size_t ws_bytes, const mtk_opts* opts, void* stream) {
    int st = check_shape(dims, N, C, n);
    if (st) return st;
    st = check_mttkrp_ptrs(X, U, N, n, M, ws);
    if (st) return st;
    mtk_opts o = defaults(opts);
    if (o.algo < 0 || o.precision < MTK_PREC_FP32 || o.precision > MTK_PREC_BF16X3) return MTK_EINVAL;
    return do_mttkrp(X, dims, N, U, C, n, M, ws, ws_bytes, static_cast<uint32_t*>(ws), o,
                     (cudaStream_t)stream);
}

int mtk_mttkrp_noalloc(const float* X, const int64_t* dims, int N, const float* const* U, int C,
                       int n, float* M, const mtk_opts* opts, uint32_t* status_bits, void* stream) {
    int st = check_shape(dims, N, C, n);
    if (st) return st;
    st = check_mttkrp_ptrs(X, U, N, n, M, M);   // no caller workspace to check
    if (st) return st;
    mtk_opts o = defaults(opts);
    if (o.algo < 0 || o.precision < MTK_PREC_FP32 || o.precision > MTK_PREC_BF16X3) return MTK_EINVAL;
    if (mttkrp_layout(dims, N, C, n, o).total > MTK_NOALLOC_SCRATCH_BYTES) return MTK_EWORKSPACE;
    // set-up, once per device (and again whenever that device's context is new, e.g.
    // after cudaDeviceReset), with that device current: the device address of the array
    static std::mutex mu;
    static void* dev_scratch[kNoAllocMaxDevices];
    static unsigned long long dev_ctx[kNoAllocMaxDevices];
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return MTK_ECUDA;
    void* ws;
    {
        std::lock_guard<std::mutex> lock(mu);
        const unsigned long long id = current_context_id();
        if (!dev_scratch[dev] || id == 0 || id != dev_ctx[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MTK_ECUDA;
            dev_scratch[dev] = p;
            dev_ctx[dev] = current_context_id();   // the lookup made the context current
        }
        ws = dev_scratch[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(ws, 0, kStatusBytes, s) != cudaSuccess) return MTK_ECUDA;
    st = do_mttkrp(X, dims, N, U, C, n, M, ws, MTK_NOALLOC_SCRATCH_BYTES, static_cast<uint32_t*>(ws), o, s);
    if (st || !status_bits) return st;
    return mtk_read_status(ws, stream, status_bits);
}

namespace {
bool split_dims_ok(const int64_t* dims, int N) {
    if (!dims || N < 1 || N > MTK_MAXN) return false;
    int64_t e = 1;
    for (int k = 0; k < N; ++k) {
        if (dims[k] < 1 || dims[k] > ((int64_t)1 << 40)) return false;
        const int64_t d = k == 0 ? planes_rows0(dims[0]) : dims[k];
        if (e > ((int64_t)1 << 46) / d) return false;
        e *= d;
    }
    return true;
}
}  // namespace

int64_t mtk_split_rows0(int64_t I0) { return I0 < 1 ? 0 : planes_rows0(I0); }

int64_t mtk_split_pitch(const int64_t* dims, int N) {
    return split_dims_ok(dims, N) ? split_pitch(planes_entries(dims, N)) : 0;
}

size_t mtk_split_bytes(const int64_t* dims, int N) {
    return split_dims_ok(dims, N) ? (size_t)(2 * split_pitch(planes_entries(dims, N))) * 2 : 0;
}

size_t mtk_split_workspace(const int64_t* dims, int N) {
    if (!split_dims_ok(dims, N)) return 0;
    return align256(kStatusBytes) + align256((size_t)split_chunks(planes_entries(dims, N)) * sizeof(double));
}

int mtk_split_tensor(const float* X, const int64_t* dims, int N, void* Xs, double* normX2, void* ws,
                     size_t ws_bytes, void* stream) {
    if (!X || !Xs || !ws || !split_dims_ok(dims, N) || !aligned4(X) || !aligned16(Xs)) return MTK_EINVAL;
    if (ws_bytes < mtk_split_workspace(dims, N)) return MTK_EWORKSPACE;
    double* part = reinterpret_cast<double*>(static_cast<char*>(ws) + align256(kStatusBytes));
    int64_t rest = 1;
    for (int k = 1; k < N; ++k) rest *= dims[k];
    const float* Xv = nullptr;
    const int st = device_view(X, &Xv);
    if (st) return st;
    if (launch_split_planes(Xv, dims[0], rest, Xs, part, normX2, (cudaStream_t)stream) != cudaSuccess)
        return MTK_ECUDA;
    return MTK_OK;
}

size_t mtk_mttkrp_split_workspace(const int64_t* dims, int N, int C, int n, const mtk_opts* opts) {
    if (check_shape(dims, N, C, n) != MTK_OK) return 0;
    if (check_split_opts(opts) != MTK_OK) return 0;
    return split_mttkrp_bytes(dims, N, C, n, defaults(opts));
}

int mtk_mttkrp_split(const void* Xs, const float* X, const int64_t* dims, int N, const float* const* U,
                     int C, int n, float* M, void* ws, size_t ws_bytes, const mtk_opts* opts,
                     void* stream) {
    int st = check_shape(dims, N, C, n);
    if (st) return st;
    if (!Xs || !aligned16(Xs)) return MTK_EINVAL;
    if (X && !aligned4(X)) return MTK_EINVAL;
    st = check_mttkrp_ptrs(X ? X : static_cast<const float*>(Xs), U, N, n, M, ws);
    if (st) return st;
    if (check_split_opts(opts) != MTK_OK) return MTK_EINVAL;
    mtk_opts o = defaults(opts);
    return do_mttkrp_split(Xs, X, dims, N, U, C, n, M, ws, ws_bytes, static_cast<uint32_t*>(ws), o,
                           (cudaStream_t)stream);
}

size_t mtk_partial_mttkrp_split_workspace(const int64_t* dims, int N, int C, int n, int right,
                                          const mtk_opts* opts) {
    if (check_shape(dims, N, C, n) != MTK_OK || !partial_sides_ok(N, n, right)) return 0;
    if (check_split_opts(opts) != MTK_OK) return 0;
    const PlanesPlan pl = partial_plan(dims, N, C, n, right, defaults(opts));
    return pl.ok ? partial_split_bytes(pl) : 0;
}

int mtk_partial_mttkrp_split(const void* Xs, const int64_t* dims, int N, const float* const* U, int C,
                             int n, int right, float* T, void* ws, size_t ws_bytes,
                             const mtk_opts* opts, void* stream) {
    int st = check_shape(dims, N, C, n);
    if (st) return st;
    if (!partial_sides_ok(N, n, right)) return MTK_EINVAL;
    if (!Xs || !aligned16(Xs) || !U || !T || !aligned4(T) || !ws) return MTK_EINVAL;
    for (int k = right ? n + 1 : 0; k < (right ? N : n); ++k)
        if (!U[k] || !aligned4(U[k])) return MTK_EINVAL;
    if (check_split_opts(opts) != MTK_OK) return MTK_EINVAL;
    const mtk_opts o = defaults(opts);
    const PlanesPlan pl = partial_plan(dims, N, C, n, right, o);
    if (!pl.ok) return MTK_EUNSUPPORTED;
    if (ws_bytes < partial_split_bytes(pl)) return MTK_EWORKSPACE;
    return run_partial_split(Xs, dims, N, U, C, n, right, T, ws, static_cast<uint32_t*>(ws), o,
                             (cudaStream_t)stream);
}

// ---- every mode's MTTKRP with the same factors (the gradient of the CP loss) ----------------
namespace {
// The dimension tree: the right partial T_R (modes 0, 1 kept) serves modes 0 and 1; for
// N = 3 mode 2 is one planes MTTKRP; for N >= 4 the left partial T_L (modes 0, 1
// contracted, modes 2..N-1 kept: prod_{k>=2} I_k C floats) serves the others, through
// multi-TTVs (N = 4) or one-mode contractions of T_L (N >= 5, while T_L is at most a
// quarter of the tensor's entries).  Workspace: status, T_R and T_L, two buffers of T_L's
// size (N >= 5), then the larger of the partial contractions' scratch and (N = 3) the
// mode-2 MTTKRP's.
int64_t tree_rest(const int64_t* dims, int N) {
    int64_t r = 1;
    for (int k = 2; k < N; ++k) r *= dims[k];
    return r;
}
bool all_tree(const int64_t* dims, int N, int C, const mtk_opts& o) {
    if (o.algo == MTK_ALGO_FUSED || N < 3 || C > 64) return false;
    if (N <= 4) return tree_ok(dims, N, C, o);
    if (!partial_plan(dims, N, C, 1, 1, o).ok || !partial_plan(dims, N, C, 2, 0, o).ok) return false;
    return (int64_t)C * 4 <= dims[0] * dims[1];
}
size_t all_split_bytes(const int64_t* dims, int N, int C, const mtk_opts& o) {
    if (all_tree(dims, N, C, o)) {
        size_t t = (size_t)dims[0] * dims[1] * C * sizeof(float);
        if (N >= 4) t += (size_t)tree_rest(dims, N) * C * sizeof(float);
        if (N >= 5) t = align256(t) + 2 * align256((size_t)tree_rest(dims, N) * C * sizeof(float));
        size_t inner = planes_scratch_bytes(partial_plan(dims, N, C, 1, 1, o));
        if (N >= 4) {
            const size_t b = planes_scratch_bytes(partial_plan(dims, N, C, 2, 0, o));
            if (b > inner) inner = b;
        }
        inner = align256(align256(kStatusBytes) + inner);
        if (N == 3) {
            const size_t m2 = split_mttkrp_bytes(dims, N, C, 2, o);
            if (m2 > inner) inner = m2;
        }
        return align256(kStatusBytes) + align256(t) + inner;
    }
    size_t w = 0;
    for (int n = 0; n < N; ++n) {
        const size_t b = split_mttkrp_bytes(dims, N, C, n, o);
        if (b > w) w = b;
    }
    return w;
}
mtk_opts all_opts(const mtk_opts& o) {
    mtk_opts q = o;
    q.algo = MTK_ALGO_FUSED;
    return q;
}
}  // namespace

size_t mtk_mttkrp_all_split_workspace(const int64_t* dims, int N, int C, const mtk_opts* opts) {
    for (int n = 0; n < N; ++n)
        if (check_shape(dims, N, C, n) != MTK_OK) return 0;
    if (check_split_opts(opts, true) != MTK_OK) return 0;
    const mtk_opts o = defaults(opts);
    for (int n = 0; n < N; ++n)
        if (!planes_for(dims, N, C, n, all_opts(o)).ok) return 0;
    return all_split_bytes(dims, N, C, o);
}

int mtk_mttkrp_all_split(const void* Xs, const int64_t* dims, int N, const float* const* U, int C,
                         float* const* M, void* ws, size_t ws_bytes, const mtk_opts* opts, void* stream) {
    for (int n = 0; n < N; ++n) {
        const int st = check_shape(dims, N, C, n);
        if (st) return st;
    }
    if (!Xs || !aligned16(Xs) || !U || !M || !ws) return MTK_EINVAL;
    for (int k = 0; k < N; ++k)
        if (!U[k] || !aligned4(U[k]) || !M[k] || !aligned4(M[k])) return MTK_EINVAL;
    if (check_split_opts(opts, true) != MTK_OK) return MTK_EINVAL;
    const mtk_opts o = defaults(opts);
    const mtk_opts om = all_opts(o);
    for (int n = 0; n < N; ++n)
        if (!planes_for(dims, N, C, n, om).ok) return MTK_EUNSUPPORTED;
    if (ws_bytes < all_split_bytes(dims, N, C, o)) return MTK_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* status = static_cast<uint32_t*>(ws);
    if (!all_tree(dims, N, C, o)) {
        for (int n = 0; n < N; ++n) {
            const int st = do_mttkrp_split(Xs, nullptr, dims, N, U, C, n, M[n], ws, ws_bytes, status, om, s);
            if (st) return st;
        }
        return MTK_OK;
    }
    Carve cv{static_cast<char*>(ws), kStatusBytes, ws_bytes};
    const int64_t rest = tree_rest(dims, N);
    float* TR = static_cast<float*>(cv.take((size_t)dims[0] * dims[1] * C * sizeof(float) +
                                            (N >= 4 ? (size_t)rest * C * sizeof(float) : 0)));
    float* TL = N >= 4 ? TR + (size_t)dims[0] * dims[1] * C : nullptr;
    float* buf[2] = {nullptr, nullptr};
    if (N >= 5) {
        buf[0] = static_cast<float*>(cv.take((size_t)rest * C * sizeof(float)));
        buf[1] = static_cast<float*>(cv.take((size_t)rest * C * sizeof(float)));
    }
    // the inner calls carve their scratch after the status word of this block
    char* inner = static_cast<char*>(cv.take(0)) - kStatusBytes;
    const size_t inner_bytes = ws_bytes - (size_t)(inner - static_cast<char*>(ws));
    // modes 0, 1 from the contraction over modes >= 2 (Algorithm 4: partial, then multi-TTV)
    int st = run_tree_partial(Xs, dims, N, U, C, 1, TR, inner, status, om, s, nullptr, 0);
    if (st) return st;
    if (launch_multi_ttv(TR, 1, dims[0], dims[1], U[1], C, 0, M[0], s) != cudaSuccess ||
        launch_multi_ttv(TR, dims[0], dims[1], 1, U[0], C, 1, M[1], s) != cudaSuccess)
        return MTK_ECUDA;
    if (N == 3) return do_mttkrp_split(Xs, nullptr, dims, N, U, C, 2, M[2], inner, inner_bytes, status, om, s);
    // modes 2.. from the contraction over modes 0, 1
    st = run_tree_partial(Xs, dims, N, U, C, 0, TL, inner, status, om, s, nullptr, 0);
    if (st) return st;
    if (N == 4) {
        if (launch_multi_ttv(TL, 1, dims[2], dims[3], U[3], C, 0, M[2], s) != cudaSuccess ||
            launch_multi_ttv(TL, dims[2], dims[3], 1, U[2], C, 1, M[3], s) != cudaSuccess)
            return MTK_ECUDA;
        return MTK_OK;
    }
    // N >= 5: for each n >= 2, contract T_L's other modes one at a time (the last mode
    // other than n, else the first), ping-ponging between two buffers; the last step
    // writes M_n row-major
    for (int n = 2; n < N; ++n) {
        int ms[MTK_MAXN];
        int nm = 0;
        for (int k = 2; k < N; ++k) ms[nm++] = k;
        const float* cur = TL;
        int b = 0;
        while (nm > 1) {
            const int p = ms[nm - 1] != n ? nm - 1 : 0;
            int64_t A = 1, B = 1;
            for (int q = 0; q < p; ++q) A *= dims[ms[q]];
            for (int q = p + 1; q < nm; ++q) B *= dims[ms[q]];
            const bool last = nm == 2;
            float* dst = last ? M[n] : buf[b];
            if (launch_ttv_mode(cur, A, dims[ms[p]], B, U[ms[p]], C, dst, last ? 1 : 0, s) != cudaSuccess)
                return MTK_ECUDA;
            for (int q = p; q + 1 < nm; ++q) ms[q] = ms[q + 1];
            --nm;
            cur = dst;
            b ^= 1;
        }
    }
    return MTK_OK;
}

// ---- FP32 FMA throughput probe ---------------------------------------------------------------
int64_t mtk_ffma_probe_out_floats(int ctas_per_sm) {
    if (ctas_per_sm < 1 || ctas_per_sm > 64) return 0;
    return (int64_t)num_sms() * ctas_per_sm * ffma_probe_threads();
}

int mtk_ffma_probe(int ctas_per_sm, int iters, float* out, double* flops, void* stream) {
    if (ctas_per_sm < 1 || ctas_per_sm > 64 || iters < 1 || iters > (1 << 24) || !out || !aligned4(out))
        return MTK_EINVAL;
    const int blocks = num_sms() * ctas_per_sm;
    if (flops) *flops = 2.0 * 8.0 * (double)iters * (double)blocks * ffma_probe_threads();
    if (launch_ffma_probe(blocks, iters, out, (cudaStream_t)stream) != cudaSuccess) return MTK_ECUDA;
    return MTK_OK;
}

// ---- tensors symmetric in modes 0 and 1, packed ------------------------------------------
namespace {
// the packed tensor's dims (Pp, dims[2], ..., dims[N-1]) and its mode for full mode n
int sym_packed_dims(const int64_t* dims, int N, int diag, int64_t* pd) {
    pd[0] = sym_packed_rows(dims[0], diag);
    for (int k = 2; k < N; ++k) pd[k - 1] = dims[k];
    return N - 1;
}
bool sym_shape_ok(const int64_t* dims, int N, int diag, int C, int n) {
    return check_shape(dims, N, C, n) == MTK_OK && N >= 3 && dims[0] == dims[1] && (diag == 0 || diag == 1);
}
// status, then W or V (Pp x C), then the packed MTTKRP's workspace
size_t sym_bytes(const int64_t* dims, int N, int diag, int C, int n, const mtk_opts& o) {
    int64_t pd[MTK_MAXN];
    const int Np = sym_packed_dims(dims, N, diag, pd);
    const int np = n >= 2 ? n - 1 : 0;
    if (!planes_for(pd, Np, C, np, o).ok) return 0;
    return align256(kStatusBytes) + align256((size_t)pd[0] * C * sizeof(float)) +
           split_mttkrp_bytes(pd, Np, C, np, o);
}
}  // namespace

int64_t mtk_sym_packed_rows(int64_t n0, int diag) {
    return n0 < 1 || (diag != 0 && diag != 1) ? 0 : sym_packed_rows(n0, diag);
}

int mtk_pack_symmetric(const float* X, const int64_t* dims, int N, int diag, float* Xp, void* stream) {
    if (!X || !Xp || !aligned4(X) || !aligned4(Xp) || !sym_shape_ok(dims, N, diag, 1, 0)) return MTK_EINVAL;
    int64_t rest = 1;
    for (int k = 2; k < N; ++k) rest *= dims[k];
    if (launch_sym_pack(X, dims[0], diag, rest, Xp, (cudaStream_t)stream) != cudaSuccess) return MTK_ECUDA;
    return MTK_OK;
}

size_t mtk_mttkrp_sym_split_workspace(const int64_t* dims, int N, int diag, int C, int n, const mtk_opts* opts) {
    if (!sym_shape_ok(dims, N, diag, C, n) || check_split_opts(opts) != MTK_OK) return 0;
    return sym_bytes(dims, N, diag, C, n, defaults(opts));
}

int mtk_mttkrp_sym_split(const void* Xps, const int64_t* dims, int N, int diag, const float* const* U, int C, int n,
                         float* M, void* ws, size_t ws_bytes, const mtk_opts* opts, void* stream) {
    if (!sym_shape_ok(dims, N, diag, C, n)) return MTK_EINVAL;
    if (!Xps || !aligned16(Xps)) return MTK_EINVAL;
    int st = check_mttkrp_ptrs(static_cast<const float*>(Xps), U, N, n, M, ws);
    if (st) return st;
    if (n < 2 && !U[1 - n]) return MTK_EINVAL;
    if (check_split_opts(opts) != MTK_OK) return MTK_EINVAL;
    const mtk_opts o = defaults(opts);
    const size_t need = sym_bytes(dims, N, diag, C, n, o);
    if (need == 0) return MTK_EUNSUPPORTED;
    if (ws_bytes < need) return MTK_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t pd[MTK_MAXN];
    const int Np = sym_packed_dims(dims, N, diag, pd);
    Carve cv{static_cast<char*>(ws), kStatusBytes, ws_bytes};
    float* buf = static_cast<float*>(cv.take((size_t)pd[0] * C * sizeof(float)));
    const size_t inner_bytes = split_mttkrp_bytes(pd, Np, C, n >= 2 ? n - 1 : 0, o);
    void* inner = cv.take(inner_bytes);
    uint32_t* status = static_cast<uint32_t*>(ws);
    const float* Up[MTK_MAXN];
    for (int k = 2; k < N; ++k) Up[k - 1] = U[k];
    if (n >= 2) {
        // W, the symmetrised pair products, as the packed mode's factor
        if (launch_sym_pair(U[0], U[1], dims[0], diag, C, buf, s) != cudaSuccess) return MTK_ECUDA;
        Up[0] = buf;
        return do_mttkrp_split(Xps, nullptr, pd, Np, Up, C, n - 1, M, inner, inner_bytes, status, o, s);
    }
    Up[0] = nullptr;
    st = do_mttkrp_split(Xps, nullptr, pd, Np, Up, C, 0, buf, inner, inner_bytes, status, o, s);
    if (st) return st;
    if (launch_sym_ttv(buf, U[1 - n], dims[0], diag, C, M, s) != cudaSuccess) return MTK_ECUDA;
    return MTK_OK;
}

static int check_batch(const mtk_batch_problem* probs, int P) {
    if (!probs || P < 1 || P > MTK_BATCH_MAXP || P > batched_max_problems()) return MTK_EINVAL;
    for (int p = 0; p < P; ++p) {
        const mtk_batch_problem& q = probs[p];
        if (q.N < 2 || q.N > MTK_BATCH_MAXN || q.n < 0 || q.n >= q.N || q.C < 1 || q.C > 32) return MTK_EINVAL;
        if (!q.X || !q.M || !aligned4(q.X) || !aligned4(q.M)) return MTK_EINVAL;
        int64_t K = 1;
        for (int k = 0; k < q.N; ++k) {
            if (q.dims[k] < 1 || q.dims[k] >= ((int64_t)1 << 31)) return MTK_EINVAL;
            if (k == q.n) continue;
            if (!q.U[k] || !aligned4(q.U[k])) return MTK_EINVAL;
            K *= q.dims[k];
            if (K >= ((int64_t)1 << 31)) return MTK_EINVAL;
        }
    }
    return MTK_OK;
}

size_t mtk_mttkrp_batched_workspace(const mtk_batch_problem* probs, int P, const mtk_opts* opts) {
    if (check_batch(probs, P) != MTK_OK) return 0;
    const mtk_opts o = defaults(opts);
    const size_t f = batched_scratch_floats(probs, P, o.splits, 2 * planes_ctas(0));
    if (f == (size_t)-1) return 0;
    return align256(kStatusBytes) + align256(f * sizeof(float));
}

int mtk_mttkrp_batched(const mtk_batch_problem* probs, int P, void* ws, size_t ws_bytes, const mtk_opts* opts,
                       void* stream) {
    int st = check_batch(probs, P);
    if (st) return st;
    if (!ws) return MTK_EINVAL;
    const mtk_opts o = defaults(opts);
    if (ws_bytes < mtk_mttkrp_batched_workspace(probs, P, opts)) return MTK_EWORKSPACE;
    float* scratch = reinterpret_cast<float*>(static_cast<char*>(ws) + align256(kStatusBytes));
    if (launch_batched(probs, P, o.splits, 2 * planes_ctas(0), scratch, (cudaStream_t)stream) != cudaSuccess)
        return MTK_ECUDA;
    return MTK_OK;
}

size_t mtk_partial_mttkrp_workspace(const int64_t* dims, int N, int C, int n, int right,
                                    const mtk_opts* opts) {
    if (check_shape(dims, N, C, n) != MTK_OK) return 0;
    mtk_opts o = defaults(opts);
    const View v = mode_view(dims, N, n);
    const int64_t Ip = right ? v.L * v.I : v.I * v.R;
    const int64_t Kp = right ? v.R : v.L;
    ContractPlan pl = plan_both(right ? 1 : v.L, Ip, &Kp, 1, C, o);
    return align256(align256(kStatusBytes) + plan_scratch(pl));
}

int mtk_partial_mttkrp(const float* X, const int64_t* dims, int N, const float* Kp, int C, int n,
                       int right, float* T, void* ws, size_t ws_bytes, const mtk_opts* opts,
                       void* stream) {
    int st = check_shape(dims, N, C, n);
    if (st) return st;
    if (!X || !Kp || !T || !ws || !aligned4(X) || !aligned4(Kp) || !aligned4(T)) return MTK_EINVAL;
    mtk_opts o = defaults(opts);
    if (o.precision < MTK_PREC_FP32 || o.precision > MTK_PREC_BF16X3) return MTK_EINVAL;
    if (ws_bytes < mtk_partial_mttkrp_workspace(dims, N, C, n, right, opts)) return MTK_EWORKSPACE;
    const View v = mode_view(dims, N, n);
    ContractParams p;
    memset(&p, 0, sizeof(p));
    p.X = X; p.C = C; p.status = static_cast<uint32_t*>(ws);
    if (right) {
        p.L = 1; p.I = v.L * v.I; p.R = v.R; p.K = v.R;
        p.W.f0 = Kp; p.W.rad0 = v.R;
        p.out = T; p.out_si = 1; p.out_sc = v.L * v.I;
    } else {
        p.L = v.L; p.I = v.I * v.R; p.R = 1; p.K = v.L;
        p.W.f0 = Kp; p.W.rad0 = v.L;
        p.out = T; p.out_si = 1; p.out_sc = v.I * v.R;
    }
    const float* kf = Kp;
    set_factors(p, &kf, &p.K, 1);
    ContractPlan pl = plan_for(p.L, p.I, p.frad, p.nfac, C, o, aligned16(X));
    Carve cv{static_cast<char*>(ws), kStatusBytes, ws_bytes};
    return run_contract(p, pl, o.precision, cv.take(plan_scratch(pl)), (cudaStream_t)stream);
}

int mtk_multi_ttv(const float* T, const int64_t* dims, int N, const float* Ko, int C, int n,
                  int right, float* M, void* stream) {
    int st = check_shape(dims, N, C, n);
    if (st) return st;
    if (!T || !Ko || !M || !aligned4(T) || !aligned4(Ko) || !aligned4(M)) return MTK_EINVAL;
    const View v = mode_view(dims, N, n);
    if (launch_multi_ttv(T, v.L, v.I, v.R, Ko, C, right ? 1 : 0, M, (cudaStream_t)stream) !=
        cudaSuccess)
        return MTK_ECUDA;
    return MTK_OK;
}

size_t mtk_gram_workspace(int64_t I, int C) {
    if (I < 1 || C < 1 || C > MTK_MAXC) return 0;
    const int nch = gram_chunks(I);
    return align256(kStatusBytes) + align256((size_t)(nch > 1 ? nch : 0) * C * C * sizeof(double));
}

int mtk_gram(const float* U, int64_t I, int C, double* G, void* ws, size_t ws_bytes, void* stream) {
    if (!U || !G || !ws || I < 1 || C < 1 || C > MTK_MAXC || !aligned4(U)) return MTK_EINVAL;
    if (ws_bytes < mtk_gram_workspace(I, C)) return MTK_EWORKSPACE;
    double* part = reinterpret_cast<double*>(static_cast<char*>(ws) + align256(kStatusBytes));
    if (launch_gram(U, I, C, G, part, gram_chunks(I), (cudaStream_t)stream) != cudaSuccess)
        return MTK_ECUDA;
    return MTK_OK;
}

size_t mtk_solve_workspace(int64_t In, int C) {
    if (In < 1 || C < 1 || C > MTK_MAXC) return 0;
    if (als_update_supported(C))            // status, tickets, the update's scratch
        return align256(kStatusBytes) + align256(als_ticket_bytes()) +
               align256(als_update_scratch_bytes(als_update_ctas(In, nullptr), C));
    const int nch = gram_chunks(In);
    return align256(kStatusBytes) + align256(solve_scratch_doubles(C) * sizeof(double)) + 256 +
           align256((size_t)(nch > 1 ? nch : 0) * C * C * sizeof(double));
}

int mtk_gram_hadamard_solve(const double* const* G, int N, int C, int n, const float* M,
                            int64_t In, float* Un, double* Gn, void* ws, size_t ws_bytes,
                            void* stream) {
    if (!G || !M || !Un || !ws || N < 2 || N > MTK_MAXN || n < 0 || n >= N || C < 1 ||
        C > MTK_MAXC || In < 1)
        return MTK_EINVAL;
    for (int k = 0; k < N; ++k)
        if (k != n && !G[k]) return MTK_EINVAL;
    if (ws_bytes < mtk_solve_workspace(In, C)) return MTK_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = static_cast<char*>(ws);
    if (als_update_supported(C)) {
        unsigned int* tick = reinterpret_cast<unsigned int*>(w + align256(kStatusBytes));
        void* scratch = w + align256(kStatusBytes) + align256(als_ticket_bytes());
        AlsUpdateArgs a;
        memset(&a, 0, sizeof(a));
        a.G = G;
        a.N = N;
        a.C = C;
        a.n = n;
        a.M = M;
        a.In = In;
        a.Un = Un;
        a.Gn = Gn;
        a.scratch = scratch;
        a.Pmax = als_update_ctas(In, nullptr);
        a.tickets = tick;
        a.status = static_cast<uint32_t*>(ws);
        if (cudaMemsetAsync(tick, 0, als_ticket_bytes(), s) != cudaSuccess || launch_als_update(a, s) != cudaSuccess)
            return MTK_ECUDA;
        return MTK_OK;
    }
    double* Hbuf = reinterpret_cast<double*>(w + align256(kStatusBytes));
    int* flag = reinterpret_cast<int*>(w + align256(kStatusBytes) + align256(solve_scratch_doubles(C) * sizeof(double)));
    if (launch_chol_solve(G, N, C, n, M, In, Un, Hbuf, flag, static_cast<uint32_t*>(ws), s) !=
        cudaSuccess)
        return MTK_ECUDA;
    if (Gn) {
        double* gpart = reinterpret_cast<double*>(w + align256(kStatusBytes) +
                                                  align256(solve_scratch_doubles(C) * sizeof(double)) + 256);
        if (launch_gram(Un, In, C, Gn, gpart, gram_chunks(In), s) != cudaSuccess) return MTK_ECUDA;
    }
    return MTK_OK;
}

size_t mtk_norm2_workspace(int64_t I) {
    if (I < 1) return 0;
    return align256(kStatusBytes) + align256((size_t)norm2_chunks(I) * sizeof(double));
}

int mtk_norm2(const float* X, int64_t I, double* out, void* ws, size_t ws_bytes, void* stream) {
    if (!X || !out || !ws || I < 1 || !aligned4(X)) return MTK_EINVAL;
    if (ws_bytes < mtk_norm2_workspace(I)) return MTK_EWORKSPACE;
    double* part = reinterpret_cast<double*>(static_cast<char*>(ws) + align256(kStatusBytes));
    if (launch_norm2(X, I, part, norm2_chunks(I), out, (cudaStream_t)stream) != cudaSuccess)
        return MTK_ECUDA;
    return MTK_OK;
}

// --- CP-ALS sweep ----------------------------------------------------------------
namespace {
struct AlsLayout {
    size_t mbuf, gbufs, gpart, hbuf, flag, upd, tick, hinv, mt, tree, total;
    int maxIn;
    int reserve;                // SMs the planes contractions leave to an overlapped factorisation
};

// split = 1: the MTTKRPs read the tensor's BF16 planes (mtk_cp_als_sweep_split);
// split = 2: the same with the dimension tree
AlsLayout als_layout(const int64_t* dims, int N, int C, const mtk_opts& o, int split) {
    AlsLayout a;
    memset(&a, 0, sizeof(a));
    int64_t maxIn = 0, maxChunks = 1;
    size_t mt = 0;
    // on the planes, a mode's factorisation H_n^{-1} runs alongside its contraction on an SM
    // the contraction leaves free (one-launch updates only)
    a.reserve = (split && als_update_supported(C)) ? 1 : 0;
    for (int k = 0; k < N; ++k) {
        if (dims[k] > maxIn) maxIn = dims[k];
        const int ch = gram_chunks(dims[k]);
        if (ch > maxChunks) maxChunks = ch;
        const size_t w = split ? split_mttkrp_bytes(dims, N, C, k, o, a.reserve) : mttkrp_layout(dims, N, C, k, o).total;
        if (w > mt) mt = w;
    }
    a.maxIn = (int)maxIn;
    Carve cv{nullptr, kStatusBytes, 0};
    a.mbuf = (size_t)maxIn * C * sizeof(float); cv.take(a.mbuf);
    a.gbufs = (size_t)N * C * C * sizeof(double); cv.take(a.gbufs);
    a.gpart = (maxChunks > 1 && !als_update_supported(C)) ? (size_t)maxChunks * C * C * sizeof(double) : 0;
    cv.take(a.gpart);
    a.hbuf = solve_scratch_doubles(C) * sizeof(double); cv.take(a.hbuf);
    a.flag = 256; cv.take(a.flag);
    if (als_update_supported(C)) {                      // one-launch updates and Grams
        size_t u = gram_all_scratch_bytes(dims, N, C);
        const size_t b = als_update_scratch_bytes(als_update_max_ctas(dims, N), C);
        a.upd = u > b ? u : b;
        a.tick = als_ticket_bytes();
        if (a.reserve) a.hinv = als_hinv_bytes(C);
    }
    cv.take(a.upd);
    cv.take(a.tick);
    cv.take(a.hinv);
    if (split == 2) {                                   // dimension tree: partials T_R, T_L
        const size_t ts = tree_scratch(dims, N, C, o, a.reserve);
        if (ts > mt) mt = ts;
        a.tree = (size_t)(dims[0] * dims[1] + (N == 4 ? dims[2] * dims[3] : 0)) * C * sizeof(float);
    }
    a.mt = mt; cv.take(a.mt);
    cv.take(a.tree);
    a.total = align256(cv.off);
    return a;
}
}  // namespace

size_t mtk_cp_als_workspace(const int64_t* dims, int N, int C, const mtk_opts* opts) {
    for (int n = 0; n < N; ++n)
        if (check_shape(dims, N, C, n) != MTK_OK) return 0;
    if (N < 2) return 0;
    mtk_opts o = defaults(opts);
    if (o.algo < 0) return 0;
    const size_t a = als_layout(dims, N, C, o, 0).total;
    size_t b = 0;
    if (check_split_opts(opts, true) == MTK_OK) {
        b = als_layout(dims, N, C, o, 1).total;
        if (tree_shape(dims, N, C)) {
            const size_t t = als_layout(dims, N, C, o, 2).total;
            if (t > b) b = t;
        }
    }
    return a > b ? a : b;
}

namespace {
// one sweep; Xs = NULL: MTTKRPs on the FP32 tensor, else on its BF16 planes (X may
// then be NULL if every mode is taken by the planes kernel)
int als_sweep(const float* X, const void* Xs, const int64_t* dims, int N, float* const* U, int C,
              const double* normX2, double* fit, void* ws, size_t ws_bytes, const mtk_opts* opts,
              void* stream) {
    if (N < 2) return MTK_EINVAL;
    for (int n = 0; n < N; ++n) {
        int st = check_shape(dims, N, C, n);
        if (st) return st;
    }
    if ((!X && !Xs) || !U || !ws || (X && !aligned4(X)) || (Xs && !aligned16(Xs))) return MTK_EINVAL;
    for (int k = 0; k < N; ++k)
        if (!U[k] || !aligned4(U[k])) return MTK_EINVAL;
    if (fit && !normX2) return MTK_EINVAL;
    mtk_opts o = defaults(opts);
    if (o.algo < 0 || o.precision < MTK_PREC_FP32 || o.precision > MTK_PREC_BF16X3) return MTK_EINVAL;
    if (Xs && check_split_opts(opts, true) != MTK_OK) return MTK_EINVAL;
    if (o.normalize < 0 || o.normalize > 1) return MTK_EINVAL;
    if (o.normalize && !als_update_supported(C)) return MTK_EUNSUPPORTED;
    const int split_form = Xs ? 1 : 0;
    const bool tree = Xs && o.algo == MTK_ALGO_TWO_STEP && tree_ok(dims, N, C, o, als_layout(dims, N, C, o, split_form).reserve);
    const AlsLayout a = als_layout(dims, N, C, o, tree ? 2 : split_form);
    if (ws_bytes < a.total) return MTK_EWORKSPACE;
    const mtk_opts om = [&]() {                         // per-mode MTTKRPs of a split sweep
        mtk_opts q = o;
        if (Xs) q.algo = MTK_ALGO_FUSED;
        return q;
    }();
    cudaStream_t s = (cudaStream_t)stream;
    Carve cv{static_cast<char*>(ws), kStatusBytes, ws_bytes};
    uint32_t* status = static_cast<uint32_t*>(ws);
    float* M = static_cast<float*>(cv.take(a.mbuf));
    double* Gall = static_cast<double*>(cv.take(a.gbufs));
    double* gpart = static_cast<double*>(cv.take(a.gpart));
    double* Hbuf = static_cast<double*>(cv.take(a.hbuf));
    int* flag = static_cast<int*>(cv.take(a.flag));
    void* upd = cv.take(a.upd);
    unsigned int* tick = static_cast<unsigned int*>(cv.take(a.tick));
    void* hinv = cv.take(a.hinv);
    char* mws = static_cast<char*>(cv.take(a.mt));
    const double* G[MTK_MAXN];
    for (int k = 0; k < N; ++k) G[k] = Gall + (size_t)k * C * C;
    const bool fused = als_update_supported(C);
    if (fused) {
        // Grams of all factors in one launch; every later update leaves the tickets at zero
        double* Gw[MTK_MAXN];
        for (int k = 0; k < N; ++k) Gw[k] = const_cast<double*>(G[k]);
        if (cudaMemsetAsync(tick, 0, a.tick, s) != cudaSuccess ||
            launch_gram_all(U, dims, N, C, Gw, upd, tick, s) != cudaSuccess)
            return MTK_ECUDA;
    } else {
        for (int k = 0; k < N; ++k)
            if (launch_gram(U[k], dims[k], C, const_cast<double*>(G[k]), gpart, gram_chunks(dims[k]), s) !=
                cudaSuccess)
                return MTK_ECUDA;
    }
    float* TR = tree ? reinterpret_cast<float*>(cv.take(a.tree)) : nullptr;
    float* TL = tree && N == 4 ? TR + (size_t)dims[0] * dims[1] * C : nullptr;
    for (int n = 0; n < N; ++n) {
        int st = MTK_OK;
        // H_n^{-1} formed alongside this mode's planes contraction (when it has one of its own)
        FactorHook hk{G, N, C, n, hinv, status};
        const FactorHook* hook = a.reserve ? &hk : nullptr;
        bool hooked = false;
        if (tree && n < 2) {
            // modes 0 and 1 from the right partial (computed once, with U_2.. as they are)
            if (n == 0) {
                st = run_tree_partial(Xs, dims, N, U, C, 1, TR, mws, status, om, s, hook, a.reserve);
                hooked = hook != nullptr;
                if (!st && launch_multi_ttv(TR, 1, dims[0], dims[1], U[1], C, 0, M, s) != cudaSuccess) st = MTK_ECUDA;
            } else if (launch_multi_ttv(TR, dims[0], dims[1], 1, U[0], C, 1, M, s) != cudaSuccess) {
                st = MTK_ECUDA;
            }
        } else if (tree && N == 4) {
            // modes 2 and 3 from the left partial (with the updated U_0, U_1)
            if (n == 2) {
                st = run_tree_partial(Xs, dims, N, U, C, 0, TL, mws, status, om, s, hook, a.reserve);
                hooked = hook != nullptr;
                if (!st && launch_multi_ttv(TL, 1, dims[2], dims[3], U[3], C, 0, M, s) != cudaSuccess) st = MTK_ECUDA;
            } else if (launch_multi_ttv(TL, dims[2], dims[3], 1, U[2], C, 1, M, s) != cudaSuccess) {
                st = MTK_ECUDA;
            }
        } else {
            st = Xs ? do_mttkrp_split(Xs, X, dims, N, U, C, n, M, mws, a.mt, status, om, s, hook, a.reserve, &hooked)
                    : do_mttkrp(X, dims, N, U, C, n, M, mws, a.mt, status, o, s);
        }
        if (st) return st;
        if (fused) {
            // U_n in one launch whose factorisation of H (and H^{-1}) overlaps the kernel
            // before it; the launch also reduces the Gram of the new U_n into G_n, which
            // the next update reads, and the last mode's computes the fit.
            AlsUpdateArgs ua;
            memset(&ua, 0, sizeof(ua));
            ua.G = G;
            ua.N = N;
            ua.C = C;
            ua.n = n;
            ua.M = M;
            ua.In = dims[n];
            ua.Un = U[n];
            const bool last = n == N - 1;
            ua.Gn = const_cast<double*>(G[n]);
            ua.scratch = upd;
            ua.Pmax = als_update_max_ctas(dims, N);
            ua.tickets = tick;
            ua.normX2 = last ? normX2 : nullptr;
            ua.fit = last ? fit : nullptr;
            ua.status = status;
            ua.programmatic = true;
            ua.hinv = hooked ? hinv : nullptr;
            ua.normalize = o.normalize != 0 && !last;
            if (launch_als_update(ua, s) != cudaSuccess) return MTK_ECUDA;
            continue;
        }
        if (launch_chol_solve(G, N, C, n, M, dims[n], U[n], Hbuf, flag, status, s) != cudaSuccess)
            return MTK_ECUDA;
        if (launch_gram(U[n], dims[n], C, const_cast<double*>(G[n]), gpart, gram_chunks(dims[n]), s) !=
            cudaSuccess)
            return MTK_ECUDA;
    }
    if (fit && !fused) {
        if (launch_residual(normX2, M, U[N - 1], dims[N - 1], G, N, C, nullptr, fit, s) !=
            cudaSuccess)
            return MTK_ECUDA;
    }
    return MTK_OK;
}
}  // namespace

int mtk_cp_als_sweep(const float* X, const int64_t* dims, int N, float* const* U, int C,
                     const double* normX2, double* fit, void* ws, size_t ws_bytes,
                     const mtk_opts* opts, void* stream) {
    if (!X) return MTK_EINVAL;
    return als_sweep(X, nullptr, dims, N, U, C, normX2, fit, ws, ws_bytes, opts, stream);
}

int mtk_cp_als_sweep_split(const void* Xs, const float* X, const int64_t* dims, int N, float* const* U,
                           int C, const double* normX2, double* fit, void* ws, size_t ws_bytes,
                           const mtk_opts* opts, void* stream) {
    if (!Xs) return MTK_EINVAL;
    const float* Xv = nullptr;
    if (X) {
        const int st = device_view(X, &Xv);
        if (st) return st;
    }
    return als_sweep(Xv, Xs, dims, N, U, C, normX2, fit, ws, ws_bytes, opts, stream);
}

int mtk_cp_residual(const double* normX2, const float* M, const float* Um, int64_t Im,
                    const double* const* G, int N, int C, double* r2, double* fit, void* stream) {
    if (!normX2 || !M || !Um || !G || N < 2 || N > MTK_MAXN || C < 1 || C > MTK_MAXC || Im < 1)
        return MTK_EINVAL;
    for (int k = 0; k < N; ++k)
        if (!G[k]) return MTK_EINVAL;
    if (launch_residual(normX2, M, Um, Im, G, N, C, r2, fit, (cudaStream_t)stream) != cudaSuccess)
        return MTK_ECUDA;
    return MTK_OK;
}

int mtk_cp_loss(const double* normX2, const float* M, const float* Um, int64_t Im,
                const double* const* G, int N, int C, float* loss, void* stream) {
    if (!normX2 || !M || !Um || !G || !loss || N < 2 || N > MTK_MAXN || C < 1 || C > MTK_MAXC || Im < 1)
        return MTK_EINVAL;
    for (int k = 0; k < N; ++k)
        if (!G[k]) return MTK_EINVAL;
    if (launch_residual(normX2, M, Um, Im, G, N, C, nullptr, nullptr, (cudaStream_t)stream, loss) != cudaSuccess)
        return MTK_ECUDA;
    return MTK_OK;
}

int mtk_cp_gradient(const float* Un, const float* Mn, const double* const* G, int N, int C, int n,
                    int64_t In, const float* scale, float* grad, void* stream) {
    if (!Un || !Mn || !G || !grad || N < 2 || N > MTK_MAXN || n < 0 || n >= N || C < 1 ||
        C > MTK_MAXC || In < 1)
        return MTK_EINVAL;
    for (int k = 0; k < N; ++k)
        if (k != n && !G[k]) return MTK_EINVAL;
    if (launch_gradient(Un, Mn, G, N, C, n, In, scale, grad, (cudaStream_t)stream) != cudaSuccess)
        return MTK_ECUDA;
    return MTK_OK;
}

}  // extern "C"
