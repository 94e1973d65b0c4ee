/*
 * oracle.c -- plain, slow, FP64 CPU reference for dense MTTKRP and CP-ALS.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path (paper_1708_08976_gb300/csrc).
 *
 * Conventions (from "Shared-Memory Parallelization of MTTKRP for Dense
 * Tensors", Hayashi, Ballard, Jiang, Tobia, 2017):
 *   - indices are 0-based (Section 2.1, Notation);
 *   - a tensor with dims I_0..I_{N-1} is stored in the natural linearization
 *     l = sum_k i_k * prod_{j<k} I_j, mode 0 fastest (Section 2.1);
 *   - factor matrices U_k are I_k x C, stored row-major (C contiguous);
 *     the paper does not fix this, we state it;
 *   - MTTKRP output M is I_n x C row-major.
 *
 * Every floating-point value is double.  Sums over the tensor are split into
 * ORACLE_CHUNKS fixed contiguous ranges of the linear index, each summed in
 * order, then the chunk results are added in chunk order, so the result does
 * not depend on the number of OpenMP threads.
 *
 * Pins: the test suite checks every function here against brute force
 * (explicit matricization times an explicit Kronecker-defined KRP), closed
 * forms for tensors built from known factors, textbook special cases (N=2 is
 * a matrix product, C=1 is a chain of TTVs), finite differences, and
 * hand-derived integer examples.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_CHUNKS 64
#define ORACLE_MAXN 16

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ENOTPD = 4 };

/* number of OpenMP threads this library will use (1 without OpenMP) */
int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

static int64_t prod_dims(const int64_t* dims, int a, int b) {
    int64_t p = 1;
    for (int k = a; k < b; ++k) p *= dims[k];
    return p;
}

/* decompose linear index l into the multi-index (mode 0 fastest, Section 2.1) */
static void unravel(int64_t l, const int64_t* dims, int N, int64_t* idx) {
    for (int k = 0; k < N; ++k) { idx[k] = l % dims[k]; l /= dims[k]; }
}

/* advance the multi-index by one in the natural order */
static void increment(int64_t* idx, const int64_t* dims, int N) {
    for (int k = 0; k < N; ++k) {
        if (++idx[k] < dims[k]) return;
        idx[k] = 0;
    }
}

static int check_args(const int64_t* dims, int N, int C, int n) {
    if (N < 1 || N > ORACLE_MAXN || C < 1 || n < 0 || n >= N) return OR_EINVAL;
    for (int k = 0; k < N; ++k) if (dims[k] < 1) return OR_EINVAL;
    return OR_OK;
}

/*
 * Mode-n MTTKRP by its element-wise definition (Section 2.2, the MTTKRP
 * bullet: M = X_(n) (U_{N-1} kr ... kr U_{n+1} kr U_{n-1} kr ... kr U_0)),
 * written out entry by entry:
 *     M(i_n, c) = sum over all entries X(i_0..i_{N-1}) * prod_{k != n} U_k(i_k, c).
 * Only the entries with linear index in [l_begin, l_end) contribute; pass
 * 0 and prod(dims) for the full MTTKRP.  X points at entry l_begin.
 * U[n] is not read.
 */
int oracle_mttkrp_range(const double* X, const int64_t* dims, int N,
                        const double* const* U, int C, int n,
                        int64_t l_begin, int64_t l_end, double* M) {
    int st = check_args(dims, N, C, n);
    if (st) return st;
    const int64_t I = prod_dims(dims, 0, N);
    if (l_begin < 0 || l_end > I || l_begin > l_end) return OR_EINVAL;
    const int64_t In = dims[n];
    double* part = (double*)calloc((size_t)ORACLE_CHUNKS * In * C, sizeof(double));
    if (!part) return OR_ENOMEM;
    const int64_t span = l_end - l_begin;

    #pragma omp parallel for schedule(dynamic, 1)
    for (int ch = 0; ch < ORACLE_CHUNKS; ++ch) {
        int64_t a = l_begin + span * ch / ORACLE_CHUNKS;
        int64_t b = l_begin + span * (ch + 1) / ORACLE_CHUNKS;
        if (a >= b) continue;
        double* Mp = part + (size_t)ch * In * C;
        double* w = (double*)malloc(sizeof(double) * C);
        int64_t idx[ORACLE_MAXN];
        unravel(a, dims, N, idx);
        for (int64_t l = a; l < b; ++l) {
            for (int c = 0; c < C; ++c) w[c] = 1.0;
            for (int k = 0; k < N; ++k) {
                if (k == n) continue;
                const double* row = U[k] + idx[k] * C;
                for (int c = 0; c < C; ++c) w[c] *= row[c];
            }
            const double x = X[l - l_begin];
            double* out = Mp + idx[n] * C;
            for (int c = 0; c < C; ++c) out[c] += x * w[c];
            increment(idx, dims, N);
        }
        free(w);
    }
    memset(M, 0, sizeof(double) * In * C);
    for (int ch = 0; ch < ORACLE_CHUNKS; ++ch) {
        const double* Mp = part + (size_t)ch * In * C;
        for (int64_t e = 0; e < In * C; ++e) M[e] += Mp[e];
    }
    free(part);
    return OR_OK;
}

int oracle_mttkrp(const double* X, const int64_t* dims, int N,
                  const double* const* U, int C, int n, double* M) {
    int st = check_args(dims, N, C, n);
    if (st) return st;
    return oracle_mttkrp_range(X, dims, N, U, C, n, 0, prod_dims(dims, 0, N), M);
}

/*
 * Selected rows of the mode-n MTTKRP of an FP32 tensor (each entry promoted
 * exactly to double), by the same element-wise definition (Section 2.2):
 *     out[q, c] = sum over entries with i_n = rows[q] of X * prod_{k != n} U_k(i_k, c).
 * Used to check full-size results row by row.  out is nrows x C row-major.
 */
int oracle_mttkrp_rows_f32(const float* X, const int64_t* dims, int N,
                           const double* const* U, int C, int n,
                           const int64_t* rows, int nrows, double* out) {
    int st = check_args(dims, N, C, n);
    if (st) return st;
    const int64_t In = dims[n];
    const int64_t IL = prod_dims(dims, 0, n);      /* modes left of n  */
    const int64_t IR = prod_dims(dims, n + 1, N);  /* modes right of n */
    const int64_t Jn = IL * IR;                    /* entries with fixed i_n */
    for (int q = 0; q < nrows; ++q)
        if (rows[q] < 0 || rows[q] >= In) return OR_EINVAL;
    /* the entries sharing i_n are enumerated by the other modes' multi-index,
       lowest mode fastest; split that enumeration into fixed chunks */
    int64_t odims[ORACLE_MAXN];
    int No = 0;
    for (int k = 0; k < N; ++k) if (k != n) odims[No++] = dims[k];
    if (No == 0) { odims[0] = 1; No = 1; }
    double* part = (double*)calloc((size_t)ORACLE_CHUNKS * nrows * C, sizeof(double));
    if (!part) return OR_ENOMEM;

    #pragma omp parallel for schedule(dynamic, 1)
    for (int ch = 0; ch < ORACLE_CHUNKS; ++ch) {
        int64_t a = Jn * ch / ORACLE_CHUNKS, b = Jn * (ch + 1) / ORACLE_CHUNKS;
        if (a >= b) continue;
        double* w = (double*)malloc(sizeof(double) * C);
        int64_t oidx[ORACLE_MAXN];
        unravel(a, odims, No, oidx);
        for (int64_t j = a; j < b; ++j) {
            /* rebuild the full multi-index and the KRP row weight */
            int64_t lin_wo_n = 0, stride = 1;
            int o = 0;
            for (int c = 0; c < C; ++c) w[c] = 1.0;
            for (int k = 0; k < N; ++k) {
                if (k == n) { stride *= dims[k]; continue; }
                const int64_t ik = (N == 1) ? 0 : oidx[o++];
                lin_wo_n += ik * stride;
                stride *= dims[k];
                const double* row = U[k] + ik * C;
                for (int c = 0; c < C; ++c) w[c] *= row[c];
            }
            for (int q = 0; q < nrows; ++q) {
                const int64_t l = lin_wo_n + rows[q] * IL;
                const double x = (double)X[l];
                double* dst = part + ((size_t)ch * nrows + q) * C;
                for (int c = 0; c < C; ++c) dst[c] += x * w[c];
            }
            increment(oidx, odims, No);
        }
        free(w);
    }
    memset(out, 0, sizeof(double) * nrows * C);
    for (int ch = 0; ch < ORACLE_CHUNKS; ++ch)
        for (int64_t e = 0; e < (int64_t)nrows * C; ++e)
            out[e] += part[(size_t)ch * nrows * C + e];
    free(part);
    return OR_OK;
}

/*
 * Khatri-Rao product of Z matrices, row by row (Section 2.1 row-wise
 * definition; Section 4.1): K = U_0 kr U_1 kr ... kr U_{Z-1}, with
 * K(j, :) = U_0(a_0, :) * ... * U_{Z-1}(a_{Z-1}, :) and the LAST operand's row
 * index fastest: j = a_{Z-1} + J_{Z-1} * (a_{Z-2} + J_{Z-2} * (...)).
 * Every row is formed from scratch (no reuse of partial products), so this is
 * independent of the reuse scheme of Algorithm 1.  K is (prod J_z) x C row-major.
 */
int oracle_krp(const double* const* U, const int64_t* rows, int Z, int C, double* K) {
    if (Z < 1 || Z > ORACLE_MAXN || C < 1) return OR_EINVAL;
    int64_t J = 1;
    for (int z = 0; z < Z; ++z) { if (rows[z] < 1) return OR_EINVAL; J *= rows[z]; }
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < J; ++j) {
        int64_t a[ORACLE_MAXN], t = j;
        for (int z = Z - 1; z >= 0; --z) { a[z] = t % rows[z]; t /= rows[z]; }
        for (int c = 0; c < C; ++c) {
            double p = 1.0;
            for (int z = 0; z < Z; ++z) p *= U[z][a[z] * C + c];
            K[j * C + c] = p;
        }
    }
    return OR_OK;
}

/*
 * Brute-force MTTKRP: build X_(n) explicitly (I_n x I_{!=n}, column index =
 * linearization of the remaining modes with the lowest mode fastest, Section
 * 2.1), build the full KRP K = U_{N-1} kr ... kr U_{n+1} kr U_{n-1} kr ... kr U_0
 * (Section 4.1) explicitly with oracle_krp, and multiply with a triple loop
 * (Section 2.3, "the most straightforward way").  Tiny inputs only.
 */
int oracle_mttkrp_brute(const double* X, const int64_t* dims, int N,
                        const double* const* U, int C, int n, double* M) {
    int st = check_args(dims, N, C, n);
    if (st) return st;
    const int64_t In = dims[n];
    const int64_t I = prod_dims(dims, 0, N);
    const int64_t J = I / In;
    double* Xn = (double*)malloc(sizeof(double) * I);
    double* K = (double*)malloc(sizeof(double) * (J > 0 ? J : 1) * C);
    if (!Xn || !K) { free(Xn); free(K); return OR_ENOMEM; }
    /* explicit matricization */
    int64_t idx[ORACLE_MAXN];
    for (int64_t l = 0; l < I; ++l) {
        unravel(l, dims, N, idx);
        int64_t col = 0, stride = 1;
        for (int k = 0; k < N; ++k) {
            if (k == n) continue;
            col += idx[k] * stride;
            stride *= dims[k];
        }
        Xn[idx[n] + In * col] = X[l];   /* column-major I_n x J */
    }
    /* explicit KRP with operands U_{N-1}, ..., U_{n+1}, U_{n-1}, ..., U_0 */
    const double* ops[ORACLE_MAXN];
    int64_t rws[ORACLE_MAXN];
    int Z = 0;
    for (int k = N - 1; k >= 0; --k) {
        if (k == n) continue;
        ops[Z] = U[k];
        rws[Z] = dims[k];
        ++Z;
    }
    if (Z == 0) {            /* N == 1: the KRP of no matrices is a row of ones */
        for (int c = 0; c < C; ++c) K[c] = 1.0;
    } else {
        st = oracle_krp(ops, rws, Z, C, K);
        if (st) { free(Xn); free(K); return st; }
    }
    for (int64_t i = 0; i < In; ++i)
        for (int c = 0; c < C; ++c) {
            double s = 0.0;
            for (int64_t j = 0; j < J; ++j) s += Xn[i + In * j] * K[j * C + c];
            M[i * C + c] = s;
        }
    free(Xn);
    free(K);
    return OR_OK;
}

/*
 * Partial MTTKRPs of the 2-step algorithm (Section 4.3, Algorithm 4), each by
 * its element-wise definition.
 *   right: R_(0:n) = X_(0:n) K_R with K_R = U_{N-1} kr ... kr U_{n+1}, i.e.
 *          R(l, i, c) = sum_r X(l, i, r) K_R(r, c), stored in the natural
 *          order of the (I^L x I_n x C) tensor: R[l + I^L*i + I^L*I_n*c].
 *   left:  L_(0:N-n-1) = X_(0:n-1)^T K_L with K_L = U_{n-1} kr ... kr U_0, i.e.
 *          L(i, r, c) = sum_l X(l, i, r) K_L(l, c), stored as
 *          L[i + I_n*r + I_n*I^R*c].
 * Here l, r are the linear indices of modes < n and > n (lowest mode fastest).
 */
int oracle_partial_mttkrp(const double* X, const int64_t* dims, int N,
                          const double* const* U, int C, int n, int right, double* out) {
    int st = check_args(dims, N, C, n);
    if (st) return st;
    const int64_t IL = prod_dims(dims, 0, n), In = dims[n], IR = prod_dims(dims, n + 1, N);
    const int64_t I = IL * In * IR;
    const int64_t outsz = right ? IL * In * C : In * IR * C;
    double* part = (double*)calloc((size_t)ORACLE_CHUNKS * outsz, sizeof(double));
    if (!part) return OR_ENOMEM;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int ch = 0; ch < ORACLE_CHUNKS; ++ch) {
        int64_t a = I * ch / ORACLE_CHUNKS, b = I * (ch + 1) / ORACLE_CHUNKS;
        if (a >= b) continue;
        double* P = part + (size_t)ch * outsz;
        double* w = (double*)malloc(sizeof(double) * C);
        int64_t idx[ORACLE_MAXN];
        unravel(a, dims, N, idx);
        for (int64_t l = a; l < b; ++l) {
            const int64_t lidx = l % IL, ridx = l / (IL * In), i = idx[n];
            for (int c = 0; c < C; ++c) w[c] = 1.0;
            for (int k = right ? n + 1 : 0; k < (right ? N : n); ++k) {
                const double* row = U[k] + idx[k] * C;
                for (int c = 0; c < C; ++c) w[c] *= row[c];
            }
            const double x = X[l];
            if (right) {
                for (int c = 0; c < C; ++c) P[lidx + IL * i + IL * In * c] += x * w[c];
            } else {
                for (int c = 0; c < C; ++c) P[i + In * ridx + In * IR * c] += x * w[c];
            }
            increment(idx, dims, N);
        }
        free(w);
    }
    memset(out, 0, sizeof(double) * outsz);
    for (int ch = 0; ch < ORACLE_CHUNKS; ++ch)
        for (int64_t e = 0; e < outsz; ++e) out[e] += part[(size_t)ch * outsz + e];
    free(part);
    return OR_OK;
}

/*
 * Multi-TTV, the second step of Algorithm 4 (Section 4.3):
 *   right (after R):  M(i, c) = sum_l R(l, i, c) * K_L(l, c)
 *   left  (after L):  M(i, c) = sum_r L(i, r, c) * K_R(r, c)
 * with K_L(l, c) = prod_{k<n} U_k(i_k(l), c) and K_R(r, c) = prod_{k>n} U_k(i_k(r), c)
 * formed entry by entry.  T is laid out as oracle_partial_mttkrp writes it.
 */
int oracle_multi_ttv(const double* T, const int64_t* dims, int N,
                     const double* const* U, int C, int n, int right, double* M) {
    int st = check_args(dims, N, C, n);
    if (st) return st;
    const int64_t IL = prod_dims(dims, 0, n), In = dims[n], IR = prod_dims(dims, n + 1, N);
    memset(M, 0, sizeof(double) * In * C);
    const int k0 = right ? 0 : n + 1, k1 = right ? n : N;
    const int64_t J = right ? IL : IR;
    int64_t sub[ORACLE_MAXN];
    int Ns = 0;
    for (int k = k0; k < k1; ++k) sub[Ns++] = dims[k];
    for (int64_t i = 0; i < In; ++i)
        for (int c = 0; c < C; ++c) {
            double s = 0.0;
            int64_t idx[ORACLE_MAXN];
            for (int k = 0; k < Ns; ++k) idx[k] = 0;
            for (int64_t j = 0; j < J; ++j) {
                double w = 1.0;
                for (int k = 0; k < Ns; ++k) w *= U[k0 + k][idx[k] * C + c];
                const double t = right ? T[j + IL * i + IL * In * c] : T[i + In * j + In * IR * c];
                s += t * w;
                if (Ns) increment(idx, sub, Ns);
            }
            M[i * C + c] = s;
        }
    return OR_OK;
}

/* Gram matrix G = U^T U of an I x C row-major matrix (Section 2.2, the second
   bullet of the factor update).  G is C x C row-major. */
int oracle_gram(const double* U, int64_t I, int C, double* G) {
    if (I < 1 || C < 1) return OR_EINVAL;
    for (int a = 0; a < C; ++a)
        for (int b = 0; b < C; ++b) {
            double s = 0.0;
            for (int64_t i = 0; i < I; ++i) s += U[i * C + a] * U[i * C + b];
            G[a * C + b] = s;
        }
    return OR_OK;
}

/* H = Hadamard product over k != n of U_k^T U_k (Section 2.2, second bullet). */
int oracle_gram_hadamard(const int64_t* dims, int N, const double* const* U, int C,
                         int n, double* H) {
    if (N < 1 || C < 1 || n < -1 || n >= N) return OR_EINVAL;
    double* G = (double*)malloc(sizeof(double) * C * C);
    if (!G) return OR_ENOMEM;
    for (int e = 0; e < C * C; ++e) H[e] = 1.0;
    for (int k = 0; k < N; ++k) {
        if (k == n) continue;
        oracle_gram(U[k], dims[k], C, G);
        for (int e = 0; e < C * C; ++e) H[e] *= G[e];
    }
    free(G);
    return OR_OK;
}

/* Cholesky factorization H = L L^T of a C x C symmetric matrix, textbook
   column-by-column (the reading of the pseudoinverse solve of Section 2.2 for
   a positive-definite H).  Returns OR_ENOTPD if a pivot is not positive. */
int oracle_cholesky(const double* H, int C, double* L) {
    memset(L, 0, sizeof(double) * C * C);
    for (int j = 0; j < C; ++j) {
        double d = H[j * C + j];
        for (int k = 0; k < j; ++k) d -= L[j * C + k] * L[j * C + k];
        if (!(d > 0.0)) return OR_ENOTPD;
        const double ljj = sqrt(d);
        L[j * C + j] = ljj;
        for (int i = j + 1; i < C; ++i) {
            double s = H[i * C + j];
            for (int k = 0; k < j; ++k) s -= L[i * C + k] * L[j * C + k];
            L[i * C + j] = s / ljj;
        }
    }
    return OR_OK;
}

/* U_n = M H^{-1} row by row given H = L L^T: solve L y = m, then L^T x = y
   (Section 2.2, third bullet).  M and U are I x C row-major. */
int oracle_chol_solve(const double* L, int C, const double* M, int64_t I, double* U) {
    double* y = (double*)malloc(sizeof(double) * C);
    if (!y) return OR_ENOMEM;
    for (int64_t i = 0; i < I; ++i) {
        const double* m = M + i * C;
        for (int a = 0; a < C; ++a) {
            double s = m[a];
            for (int k = 0; k < a; ++k) s -= L[a * C + k] * y[k];
            y[a] = s / L[a * C + a];
        }
        double* u = U + i * C;
        for (int a = C - 1; a >= 0; --a) {
            double s = y[a];
            for (int k = a + 1; k < C; ++k) s -= L[k * C + a] * u[k];
            u[a] = s / L[a * C + a];
        }
    }
    free(y);
    return OR_OK;
}

/* squared Frobenius norm of the tensor, fixed chunk order */
double oracle_norm2(const double* X, int64_t I) {
    double part[ORACLE_CHUNKS];
    #pragma omp parallel for schedule(static)
    for (int ch = 0; ch < ORACLE_CHUNKS; ++ch) {
        int64_t a = I * ch / ORACLE_CHUNKS, b = I * (ch + 1) / ORACLE_CHUNKS;
        double s = 0.0;
        for (int64_t l = a; l < b; ++l) s += X[l] * X[l];
        part[ch] = s;
    }
    double s = 0.0;
    for (int ch = 0; ch < ORACLE_CHUNKS; ++ch) s += part[ch];
    return s;
}

/* ||X - [[U_0..U_{N-1}]]||^2 by explicit reconstruction of every model entry
   Y(i_0..) = sum_c prod_k U_k(i_k, c) (Section 2.2, CP model).  Tiny inputs. */
double oracle_residual2_explicit(const double* X, const int64_t* dims, int N,
                                 const double* const* U, int C) {
    const int64_t I = prod_dims(dims, 0, N);
    double part[ORACLE_CHUNKS];
    #pragma omp parallel for schedule(static)
    for (int ch = 0; ch < ORACLE_CHUNKS; ++ch) {
        int64_t a = I * ch / ORACLE_CHUNKS, b = I * (ch + 1) / ORACLE_CHUNKS;
        double s = 0.0;
        int64_t idx[ORACLE_MAXN];
        if (a < b) unravel(a, dims, N, idx);
        for (int64_t l = a; l < b; ++l) {
            double y = 0.0;
            for (int c = 0; c < C; ++c) {
                double p = 1.0;
                for (int k = 0; k < N; ++k) p *= U[k][idx[k] * C + c];
                y += p;
            }
            const double d = X[l] - y;
            s += d * d;
            increment(idx, dims, N);
        }
        part[ch] = s;
    }
    double s = 0.0;
    for (int ch = 0; ch < ORACLE_CHUNKS; ++ch) s += part[ch];
    return s;
}

/*
 * Residual through the inner-product identity, without reconstructing the
 * model (the paper notes the residual cost but gives no formula; this is the
 * standard expansion):
 *   ||X - Y||^2 = ||X||^2 - 2 <M_m, U_m> + sum_{a,b} prod_k (U_k^T U_k)(a, b)
 * where M_m is the mode-m MTTKRP of X with the current factors (any m).
 */
double oracle_residual2_identity(double normX2, const double* Mm, const double* Um,
                                 int64_t Im, const int64_t* dims, int N,
                                 const double* const* U, int C) {
    double inner = 0.0;
    for (int64_t e = 0; e < Im * C; ++e) inner += Mm[e] * Um[e];
    double* H = (double*)malloc(sizeof(double) * C * C);
    oracle_gram_hadamard(dims, N, U, C, -1, H);
    double y2 = 0.0;
    for (int e = 0; e < C * C; ++e) y2 += H[e];
    free(H);
    return normX2 - 2.0 * inner + y2;
}

/*
 * One CP-ALS sweep (Section 2.2): for n = 0..N-1 in order, with the other
 * factors fixed at their latest values,
 *     M = MTTKRP(X, n);  H = Hadamard_{k != n} U_k^T U_k;  U_n = M H^{-1}
 * (H^{-1} through Cholesky; the paper writes the pseudoinverse).  After the
 * sweep, *fit = 1 - sqrt(max(0, residual2)) / ||X|| with residual2 from the
 * identity above at the last mode.  On a non-positive-definite H the sweep
 * stops with OR_ENOTPD and that factor is left unchanged.
 */
/*
 * Column normalisation of a factor, an optional step of CP-ALS.  The paper's ALS
 * (Section 2.2) has none; the reading adopted here is the usual one of CP-ALS codes:
 * lambda_c = ||U(:, c)||_2 and U(:, c) / lambda_c, a column of zeros left as it is
 * (lambda_c = 0).  U is I x C row-major; lambda (may be NULL) receives the C norms.
 */
void oracle_normalize_columns(double* U, int64_t I, int C, double* lambda) {
    for (int c = 0; c < C; ++c) {
        double s = 0.0;
        for (int64_t i = 0; i < I; ++i) s += U[i * C + c] * U[i * C + c];
        const double l = sqrt(s);
        if (lambda) lambda[c] = l;
        if (l > 0.0)
            for (int64_t i = 0; i < I; ++i) U[i * C + c] /= l;
    }
}

/*
 * One CP-ALS sweep (Section 2.2): for n = 0..N-1 in order, M = MTTKRP(X, n) with the
 * factors as they are at that point (the ones before n already updated), H = Hadamard
 * of the Grams of the other factors, U_n = M H^{-1} by Cholesky.  normalize != 0: after
 * its update every factor but the last is scaled to unit column norms (the last one then
 * carries the weights, so [[U_0, ..., U_{N-1}]] is the model without a separate lambda).
 * fit (may be NULL): 1 - ||X - [[U]]|| / ||X||.
 */
int oracle_als_sweep_opt(const double* X, const int64_t* dims, int N, double* const* U,
                         int C, int normalize, double* fit) {
    int st = check_args(dims, N, C, 0);
    if (st) return st;
    int64_t maxI = 0;
    for (int k = 0; k < N; ++k) if (dims[k] > maxI) maxI = dims[k];
    double* M = (double*)malloc(sizeof(double) * maxI * C);
    double* H = (double*)malloc(sizeof(double) * C * C);
    double* L = (double*)malloc(sizeof(double) * C * C);
    if (!M || !H || !L) { free(M); free(H); free(L); return OR_ENOMEM; }
    for (int n = 0; n < N && !st; ++n) {
        st = oracle_mttkrp(X, dims, N, (const double* const*)U, C, n, M);
        if (st) break;
        oracle_gram_hadamard(dims, N, (const double* const*)U, C, n, H);
        st = oracle_cholesky(H, C, L);
        if (st) break;
        oracle_chol_solve(L, C, M, dims[n], U[n]);
        if (normalize && n < N - 1) oracle_normalize_columns(U[n], dims[n], C, NULL);
    }
    if (!st && fit) {
        const int64_t I = prod_dims(dims, 0, N);
        const double nx2 = oracle_norm2(X, I);
        const double r2 = oracle_residual2_identity(nx2, M, U[N - 1], dims[N - 1], dims, N,
                                                    (const double* const*)U, C);
        *fit = 1.0 - sqrt(r2 > 0.0 ? r2 : 0.0) / sqrt(nx2);
    }
    free(M); free(H); free(L);
    return st;
}

int oracle_als_sweep(const double* X, const int64_t* dims, int N, double* const* U,
                     int C, double* fit) {
    return oracle_als_sweep_opt(X, dims, N, U, C, 0, fit);
}

/*
 * Gradient of f(U) = 0.5 ||X - [[U_0..U_{N-1}]]||^2 with respect to U_n:
 *     df/dU_n = U_n H_n - M_n,  H_n = Hadamard_{k != n} U_k^T U_k,  M_n = MTTKRP(X, n)
 * (MTTKRP is part of the gradient, Section 2.2).  G is I_n x C row-major.
 */
int oracle_grad(const double* X, const int64_t* dims, int N, const double* const* U,
                int C, int n, double* G) {
    int st = check_args(dims, N, C, n);
    if (st) return st;
    const int64_t In = dims[n];
    double* M = (double*)malloc(sizeof(double) * In * C);
    double* H = (double*)malloc(sizeof(double) * C * C);
    if (!M || !H) { free(M); free(H); return OR_ENOMEM; }
    st = oracle_mttkrp(X, dims, N, U, C, n, M);
    if (!st) {
        oracle_gram_hadamard(dims, N, U, C, n, H);
        for (int64_t i = 0; i < In; ++i)
            for (int b = 0; b < C; ++b) {
                double s = 0.0;
                for (int a = 0; a < C; ++a) s += U[n][i * C + a] * H[a * C + b];
                G[i * C + b] = s - M[i * C + b];
            }
    }
    free(M); free(H);
    return st;
}
