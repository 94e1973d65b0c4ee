"""Pins for the FP64 oracle (CPU only).

Each check ties the oracle to something other than itself: numpy brute force
(explicit matricization by reshape and an explicit KRP from column-wise
Kronecker products, Section 2.1), closed forms for tensors built from known
factors, textbook special cases, finite differences and hand-derived
integer examples (tests/golden/hand_examples.json).  A dropped term, a wrong
index order or a transposed operand anywhere in oracle.c fails one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


# ------------------------------------------------------------ independent numpy
def np_krp_columnwise(mats):
    """K(:, c) = mats[0](:, c) kron mats[1](:, c) kron ... (Section 2.1, column-wise
    definition), so the last operand's row index is fastest."""
    C = mats[0].shape[1]
    cols = []
    for c in range(C):
        v = np.ones(1)
        for m in mats:
            v = np.kron(v, m[:, c])
        cols.append(v)
    return np.stack(cols, axis=1)


def np_matricize(X, dims, n):
    """X_(n): I_n x prod_{k!=n} I_k, columns = remaining modes linearized with the
    lowest mode fastest (Section 2.1)."""
    Xt = synth.as_natural(np.asarray(X, dtype=np.float64), dims)
    return np.moveaxis(Xt, n, 0).reshape(dims[n], -1, order="F")


def np_mttkrp(X, dims, U, n):
    """M = X_(n) (U_{N-1} kr ... kr U_{n+1} kr U_{n-1} kr ... kr U_0) (Section 2.2)."""
    ops = [np.asarray(U[k], dtype=np.float64) for k in range(len(dims) - 1, -1, -1) if k != n]
    if not ops:
        C = np.asarray(U[n]).shape[1]
        K = np.ones((1, C))
    else:
        K = np_krp_columnwise(ops)
    return np_matricize(X, dims, n) @ K


def cp_full(F):
    """[[F_0, ..., F_{N-1}]] as a flat natural-order tensor, by einsum."""
    N = len(F)
    letters = "abcdefgh"[:N]
    expr = ",".join(f"{l}z" for l in letters) + "->" + letters
    T = np.einsum(expr, *F)
    return T.reshape(-1, order="F"), tuple(f.shape[0] for f in F)


# ------------------------------------------------------------------- pins
def test_hand_mttkrp_2x2x2():
    g = json.load(open(GOLD))["mttkrp_2x2x2"]
    dims = g["dims"]
    X = np.array(g["X"], dtype=np.float64)
    U = [np.array(u, dtype=np.float64) for u in g["U"]]
    for n in range(3):
        exp = np.array(g["M"][n], dtype=np.float64)
        assert np.array_equal(oracle.mttkrp(X, dims, U, n), exp)
        assert np.array_equal(oracle.mttkrp_brute(X, dims, U, n), exp)
        assert np.array_equal(np_mttkrp(X, dims, U, n), exp)


def test_hand_krp():
    gold = json.load(open(GOLD))
    for key in ("krp_two", "krp_three"):
        g = gold[key]
        U = [np.array(u, dtype=np.float64) for u in g["U"]]
        exp = np.array(g["K"], dtype=np.float64)
        assert np.array_equal(oracle.krp(U), exp)
        assert np.array_equal(np_krp_columnwise(U), exp)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("C", [1, 3])
def test_definition_vs_brute(N, C):
    g = np.random.default_rng(100 + 10 * N + C)
    sizes = [1, 2, 3, 5]
    for trial in range(6 if N < 5 else 3):
        dims = tuple(int(g.choice(sizes)) for _ in range(N))
        X, dims, U = synth.random_case(dims, C, seed=1000 * N + 10 * C + trial)
        for n in range(N):
            ref = np_mttkrp(X, dims, U, n)
            got = oracle.mttkrp(X, dims, U, n)
            brute = oracle.mttkrp_brute(X, dims, U, n)
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(brute, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims", [(7, 6, 5), (4, 3, 5, 2), (3, 2, 2, 3, 2)])
def test_closed_form_cp(dims):
    """X = [[A]] exactly => M_n = A_n * Hadamard_{k!=n}(A_k^T U_k) for any U."""
    g = np.random.default_rng(7)
    R, C = 4, 3
    A = [g.standard_normal((d, R)) for d in dims]
    U = [g.standard_normal((d, C)) for d in dims]
    X, _ = cp_full(A)
    for n in range(len(dims)):
        W = np.ones((R, C))
        for k in range(len(dims)):
            if k != n:
                W *= A[k].T @ U[k]
        np.testing.assert_allclose(oracle.mttkrp(X, dims, U, n), A[n] @ W, rtol=1e-11, atol=1e-11)
    # with U = A, the spec form U_n * Hadamard of the Grams
    for n in range(len(dims)):
        H = np.ones((R, R))
        for k in range(len(dims)):
            if k != n:
                H *= A[k].T @ A[k]
        np.testing.assert_allclose(oracle.mttkrp(X, dims, A, n), A[n] @ H, rtol=1e-11, atol=1e-11)


def test_two_way_is_matrix_product():
    X, dims, U = synth.random_case((9, 7), 4, seed=3)
    X2 = X.reshape(dims, order="F")                       # column-major I0 x I1
    np.testing.assert_allclose(oracle.mttkrp(X, dims, U, 0), X2 @ U[1], rtol=1e-13)
    np.testing.assert_allclose(oracle.mttkrp(X, dims, U, 1), X2.T @ U[0], rtol=1e-13)


def test_rank_one_is_ttv_chain():
    X, dims, U = synth.random_case((4, 5, 3, 2), 1, seed=4)
    Xt = synth.as_natural(X, dims)
    for n in range(4):
        T = Xt
        for k in range(3, -1, -1):                        # contract highest modes first
            if k != n:
                T = np.tensordot(T, U[k][:, 0], axes=([k], [0]))
        np.testing.assert_allclose(oracle.mttkrp(X, dims, U, n)[:, 0], T, rtol=1e-12)


def test_linearity_and_permutation():
    X, dims, U = synth.random_case((5, 4, 3, 2), 3, seed=5)
    Y, _, _ = synth.random_case((5, 4, 3, 2), 3, seed=6)
    for n in range(4):
        lhs = oracle.mttkrp(2.5 * X - 0.75 * Y, dims, U, n)
        rhs = 2.5 * oracle.mttkrp(X, dims, U, n) - 0.75 * oracle.mttkrp(Y, dims, U, n)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-11, atol=1e-12)
    # permuting the modes (and the factor list) permutes the MTTKRPs
    perm = (2, 0, 3, 1)
    Xp = np.transpose(synth.as_natural(X, dims), perm).reshape(-1, order="F")
    dp = tuple(dims[p] for p in perm)
    Up = [U[p] for p in perm]
    for j in range(4):
        np.testing.assert_allclose(oracle.mttkrp(Xp, dp, Up, j), oracle.mttkrp(X, dims, U, perm[j]),
                                   rtol=1e-12, atol=1e-12)


def test_range_and_rows():
    X, dims, U = synth.random_case((6, 5, 7), 4, seed=8)
    I = X.size
    for n in range(3):
        full = oracle.mttkrp(X, dims, U, n)
        cuts = [0, 17, 64, 150, I]
        acc = sum(oracle.mttkrp_range(X[a:b], a, b, dims, U, n) for a, b in zip(cuts[:-1], cuts[1:]))
        np.testing.assert_allclose(acc, full, rtol=1e-12, atol=1e-12)
        X32 = X.astype(np.float32)
        rows = [dims[n] - 1, 0, 2]
        ref = np_mttkrp(X32.astype(np.float64), dims, U, n)[rows]
        np.testing.assert_allclose(oracle.mttkrp_rows_f32(X32, dims, U, n, rows), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("Z", [1, 2, 3, 4])
def test_krp_vs_kron(Z):
    g = np.random.default_rng(Z)
    U = [g.standard_normal((int(g.integers(1, 6)), 5)) for _ in range(Z)]
    np.testing.assert_allclose(oracle.krp(U), np_krp_columnwise(U), rtol=1e-14)


@pytest.mark.parametrize("dims", [(4, 3, 5), (3, 4, 2, 3), (2, 3, 2, 2, 3)])
def test_two_step_pieces(dims):
    """Algorithm 4: the partial MTTKRPs are X_(0:n) K_R and X_(0:n-1)^T K_L, and the
    multi-TTV of either finishes the MTTKRP."""
    C = 3
    X, dims, U = synth.random_case(dims, C, seed=11)
    N = len(dims)
    Xt = synth.as_natural(X, dims)
    for n in range(N):
        IL = int(np.prod(dims[:n])); In = dims[n]; IR = int(np.prod(dims[n + 1:]))
        KR = np_krp_columnwise([U[k] for k in range(N - 1, n, -1)]) if n < N - 1 else np.ones((1, C))
        KL = np_krp_columnwise([U[k] for k in range(n - 1, -1, -1)]) if n > 0 else np.ones((1, C))
        X0n = Xt.reshape(IL * In, IR, order="F")             # X_(0:n), column-major
        X0n1 = Xt.reshape(IL, In * IR, order="F")            # X_(0:n-1)
        R = oracle.partial_mttkrp(X, dims, U, n, right=True)
        Lp = oracle.partial_mttkrp(X, dims, U, n, right=False)
        np.testing.assert_allclose(R.reshape(IL * In, C, order="F"), X0n @ KR, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(Lp.reshape(In * IR, C, order="F"), X0n1.T @ KL, rtol=1e-12, atol=1e-12)
        ref = np_mttkrp(X, dims, U, n)
        np.testing.assert_allclose(oracle.multi_ttv(R, dims, U, n, right=True), ref, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(oracle.multi_ttv(Lp, dims, U, n, right=False), ref, rtol=1e-11, atol=1e-12)


def test_gram_cholesky_solve():
    g = np.random.default_rng(12)
    U = g.standard_normal((40, 6))
    G = oracle.gram(U)
    np.testing.assert_allclose(G, U.T @ U, rtol=1e-13)
    dims = (40, 30, 20)
    Us = [U, g.standard_normal((30, 6)), g.standard_normal((20, 6))]
    H = oracle.gram_hadamard(dims, Us, 1)
    np.testing.assert_allclose(H, (Us[0].T @ Us[0]) * (Us[2].T @ Us[2]), rtol=1e-13)
    L = oracle.cholesky(H)
    np.testing.assert_allclose(L, np.linalg.cholesky(H), rtol=1e-12, atol=1e-12)
    M = g.standard_normal((25, 6))
    Un = oracle.chol_solve(L, M)
    np.testing.assert_allclose(Un @ H, M, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(Un, np.linalg.solve(H, M.T).T, rtol=1e-10, atol=1e-12)
    # a zero column in one factor gives an exactly zero pivot: reported, not solved
    Ud = [u.copy() for u in Us]
    Ud[2][:, 3] = 0.0
    with pytest.raises(oracle.OracleError):
        oracle.cholesky(oracle.gram_hadamard(dims, Ud, 0))
    with pytest.raises(oracle.OracleError):
        oracle.cholesky(-np.eye(4))


def np_als_sweep(X, dims, U):
    """Independent CP-ALS sweep: explicit matricization, explicit KRP, normal
    equations by numpy's general solver (Section 2.2)."""
    U = [u.copy() for u in U]
    N = len(dims)
    for n in range(N):
        M = np_mttkrp(X, dims, U, n)
        H = np.ones((U[0].shape[1],) * 2)
        for k in range(N):
            if k != n:
                H *= U[k].T @ U[k]
        U[n] = np.linalg.solve(H, M.T).T
    return U


def test_als_sweep_matches_numpy_and_fixed_point():
    X, dims, U = synth.random_case((7, 6, 5, 4), 3, seed=13, dist="uniform")
    Uo, fit = oracle.als_sweep(X, dims, U)
    Un = np_als_sweep(X, dims, U)
    for a, b in zip(Uo, Un):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-10)
    r2 = oracle.residual2_explicit(X, dims, Uo)
    np.testing.assert_allclose(fit, 1 - np.sqrt(r2) / np.sqrt(np.sum(X * X)), rtol=1e-9)
    # loss is non-increasing over sweeps (each update is an exact least-squares solve)
    last = oracle.residual2_explicit(X, dims, U)
    Ucur = U
    for _ in range(4):
        Ucur, _ = oracle.als_sweep(X, dims, Ucur)
        cur = oracle.residual2_explicit(X, dims, Ucur)
        assert cur <= last * (1 + 1e-12)
        last = cur
    # exact rank-3 CP with its own factors as the start is a fixed point with fit 1
    g = np.random.default_rng(14)
    A = [g.random((d, 3)) + 0.1 for d in (6, 5, 4)]
    Xe, de = cp_full(A)
    Ua, fit_a = oracle.als_sweep(Xe, de, A)
    for a, b in zip(Ua, A):
        np.testing.assert_allclose(a, b, rtol=1e-8, atol=1e-10)
    assert abs(fit_a - 1.0) < 1e-6


@pytest.mark.parametrize("dims,C", [((7, 6, 5), 3), ((6, 5, 4, 3), 4), ((5, 4, 3, 3, 2), 2)])
def test_als_sweep_normalized_same_model(dims, C):
    """The optional column normalisation leaves the model unchanged: ALS is equivariant
    under column scaling (scaling U_k by a diagonal D multiplies M_n and H_n so that the
    next U_n comes out scaled by D^{-1}), so over several sweeps the normalised and plain
    runs give the same reconstruction [[U]] and fit; the normalised factors but the last
    have unit columns, the last one carries the weights."""
    X, dims, U = synth.random_case(dims, C, seed=31 + len(dims), dist="uniform")
    Ua, Ub = U, U
    N = len(dims)
    for _ in range(3):
        Ua, fa = oracle.als_sweep(X, dims, Ua)
        Ub, fb = oracle.als_sweep(X, dims, Ub, normalize=True)
        Ta, _ = cp_full(Ua)
        Tb, _ = cp_full(Ub)
        np.testing.assert_allclose(Tb, Ta, rtol=1e-9, atol=1e-11 * np.abs(Ta).max())
        assert abs(fa - fb) < 1e-10
        for k in range(N - 1):
            np.testing.assert_allclose(np.linalg.norm(Ub[k], axis=0), 1.0, rtol=1e-13)
        assert np.abs(np.linalg.norm(Ub[N - 1], axis=0) - 1.0).max() > 1e-3
    # the normalisation step alone: unit columns, the norms returned, zero columns kept
    g = np.random.default_rng(5)
    A = g.standard_normal((9, 4))
    A[:, 2] = 0.0
    An, lam = oracle.normalize_columns(A)
    np.testing.assert_allclose(lam, [np.sqrt(np.sum(A[:, c] ** 2)) for c in range(4)], rtol=1e-15)
    np.testing.assert_allclose(An[:, [0, 1, 3]] * lam[[0, 1, 3]], A[:, [0, 1, 3]], rtol=1e-15)
    assert np.all(An[:, 2] == 0.0)


def test_residual_identity():
    X, dims, U = synth.random_case((6, 5, 4), 4, seed=15)
    for m in range(3):
        Mm = oracle.mttkrp(X, dims, U, m)
        r2 = oracle.residual2_identity(oracle.norm2(X), Mm, U[m], dims, U)
        np.testing.assert_allclose(r2, oracle.residual2_explicit(X, dims, U), rtol=1e-10)


def test_gradient_finite_differences():
    X, dims, U = synth.fd5()
    for n in range(5):
        G = oracle.grad(X, dims, U, n)
        FD = np.zeros_like(G)
        for i, c in itertools.product(range(dims[n]), range(3)):
            h = 1e-6 * max(1.0, abs(U[n][i, c]))
            Up = [u.copy() for u in U]; Up[n][i, c] += h
            Um = [u.copy() for u in U]; Um[n][i, c] -= h
            FD[i, c] = (oracle.loss_explicit(X, dims, Up) - oracle.loss_explicit(X, dims, Um)) / (2 * h)
        np.testing.assert_allclose(G, FD, rtol=1e-6, atol=1e-7)
    # the gradient vanishes at the exact factors of an exact CP tensor
    g = np.random.default_rng(16)
    A = [g.standard_normal((d, 3)) for d in dims]
    Xe, _ = cp_full(A)
    for n in range(5):
        assert np.max(np.abs(oracle.grad(Xe, dims, A, n))) < 1e-10


def test_thread_count_independent():
    X, dims, U = synth.random_case((9, 8, 7), 5, seed=17)
    t0 = oracle.num_threads()
    a = oracle.mttkrp(X, dims, U, 1)
    oracle.set_num_threads(1)
    b = oracle.mttkrp(X, dims, U, 1)
    oracle.set_num_threads(t0)
    assert np.array_equal(a, b)
