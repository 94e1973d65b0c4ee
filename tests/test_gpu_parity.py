"""GPU parity: every CUDA path through the C ABI against the FP64 oracle, element by
element, on the same seeded inputs.

Tolerances (relative Frobenius error against the oracle on the FP64 inputs):
  * FP32 paths: 1e-6 on small cases (input rounding to FP32 is ~6e-8 per entry; FP32
    accumulation over at most a few thousand terms per split adds ~1e-7).
  * KRP: 4e-7 per entry relative (at most Z-1 FP32 roundings, Z <= 4).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import f32_round, factors_dev, rel_fro, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08976_gb300 as mtk  # noqa: E402

ALGOS = ["fused", "materialized", "two_step"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mtk.load()


def run_mttkrp(X, dims, U, n, **kw):
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    M = mtk.mttkrp(Xd, dims, Ud, n, **kw)
    torch.cuda.synchronize()
    return M.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("algo", ALGOS)
def test_tiny3_all_modes(algo):
    """60x50x40 FP64 tensor, rank 8: FP32 GPU path within 1e-6 of the FP64 oracle."""
    X, dims, U = synth.tiny3()
    for n in range(3):
        ref = oracle.mttkrp(X, dims, U, n)
        got = run_mttkrp(X, dims, U, n, algo=algo, precision="fp32")
        assert rel_fro(got, ref) < 1e-6, (algo, n, rel_fro(got, ref))


ODD_SHAPES = [
    ((1, 7, 3), 3), ((5, 1, 9), 1), ((13, 11, 1), 2), ((2, 3, 5, 7), 25), ((31, 37), 33),
    ((6, 5, 4, 3, 2), 3), ((3, 2, 2, 3, 2, 4), 5), ((67, 3, 129), 8), ((130, 66, 5), 64),
    ((17, 19, 23), 32), ((257, 9, 33), 16), ((4, 300, 2, 3), 7),
]


@pytest.mark.parametrize("dims,C", ODD_SHAPES)
@pytest.mark.parametrize("algo", ALGOS)
def test_odd_shapes(dims, C, algo):
    """Ragged tiles, unit modes, primes, C not a multiple of 4, N from 2 to 6."""
    X, dims, U = synth.random_case(dims, C, seed=sum(dims) + C)
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    for n in range(len(dims)):
        ref = oracle.mttkrp(Xr, dims, Ur, n)
        got = run_mttkrp(X, dims, U, n, algo=algo, precision="fp32")
        assert rel_fro(got, ref) < 2e-6, (dims, C, algo, n, rel_fro(got, ref))


@pytest.mark.parametrize("splits", [1, 2, 7, 64])
def test_split_counts_agree(splits):
    X, dims, U = synth.random_case((40, 30, 50), 12, seed=3)
    Xr = X.astype(np.float32).astype(np.float64)
    for n in range(3):
        ref = oracle.mttkrp(Xr, dims, f32_round(U), n)
        got = run_mttkrp(X, dims, U, n, algo="fused", precision="fp32", splits=splits)
        assert rel_fro(got, ref) < 1e-6


def test_deterministic_repeat():
    X, dims, U = synth.random_case((64, 48, 80), 25, seed=4)
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    for n in range(3):
        a = mtk.mttkrp(Xd, dims, Ud, n).clone()
        b = mtk.mttkrp(Xd, dims, Ud, n).clone()
        assert torch.equal(a, b)


@pytest.mark.parametrize("Z", [1, 2, 3, 4])
@pytest.mark.parametrize("reuse", [True, False])
def test_khatri_rao(Z, reuse):
    g = np.random.default_rng(50 + Z)
    rows = [int(g.integers(1, 40)) for _ in range(Z)]
    for C in (1, 7, 25, 50):
        U = [g.standard_normal((r, C)) for r in rows]
        Ur = f32_round(U)
        ref = oracle.krp(Ur)
        got = mtk.khatri_rao(factors_dev(U, torch), reuse=reuse)
        torch.cuda.synchronize()
        got = got.cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, ref, rtol=4e-7, atol=1e-30)


KRP_SHAPES = [
    ((7, 5, 3, 2, 3), 3),         # Z = 5: the generic naive kernel
    ((3, 2, 2, 3, 2, 5), 5),      # Z = 6
    ((4099,), 25),                # Z = 1 (a copy): several tiles, a ragged last group
    ((1, 4097), 7),               # a one-row operand first
    ((37, 113, 5), 50),           # C = 50: two 16-byte words per lane in some rows
    ((300, 301), 1),              # C = 1: four rows per 16-byte word
    ((2, 3), 33),                 # C > 32: lanes take two words
    ((61, 1, 59), 25),            # a one-row operand inside
]


@pytest.mark.parametrize("rows,C", KRP_SHAPES)
@pytest.mark.parametrize("reuse", [True, False])
def test_khatri_rao_shapes(rows, C, reuse):
    """Row rule of Section 2.1 (oracle, no reuse) against both kernels: tiles of rows,
    groups of four rows written as 16-byte words, ragged last groups, Z up to 6."""
    g = np.random.default_rng(sum(rows) + C)
    U = [g.standard_normal((r, C)) for r in rows]
    Ur = f32_round(U)
    ref = oracle.krp(Ur)
    got = mtk.khatri_rao(factors_dev(U, torch), reuse=reuse).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, ref, rtol=4e-7, atol=1e-30)


@pytest.mark.parametrize("reuse", [True, False])
def test_khatri_rao_unaligned_output(reuse):
    """An output that starts 4 bytes past a 16-byte boundary takes the scalar stores;
    the floats around it are left as they were."""
    g = np.random.default_rng(77)
    rows, C = (45, 23), 25
    U = [g.standard_normal((r, C)) for r in rows]
    ref = oracle.krp(f32_round(U))
    J = rows[0] * rows[1]
    buf = torch.full((J * C + 2,), 7.0, dtype=torch.float32, device="cuda")
    out = buf[1:1 + J * C].view(J, C)
    assert out.data_ptr() % 16 != 0
    mtk.khatri_rao(factors_dev(U, torch), reuse=reuse, out=out)
    got = buf.cpu().numpy()
    assert got[0] == 7.0 and got[-1] == 7.0
    np.testing.assert_allclose(got[1:-1].reshape(J, C).astype(np.float64), ref, rtol=4e-7, atol=1e-30)


def test_khatri_rao_hand_example():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))
    for key in ("krp_two", "krp_three"):
        U = [np.array(u, dtype=np.float32) for u in g[key]["U"]]
        got = mtk.khatri_rao(factors_dev(U, torch)).cpu().numpy()
        assert np.array_equal(got, np.array(g[key]["K"], dtype=np.float32))


def test_hand_mttkrp_exact():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))["mttkrp_2x2x2"]
    X = np.array(g["X"], dtype=np.float32)
    U = [np.array(u, dtype=np.float32) for u in g["U"]]
    for algo in ALGOS:
        for n in range(3):
            got = run_mttkrp(X, g["dims"], U, n, algo=algo, precision="fp32")
            assert np.array_equal(got, np.array(g["M"][n], dtype=np.float64)), (algo, n)


@pytest.mark.parametrize("dims", [(12, 7, 9), (5, 8, 6, 4), (3, 4, 5, 3, 2)])
def test_two_step_pieces(dims):
    C = 6
    X, dims, U = synth.random_case(dims, C, seed=21)
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    N = len(dims)
    Xd = to_dev(X, torch)
    for n in range(N):
        KR_ops = [U[k] for k in range(N - 1, n, -1)]
        KL_ops = [U[k] for k in range(n - 1, -1, -1)]
        C1 = np.ones((1, C))
        KR = mtk.khatri_rao(factors_dev(KR_ops, torch)) if KR_ops else to_dev(C1, torch)
        KL = mtk.khatri_rao(factors_dev(KL_ops, torch)) if KL_ops else to_dev(C1, torch)
        for right in (True, False):
            T = mtk.partial_mttkrp(Xd, dims, KR if right else KL, n, right)
            ref_T = oracle.partial_mttkrp(Xr, dims, Ur, n, right)
            assert rel_fro(T.cpu().numpy(), ref_T) < 1e-6, (n, right)
            M = mtk.multi_ttv(T, dims, KL if right else KR, n, right)
            ref_M = oracle.mttkrp(Xr, dims, Ur, n)
            assert rel_fro(M.cpu().numpy(), ref_M) < 1e-6, (n, right)


def test_gram_and_solve():
    g = np.random.default_rng(30)
    dims = (40, 30, 20)
    C = 6
    U = [g.random((d, C)).astype(np.float32) for d in dims]
    Ud = factors_dev(U, torch)
    G = [mtk.gram(u) for u in Ud]
    for k in range(3):
        np.testing.assert_allclose(G[k].cpu().numpy(), oracle.gram(U[k]), rtol=1e-13)
    M = g.standard_normal((dims[1], C)).astype(np.float32)
    Md = to_dev(M, torch)
    Un = torch.empty_like(Ud[1])
    Gn = torch.empty((C, C), dtype=torch.float64, device="cuda")
    ws = mtk.Workspace()
    mtk.gram_hadamard_solve(G, 1, Md, Un, Gn=Gn, ws=ws)
    assert ws.status() == 0
    H = oracle.gram_hadamard(dims, [u.astype(np.float64) for u in U], 1)
    ref = oracle.chol_solve(oracle.cholesky(H), M.astype(np.float64))
    assert rel_fro(Un.cpu().numpy(), ref) < 1e-6
    np.testing.assert_allclose(Gn.cpu().numpy(), oracle.gram(Un.cpu().numpy()), rtol=1e-12)


def test_not_positive_definite_reported():
    """A zero column in a factor makes H singular: MTK_ENOTPD, U_n left unchanged."""
    g = np.random.default_rng(31)
    dims = (20, 15, 10)
    C = 4
    U = [g.random((d, C)).astype(np.float32) for d in dims]
    U[2][:, 1] = 0.0
    Ud = factors_dev(U, torch)
    G = [mtk.gram(u) for u in Ud]
    M = to_dev(g.standard_normal((dims[0], C)), torch)
    before = Ud[0].clone()
    ws = mtk.Workspace()
    ws.get(1 << 16)
    mtk.gram_hadamard_solve(G, 0, M, Ud[0], ws=ws)
    assert ws.status() == 4
    assert torch.equal(before, Ud[0])


def test_norm2():
    X, dims, _ = synth.random_case((70, 33, 41), 2, seed=32)
    got = mtk.norm2(to_dev(X, torch)).item()
    ref = oracle.norm2(X.astype(np.float32).astype(np.float64))
    assert abs(got - ref) / ref < 1e-6


def oracle_sweep_with_cond(X, dims, U):
    """The oracle's sweep, one mode at a time, with cond(H_n) of every solve."""
    Uc = [u.copy() for u in U]
    conds = []
    for n in range(len(dims)):
        H = oracle.gram_hadamard(dims, Uc, n)
        conds.append(float(np.linalg.cond(H)))
        Uc[n] = oracle.chol_solve(oracle.cholesky(H), oracle.mttkrp(X, dims, Uc, n))
    return Uc, conds


@pytest.mark.parametrize("algo", ["fused", "two_step", "materialized"])
def test_als_sweep_tiny3(algo):
    """One CP-ALS sweep on the 60x50x40 rank-8 case against the FP64 oracle sweep.

    The solve U_n = M H^{-1} amplifies the ~1e-7 relative error of an FP32 MTTKRP by
    up to cond(H_n) (21, 68 and 327 for the three modes here), so factor n is held to
    1e-6 + 2e-7 * cond(H_n); the fit to 1e-6 absolute."""
    X, dims, U = synth.tiny3()
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    ref_U, ref_fit = oracle.als_sweep(Xr, dims, Ur)
    _, conds = oracle_sweep_with_cond(Xr, dims, Ur)
    Ud = factors_dev(U, torch)
    als = mtk.ALS(to_dev(X, torch), dims, Ud, algo=algo, precision="fp32")
    als.sweep()
    assert als.status() == 0
    for k in range(3):
        err = rel_fro(Ud[k].cpu().numpy(), ref_U[k])
        assert err < 1e-6 + 2e-7 * conds[k], (k, err, conds[k])
    assert abs(als.fit.item() - ref_fit) < 1e-6


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_als_fixed_point_exact_cp(prec):
    """An exact rank-3 CP tensor is a fixed point of the ALS sweep started at its factors.
    Factor n moves only by the FP32 rounding of X and of the factors (relative ~6e-8 each)
    and the MTTKRP's own error (~1e-7 in these forms), amplified by cond(H_n) (11 to 21
    here): held to 1e-6 + 2e-7 cond(H_n).  The fit comes from the residual identity
    ||X||^2 - 2 <X, Xhat> + ||Xhat||^2, whose terms cancel to the residual: a relative
    error e of the terms leaves 1 - fit up to sqrt(2 e): e = 1.5e-7 (FP32) and 1e-6 (bf16x3,
    whose MTTKRP error is 6e-7 to 8e-7 on the full-size workload) give 5.5e-4 and 1.4e-3."""
    g = np.random.default_rng(33)
    A = [g.random((d, 3)) + 0.2 for d in (30, 20, 10)]
    X = np.einsum("az,bz,cz->abc", *A).reshape(-1, order="F")
    dims = (30, 20, 10)
    A32 = f32_round(A)
    Ud = factors_dev(A, torch)
    als = mtk.ALS(to_dev(X, torch), dims, Ud, precision=prec)
    als.sweep()
    assert als.status() == 0
    for k in range(3):
        H = oracle.gram_hadamard(dims, A32, k)
        tol = 1e-6 + 2e-7 * np.linalg.cond(H)
        assert rel_fro(Ud[k].cpu().numpy(), A32[k]) < tol, (k, tol)
    e = {"fp32": 1.5e-7, "bf16x3": 1e-6}[prec]
    assert abs(als.fit.item() - 1.0) < np.sqrt(2.0 * e)


def test_gradient_matches_oracle_and_fd():
    """Hand-written backward against the oracle gradient, and against central finite
    differences of the oracle's FP64 loss (6x5x4x3x2, rank 3)."""
    X, dims, U = synth.fd5()
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    Xd = to_dev(X, torch)
    Ud = [u.requires_grad_(True) for u in factors_dev(U, torch)]
    loss = mtk.cp_loss(Xd, dims, Ud)
    loss.backward()
    np.testing.assert_allclose(loss.item(), oracle.loss_explicit(Xr, dims, Ur), rtol=1e-5)
    for n in range(5):
        got = Ud[n].grad.cpu().numpy().astype(np.float64)
        ref = oracle.grad(Xr, dims, Ur, n)
        assert rel_fro(got, ref) < 1e-5
        FD = np.zeros_like(ref)
        for i in range(dims[n]):
            for c in range(3):
                h = 1e-6 * max(1.0, abs(Ur[n][i, c]))
                Up = [u.copy() for u in Ur]; Up[n][i, c] += h
                Um = [u.copy() for u in Ur]; Um[n][i, c] -= h
                FD[i, c] = (oracle.loss_explicit(Xr, dims, Up) - oracle.loss_explicit(Xr, dims, Um)) / (2 * h)
        np.testing.assert_allclose(got, FD, rtol=1e-4, atol=1e-4 * np.abs(FD).max())
        assert rel_fro(got, FD) < 1e-5


def test_ffma_probe_counts_and_values():
    """The FMA probe reports 2 x 8 x iters flops per thread and leaves finite chain sums
    (x <- 0.999 x + 1e-4 from x_0 = (t + j) 1e-3 stays in [0, 0.3))."""
    lib = mtk.load()
    n = lib.mtk_ffma_probe_out_floats(2)
    out = torch.full((n,), float("nan"), device="cuda")
    flops = mtk.ffma_probe(2, 100, out=out)
    torch.cuda.synchronize()
    assert flops == 2.0 * 8 * 100 * n
    v = out.cpu().numpy()
    assert np.all(np.isfinite(v)) and v.min() >= 0.0 and v.max() < 8 * 0.3
