"""GPU parity of the one-launch factor update (U_n = M H^{-1} by an FP64 L D L^T of
H = Hadamard_{k != n} G_k, and G_n = U_n^T U_n in double-FP32) against the FP64 oracle,
through mtk_gram_hadamard_solve.

Bounds: U_n is an FP64 solve rounded to FP32, so it matches the oracle's Cholesky solve
to a few FP32 ulps (1e-6 relative Frobenius, independent of cond(H) at these sizes); the
Gram of the returned U_n matches the oracle's FP64 Gram of the same FP32 rows to 1e-12
relative to sqrt(G_aa G_bb) (double-FP32 sums carry ~2^-44 relative error per term).
Shapes span one CTA, ragged row groups, more than one first-level reduction group,
more rows than 304 CTAs of 4 rows (the multi-pass path) and C = 1 .. 64.
"""
import numpy as np
import pytest

import oracle
from helpers import factors_dev, rel_fro, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08976_gb300 as mtk  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mtk.load()


def make_case(dims, C, n, seed):
    g = np.random.default_rng(seed)
    U = [(g.standard_normal((d, C)) / np.sqrt(d)).astype(np.float32) for d in dims]
    M = g.standard_normal((dims[n], C)).astype(np.float32)
    return U, M


def run_update(U, M, n, want_gram=True):
    Ud = factors_dev(U, torch)
    G = [mtk.gram(u) for u in Ud]
    Un = torch.empty_like(Ud[n])
    Gn = torch.empty((M.shape[1], M.shape[1]), dtype=torch.float64, device="cuda") if want_gram else None
    ws = mtk.Workspace()
    mtk.gram_hadamard_solve(G, n, to_dev(M, torch), Un, Gn=Gn, ws=ws)
    return Un, Gn, ws.status()


def check_gram(Gn, Un):
    ref = oracle.gram(Un.cpu().numpy())
    got = Gn.cpu().numpy()
    d = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(got - ref) <= 1e-12 * d + 1e-300), np.max(np.abs(got - ref) / d)
    np.testing.assert_array_equal(got, got.T)


@pytest.mark.parametrize("dims,C,n", [
    ((1, 6, 5), 3, 0),            # one row
    ((30, 7, 9), 1, 1),           # C = 1, two ragged CTAs of rows
    ((40, 30, 20, 12), 25, 0),    # 10 CTAs, two first-level groups
    ((200, 200, 300, 40), 25, 2), # the benchmark's mode 2 (75 CTAs, 10 groups)
    ((1300, 20, 30), 17, 0),      # more rows than 304 CTAs of 4: 8 rows per CTA
    ((5000, 40, 60), 64, 0),      # C = 64, 20 rows per CTA
    ((50, 64, 33), 33, 2),        # C > 32: two columns per lane
])
def test_update_matches_oracle(dims, C, n):
    U, M = make_case(dims, C, n, seed=sum(dims) + C)
    Un, Gn, st = run_update(U, M, n)
    assert st == 0
    H = oracle.gram_hadamard(dims, [u.astype(np.float64) for u in U], n)
    ref = oracle.chol_solve(oracle.cholesky(H), M.astype(np.float64))
    assert rel_fro(Un.cpu().numpy(), ref) < 1e-6
    check_gram(Gn, Un)


def test_update_deterministic():
    U, M = make_case((300, 50, 40), 25, 0, seed=5)
    a = run_update(U, M, 0)
    b = run_update(U, M, 0)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_update_not_pd_keeps_factor_and_gram():
    """A zero column of a factor makes H singular: MTK_ENOTPD, U_n unchanged, and the
    requested Gram is that of the unchanged U_n."""
    g = np.random.default_rng(8)
    dims, C, n = (60, 45, 30), 20, 0
    U = [g.standard_normal((d, C)).astype(np.float32) for d in dims]
    U[2][:, 7] = 0.0
    Ud = factors_dev(U, torch)
    G = [mtk.gram(u) for u in Ud]
    before = Ud[n].clone()
    Gn = torch.empty((C, C), dtype=torch.float64, device="cuda")
    ws = mtk.Workspace()
    mtk.gram_hadamard_solve(G, n, to_dev(g.standard_normal((dims[n], C)), torch), Ud[n], Gn=Gn, ws=ws)
    assert ws.status() == 4
    assert torch.equal(before, Ud[n])
    check_gram(Gn, Ud[n])


def oracle_sweep_conds(X, dims, U):
    """cond(H_n) of every solve of the oracle's Gauss-Seidel sweep."""
    Uc = [u.copy() for u in U]
    conds = []
    for n in range(len(dims)):
        H = oracle.gram_hadamard(dims, Uc, n)
        conds.append(float(np.linalg.cond(H)))
        Uc[n] = oracle.chol_solve(oracle.cholesky(H), oracle.mttkrp(X, dims, Uc, n))
    return conds


@pytest.mark.parametrize("dims,C", [
    ((60, 50, 45), 40),          # C > 32: two columns per lane in the solves
    ((80, 70), 6),               # N = 2: the last mode reduces the first mode's Gram
    ((8, 7, 6, 5, 4), 5),        # N = 5: five Grams in the one-launch Gram kernel
    ((70, 80, 90), 64),          # C = 64, the largest one-launch update
])
def test_sweep_update_paths(dims, C):
    """FP32 CP-ALS sweeps through the one-launch updates (the Gram of each new factor
    reduced by the next mode's update, the last mode's Gram and the fit by tickets)
    against the oracle's sweep.  The solve amplifies the ~1e-7 relative error of an FP32
    MTTKRP by up to cond(H_n): factor n is held to 1e-6 + 2e-7 cond(H_n), the fit to 1e-6."""
    import synth
    from helpers import f32_round
    X, dims, U = synth.random_case(dims, C, seed=sum(dims) * 7 + C)
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    ref_U, ref_fit = oracle.als_sweep(Xr, dims, Ur)
    conds = oracle_sweep_conds(Xr, dims, Ur)
    Ud = factors_dev(U, torch)
    als = mtk.ALS(to_dev(X, torch), dims, Ud, precision="fp32")
    als.sweep()
    assert als.status() == 0
    for k in range(len(dims)):
        err = rel_fro(Ud[k].double().cpu().numpy(), ref_U[k])
        assert err < 1e-6 + 2e-7 * conds[k], (k, err, conds[k])
    assert abs(als.fit.item() - ref_fit) < 1e-6
    # a second sweep from the same start gives bitwise the same factors
    Ue = factors_dev(U, torch)
    als2 = mtk.ALS(to_dev(X, torch), dims, Ue, precision="fp32")
    als2.sweep()
    for a, b in zip(Ud, Ue):
        assert torch.equal(a, b)


@pytest.mark.parametrize("dims,C,n", [((150, 120, 90), 80, 1), ((300, 260), 128, 0)])
def test_solve_rank_above_64(dims, C, n):
    """Ranks above 64 take the other solve path (FP64 Cholesky and explicit inverse in one
    CTA, then a wide kernel applies it; the Gram of U_n by the chunked FP64 Gram kernels):
    the same bounds against the oracle's textbook Cholesky solve."""
    U, M = make_case(dims, C, n, seed=C + n)
    Un, Gn, st = run_update(U, M, n)
    assert st == 0
    H = oracle.gram_hadamard(dims, [u.astype(np.float64) for u in U], n)
    ref = oracle.chol_solve(oracle.cholesky(H), M.astype(np.float64))
    assert rel_fro(Un.cpu().numpy(), ref) < 1e-6
    ref_g = oracle.gram(Un.cpu().numpy())
    np.testing.assert_allclose(Gn.cpu().numpy(), ref_g, rtol=1e-12, atol=1e-12 * np.abs(ref_g).max())
