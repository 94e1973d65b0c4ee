"""Full-size GPU parity on the benchmark workloads, in the launch configuration the
benchmark uses.

* cube512 (512^3, C = 32): every mode x algorithm x precision on sampled rows, the
  oracle computing each sampled row of M from the FP32 tensor one by one.
* corr4 (200x200x300x40, C = 25): the full M of every mode for every precision
  against the FP64 oracle, bound 1e-5 relative Frobenius error (bf16x2 is held to
  its derived bound, see test_gpu_tc.py, and reported); one CP-ALS sweep.
* cube32x5 (32^5, C = 16): the hand-written backward against the oracle gradient.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08976_gb300 as mtk  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mtk.load()


def bf16x2_bound(Xr64_rows_fn, ref):
    """3x the expected representation error of 2-piece BF16 tensor entries plus the
    FP32 accumulation allowance (test_gpu_tc.py derives it)."""
    M2 = Xr64_rows_fn()
    rho = np.sqrt(max(M2.sum(), 0.0)) / max(np.linalg.norm(ref), 1e-300)
    return 3.0 * 2.0 ** -16 / np.sqrt(3.0) * rho + 2e-6


@pytest.fixture(scope="module")
def cube():
    X, dims, U = synth.cube512()
    return X, dims, U, torch.from_numpy(X).cuda(), [torch.from_numpy(u).cuda() for u in U]


@pytest.mark.parametrize("prec", ["fp32", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("algo", ["fused", "materialized", "two_step"])
def test_cube512_sampled_rows(cube, prec, algo):
    X, dims, U, Xd, Ud = cube
    U64 = [u.astype(np.float64) for u in U]
    g = np.random.default_rng(40)
    for n in range(3):
        M = mtk.mttkrp(Xd, dims, Ud, n, precision=prec, algo=algo)
        rows = np.unique(np.concatenate([[0, dims[n] - 1], g.integers(0, dims[n], 6)]))
        ref = oracle.mttkrp_rows_f32(X, dims, U64, n, rows)
        got = M[torch.as_tensor(rows, device="cuda")].double().cpu().numpy()
        err = rel_fro(got, ref)
        if prec == "bf16x2":
            X2 = (X.astype(np.float64) ** 2).astype(np.float32)
            tol = bf16x2_bound(lambda: oracle.mttkrp_rows_f32(X2, dims, [u * u for u in U64], n, rows), ref)
        else:
            tol = 1e-5
        assert err < tol, (n, prec, algo, err, tol)


@pytest.fixture(scope="module")
def corr():
    X, dims, U = synth.corr4()
    return X, dims, U, torch.from_numpy(X).cuda(), [torch.from_numpy(u).cuda() for u in U]


@pytest.fixture(scope="module")
def corr_ref(corr):
    X, dims, U, _, _ = corr
    X64 = X.astype(np.float64)
    U64 = [u.astype(np.float64) for u in U]
    refs = [oracle.mttkrp(X64, dims, U64, n) for n in range(4)]
    sq = [oracle.mttkrp(X64 * X64, dims, [u * u for u in U64], n) for n in range(4)]
    del X64
    return refs, sq


@pytest.mark.parametrize("prec", ["fp32", "bf16x2", "bf16x3"])
def test_corr4_full_M(corr, corr_ref, prec):
    """Every mode-n MTTKRP of the 4-way correlation-shaped workload, the whole M."""
    X, dims, U, Xd, Ud = corr
    refs, sq = corr_ref
    for n in range(4):
        M = mtk.mttkrp(Xd, dims, Ud, n, precision=prec).double().cpu().numpy()
        err = rel_fro(M, refs[n])
        if prec == "bf16x2":
            rho = np.sqrt(sq[n].sum()) / np.linalg.norm(refs[n])
            tol = 3.0 * 2.0 ** -16 / np.sqrt(3.0) * rho + 2e-6
        else:
            tol = 1e-5
        assert err < tol, (n, prec, err, tol)
        if prec != "bf16x2":
            assert err < 1e-5


def test_corr4_als_sweep(corr):
    """One CP-ALS sweep on the full workload against the oracle's sweep; factor n is held
    to 1e-5 + 2e-7 cond(H_n) (the solve amplifies the MTTKRP error by cond(H_n))."""
    X, dims, U, Xd, _ = corr
    X64 = X.astype(np.float64)
    U64 = [u.astype(np.float64) for u in U]
    Uc = [u.copy() for u in U64]
    conds = []
    for n in range(4):
        H = oracle.gram_hadamard(dims, Uc, n)
        conds.append(float(np.linalg.cond(H)))
        Uc[n] = oracle.chol_solve(oracle.cholesky(H), oracle.mttkrp(X64, dims, Uc, n))
    ref_U, ref_fit = oracle.als_sweep(X64, dims, U64)
    del X64
    for prec in ("bf16x3", "fp32", "planes", "planes-tree"):
        Ud = [torch.from_numpy(u).cuda() for u in U]
        if prec == "planes":
            als = mtk.ALS(Xd, dims, Ud, presplit=True)
        elif prec == "planes-tree":
            als = mtk.ALS(Xd, dims, Ud, presplit=True, algo="two_step")
        else:
            als = mtk.ALS(Xd, dims, Ud, precision=prec)
        als.sweep()
        assert als.status() == 0
        for k in range(4):
            err = rel_fro(Ud[k].cpu().numpy(), ref_U[k])
            tol = 1e-5 + 2e-7 * conds[k]
            if prec.startswith("planes"):       # bf16x2 accuracy of the MTTKRP (see test_gpu_split.py)
                tol = 3e-5 + 1e-6 * conds[k]
            assert err < tol, (prec, k, err, conds[k])
        assert abs(als.fit.item() - ref_fit) < 1e-5


def test_cube32x5_gradient():
    X, dims, U = synth.cube32x5()
    U64 = [u.astype(np.float64) for u in U]
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda().requires_grad_(True) for u in U]
    loss = mtk.cp_loss(Xd, dims, Ud, precision="bf16x3")
    loss.backward()
    X64 = X.astype(np.float64)
    for n in range(5):
        ref = oracle.grad(X64, dims, U64, n)
        assert rel_fro(Ud[n].grad.double().cpu().numpy(), ref) < 1e-5, n


def test_corr4_twenty_sweeps(corr):
    """Twenty CP-ALS sweeps on the full workload, the dimension tree on the planes (the
    benchmark's form) and the FP32 form, against twenty sweeps of the FP64 oracle from the
    same start.  The fit after every sweep is compared: the MTTKRP's error against the FP64
    oracle (bf16x2 planes 2e-6 to 5e-6, FP32 7e-7 to 1.5e-6 per mode) moves each update by up
    to cond(H_n) times that, and ALS damps such differences from one sweep to the next, so
    the fits agree to 1e-5 (bf16x2) and 5e-6 (FP32: a few times its largest per-mode
    error; the FP32 fits differ from the oracle's by up to 2.1e-6 in the first sweeps)."""
    X, dims, U, Xd, _ = corr
    X64 = X.astype(np.float64)
    Uc = [u.astype(np.float64) for u in U]
    ref_fits = []
    for _ in range(20):
        Uc, f = oracle.als_sweep(X64, dims, Uc)
        ref_fits.append(f)
    del X64
    for form, tol in (("planes-tree", 1e-5), ("fp32", 5e-6)):
        Ud = [torch.from_numpy(u).cuda() for u in U]
        if form == "planes-tree":
            als = mtk.ALS(Xd, dims, Ud, presplit=True, algo="two_step")
        else:
            als = mtk.ALS(Xd, dims, Ud, precision="fp32")
        for it in range(20):
            als.sweep()
            f = als.fit.item()
            assert abs(f - ref_fits[it]) < tol, (form, it, f, ref_fits[it])
        assert als.status() == 0
    assert ref_fits[-1] >= ref_fits[0] - 1e-12
