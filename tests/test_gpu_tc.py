"""GPU parity of the tensor-core (tcgen05) split-BF16 contraction against the FP64 oracle.

Tolerances (relative Frobenius error against the oracle on the FP32-rounded inputs):
  * bf16x3: tensor entries carried to 24 bits (3 BF16 pieces), KRP entries to 24 bits,
    FP32 accumulation -> same bound as the FP32 path, 2e-6.
  * bf16x2: tensor entries carried to 16 bits: each x is represented with an error
    d <= 2^-16 |x|, spread about uniformly, so E[d^2] <= (2^-16)^2 |x|^2 / 3 and the
    expected relative Frobenius error of M is 2^-16/sqrt(3) * rho with
    rho = sqrt(sum_{i,c} sum_t x_t^2 w_t^2) / ||M||_F; the double sum is the MTTKRP of
    X*X with the factors U*U (oracle).  The test allows 3x that expectation plus the
    FP32 accumulation allowance of 2e-6.
Shapes that the tensor-core kernel does not take (I^L not a multiple of 4, C > 64, ...)
run on the FP32 kernel; the same bounds hold.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import f32_round, factors_dev, rel_fro, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08976_gb300 as mtk  # noqa: E402

TOL = {"bf16x3": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mtk.load()


def split_bound(Xr, dims, Ur, n, ref, prec):
    if prec == "bf16x3":
        return TOL["bf16x3"]
    M2 = oracle.mttkrp(Xr * Xr, dims, [u * u for u in Ur], n)
    rho = np.sqrt(max(M2.sum(), 0.0)) / max(np.linalg.norm(ref), 1e-300)
    return 3.0 * 2.0 ** -16 / np.sqrt(3.0) * rho + 2e-6


def check_all_modes(X, dims, U, prec, algo="fused", splits=0):
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    errs = []
    for n in range(len(dims)):
        ref = oracle.mttkrp(Xr, dims, Ur, n)
        got = mtk.mttkrp(Xd, dims, Ud, n, precision=prec, algo=algo, splits=splits)
        torch.cuda.synchronize()
        e = rel_fro(got.cpu().numpy(), ref)
        errs.append(e)
        tol = split_bound(Xr, dims, Ur, n, ref, prec)
        assert e < tol, (dims, prec, algo, n, e, tol)
    return errs


@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
def test_tiny3(prec):
    X, dims, U = synth.tiny3()
    check_all_modes(X, dims, U, prec)


TC_SHAPES = [
    ((64, 32, 48), 25), ((200, 20, 36), 25), ((8, 12, 100), 64), ((4, 130, 9), 8),
    ((12, 5, 8, 6), 16), ((40, 44, 3, 8), 32), ((130, 4, 66), 1), ((4, 4, 4, 4, 4), 3),
    ((6, 5, 7), 5), ((36, 36, 36), 65),
    # small I_n with several runs of the head: run packing in the 128 MMA rows
    ((64, 10, 40), 25), ((32, 16, 6, 40), 16), ((8, 64, 30), 12),
]


@pytest.mark.parametrize("dims,C", TC_SHAPES)
@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
def test_shapes(dims, C, prec):
    X, dims, U = synth.random_case(dims, C, seed=7 * sum(dims) + C)
    check_all_modes(X, dims, U, prec)


@pytest.mark.parametrize("splits", [1, 3, 17])
def test_splits(splits):
    X, dims, U = synth.random_case((64, 48, 96), 25, seed=9)
    check_all_modes(X, dims, U, "bf16x2", splits=splits)


@pytest.mark.parametrize("algo", ["materialized", "two_step"])
@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
def test_other_algorithms(algo, prec):
    X, dims, U = synth.random_case((24, 20, 16, 12), 12, seed=10)
    check_all_modes(X, dims, U, prec, algo=algo)


def test_deterministic():
    X, dims, U = synth.random_case((64, 40, 80), 25, seed=11)
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    for n in range(3):
        a = mtk.mttkrp(Xd, dims, Ud, n, precision="bf16x2").clone()
        b = mtk.mttkrp(Xd, dims, Ud, n, precision="bf16x2").clone()
        assert torch.equal(a, b)


def test_status_clean():
    X, dims, U = synth.random_case((64, 40, 80), 25, seed=12)
    ws = mtk.Workspace()
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    for n in range(3):
        mtk.mttkrp(Xd, dims, Ud, n, precision="bf16x2", ws=ws)
    assert ws.status() == 0
