"""Tensors symmetric in modes 0 and 1, stored packed (the paper's fMRI variant with the
pair of region modes kept as one mode of a triangle's entries, Section 5.3.3), through
the C ABI.

* mtk_pack_symmetric against the packing written out in numpy: bit-exact, padding rows
  zero; with the diagonal (a >= b) and without it (a > b, the paper's 19,900-row form).
* mtk_mttkrp_sym_split (BF16 planes of the packed tensor) against the FP64 oracle's
  MTTKRP of the FULL symmetric tensor (its diagonal zeroed for the form without it),
  every mode, with different U_0 and U_1 so that the symmetrised pair products and the
  triangle walk of modes 0 and 1 are both exercised; row counts with every remainder
  mod 8 (the ragged padding of the packed mode).
* shapes outside the path: dims[0] != dims[1] and N = 2 are refused on the host.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08976_gb300 as mtk  # noqa: E402
from paper_1708_08976_gb300 import _lib as L  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mtk.load()


def symmetric_case(n0, rest, C, seed):
    """X symmetric in modes 0 and 1 (the FP32 mean of a normal draw and its transpose),
    factors N(0, 1) with U_0 != U_1."""
    dims = (n0, n0) + tuple(rest)
    Y, _, U = synth.random_case(dims, C, seed, np.float32)
    Yn = synth.as_natural(Y, dims)
    Xn = (Yn + Yn.swapaxes(0, 1)) * np.float32(0.5)
    X = np.asfortranarray(Xn).reshape(-1, order="F")
    return np.ascontiguousarray(X), dims, U


def packed_numpy(X, dims, diag):
    """The packed layout written out: row by row of a, the entries X(a, b, r) with b <= a
    (diag) or b < a, each row r of the packed tensor Pp long."""
    n0 = dims[0]
    rest = int(np.prod(dims[2:]))
    rows = n0 * (n0 + 1) // 2 if diag else n0 * (n0 - 1) // 2
    m = 64 if rows >= 2048 else 8
    Pp = (rows + m - 1) // m * m
    X3 = X.reshape(rest, n0, n0)                   # [r, b, a]
    out = np.zeros((rest, Pp), dtype=X.dtype)
    p = 0
    for a in range(n0):
        k = a + 1 if diag else a
        out[:, p:p + k] = X3[:, :k, a]
        p += k
    assert p == rows
    return out.reshape(-1), Pp


def zero_diagonal(X, dims):
    Xn = synth.as_natural(X.copy(), dims)
    for a in range(dims[0]):
        Xn[a, a] = 0.0
    return np.ascontiguousarray(np.asfortranarray(Xn).reshape(-1, order="F"))


# n0 (n0 + 1) / 2 mod 8 over these n0: 12 -> 6, 13 -> 3, 16 -> 0, 20 -> 2, 33 -> 1, 10 -> 7, 9 -> 5;
# n0 (n0 - 1) / 2 mod 8: 12 -> 2, 13 -> 6, 16 -> 0, 20 -> 6, 33 -> 0, 10 -> 5, 9 -> 4
SHAPES = [
    ((12, (40,)), 8),
    ((13, (24, 5)), 16),
    ((16, (64,)), 25),
    ((20, (30, 8)), 10),
    ((33, (16, 5)), 12),
    ((10, (8, 6, 3)), 7),
    ((9, (40,)), 64),
    ((330, (2,)), 8),             # n0 above the banded packing's limit (320): the per-entry packing
]


@pytest.mark.parametrize("diag", [True, False])
@pytest.mark.parametrize("shape,C", SHAPES)
def test_pack_symmetric_exact(shape, C, diag):
    n0, rest = shape
    X, dims, _ = symmetric_case(n0, rest, 1, 30 + n0)
    ref, Pp = packed_numpy(X, dims, diag)
    assert mtk.load().mtk_sym_packed_rows(n0, int(diag)) == Pp
    Xp = mtk.pack_symmetric(torch.from_numpy(X).cuda(), dims, diag=diag)
    torch.cuda.synchronize()
    assert np.array_equal(Xp.cpu().numpy(), ref)


@pytest.mark.parametrize("diag", [True, False])
@pytest.mark.parametrize("shape,C", SHAPES)
def test_mttkrp_sym_parity(shape, C, diag):
    n0, rest = shape
    X, dims, U = symmetric_case(n0, rest, C, 50 + n0 + C)
    Xd = torch.from_numpy(X).cuda()
    Xp = mtk.pack_symmetric(Xd, dims, diag=diag)
    Xps, _ = mtk.split_tensor(Xp, mtk.sym_packed_dims(dims, diag=diag))
    Ud = [torch.from_numpy(u).cuda() for u in U]
    X64 = (X if diag else zero_diagonal(X, dims)).astype(np.float64)
    U64 = [u.astype(np.float64) for u in U]
    for n in range(len(dims)):
        M = mtk.mttkrp_sym(Xps, dims, Ud, n, diag=diag)
        ref = oracle.mttkrp(X64, dims, U64, n)
        err = rel_fro(M.double().cpu().numpy(), ref)
        assert err < 1e-5, (dims, C, n, diag, err)


def test_mttkrp_sym_refuses():
    lib = mtk.load()
    o = L.opts()
    # modes 0 and 1 of different sizes, and a 2-way tensor
    assert lib.mtk_mttkrp_sym_split_workspace(L.dims_arr([12, 13, 40]), 3, 1, 8, 2, ctypes.byref(o)) == 0
    assert lib.mtk_mttkrp_sym_split_workspace(L.dims_arr([12, 12]), 2, 1, 8, 0, ctypes.byref(o)) == 0
    X = torch.zeros(12 * 13 * 40, device="cuda")
    Xp = torch.zeros(10000, device="cuda")
    st = lib.mtk_pack_symmetric(X.data_ptr(), L.dims_arr([12, 13, 40]), 3, 1, Xp.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == L.MTK_EINVAL
