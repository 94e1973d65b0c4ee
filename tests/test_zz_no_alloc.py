"""mtk_mttkrp_noalloc (the MTTKRP entry point that allocates nothing: its workspace is
a fixed device array inside the library) against mtk_mttkrp with a caller workspace,
through the C ABI, on consecutive calls that share the fixed array.

Collected last on purpose: it must pass in a fresh process and after every other
test has run kernels and left the library state behind."""
import ctypes

import numpy as np
import pytest

import synth
from helpers import rel_fro
from paper_1708_08976_gb300 import _lib as L

TOL = 1e-5      # relative Frobenius bound used by the MTTKRP parity tests


def _call_noalloc(lib, Xp, dims, Up, C, n, Mp, o, bits, stream):
    return lib.mtk_mttkrp_noalloc(Xp, L.dims_arr(dims), len(dims), L.ptr_arr(Up), C, n, Mp,
                                  ctypes.byref(o), bits, stream)


def test_noalloc_rejects_oversize_before_launch():
    """The size check runs on the host before anything touches a device (the
    pointers here are never dereferenced): the materialised KRP of a 200x200x300x40
    tensor needs far more than the fixed array."""
    lib = L.load()
    dims = [200, 200, 300, 40]
    o = L.opts(algo=L.ALGO_MATERIALIZED, precision=L.PREC_FP32)
    assert lib.mtk_mttkrp_workspace(L.dims_arr(dims), 4, 25, 3, ctypes.byref(o)) > 16 << 20
    fake = [4096 * (k + 1) for k in range(4)]
    st = _call_noalloc(lib, 1 << 20, dims, fake, 25, 3, 1 << 21, o, None, None)
    assert st == L.MTK_EWORKSPACE


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()
    return torch


def _reference(torch, lib, Xd, dims, Ud, C, n, o, stream):
    need = lib.mtk_mttkrp_workspace(L.dims_arr(dims), len(dims), C, n, ctypes.byref(o))
    assert need > 0
    ws = torch.zeros(need, dtype=torch.uint8, device="cuda")
    M = torch.empty((dims[n], C), dtype=torch.float32, device="cuda")
    st = lib.mtk_mttkrp(Xd.data_ptr(), L.dims_arr(dims), len(dims),
                        L.ptr_arr([u.data_ptr() for u in Ud]), C, n, M.data_ptr(), ws.data_ptr(),
                        need, ctypes.byref(o), stream)
    assert st == L.MTK_OK
    bits = ctypes.c_uint32(0)
    assert lib.mtk_read_status(ws.data_ptr(), stream, ctypes.byref(bits)) == L.MTK_OK
    return M.double().cpu().numpy()


def _noalloc(torch, lib, Xd, dims, Ud, C, n, o, stream):
    M = torch.full((dims[n], C), float("nan"), dtype=torch.float32, device="cuda")
    bits = ctypes.c_uint32(0xFFFFFFFF)
    st = _call_noalloc(lib, Xd.data_ptr(), dims, [u.data_ptr() for u in Ud], C, n, M.data_ptr(), o,
                       ctypes.byref(bits), stream)
    assert st == L.MTK_OK, L.status_string(st)
    assert bits.value == 0
    return M.double().cpu().numpy()


def _inputs(torch, dims, C, seed):
    g = np.random.default_rng(seed)
    X = g.standard_normal(int(np.prod(dims)), dtype=np.float32)
    U = [g.random((d, C), dtype=np.float32) for d in dims]
    return torch.from_numpy(X).cuda(), [torch.from_numpy(u).cuda() for u in U]


CASES = [
    ("fp32", L.ALGO_FUSED), ("bf16x2", L.ALGO_FUSED), ("bf16x3", L.ALGO_FUSED),
    ("fp32", L.ALGO_TWO_STEP), ("bf16x3", L.ALGO_TWO_STEP), ("bf16x2", L.ALGO_MATERIALIZED),
]
PREC = {"fp32": L.PREC_FP32, "bf16x2": L.PREC_BF16X2, "bf16x3": L.PREC_BF16X3}


@pytest.mark.gpu
@pytest.mark.parametrize("prec,algo", CASES)
def test_noalloc_matches_mttkrp_small(torch_cuda, prec, algo):
    """A ragged 3-way shape (several tiles, ragged tails), every mode, each mode's
    call made twice in a row; consecutive calls change the plan and so the layout
    of the shared array."""
    torch = torch_cuda
    lib = L.load()
    dims, C = [37, 23, 290], 20
    Xd, Ud = _inputs(torch, dims, C, 11)
    o = L.opts(algo=algo, precision=PREC[prec])
    stream = torch.cuda.current_stream().cuda_stream
    for n in range(3):
        ref = _reference(torch, lib, Xd, dims, Ud, C, n, o, stream)
        for _ in range(2):
            got = _noalloc(torch, lib, Xd, dims, Ud, C, n, o, stream)
            assert np.isfinite(got).all()
            assert rel_fro(got, ref) < TOL, (prec, algo, n)


@pytest.mark.gpu
def test_noalloc_matches_mttkrp_corr4(torch_cuda):
    """The 200x200x300x40, C = 25 workload in the benchmark's precision, every mode,
    two passes over the modes; no device memory is taken by these calls."""
    torch = torch_cuda
    lib = L.load()
    X, dims, U = synth.corr4()
    dims = list(dims)
    C = U[0].shape[1]
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in U]
    o = L.opts(algo=L.ALGO_FUSED, precision=L.PREC_BF16X2)
    stream = torch.cuda.current_stream().cuda_stream
    refs = [_reference(torch, lib, Xd, dims, Ud, C, n, o, stream) for n in range(4)]
    outs = [torch.empty((dims[n], C), dtype=torch.float32, device="cuda") for n in range(4)]
    bits = ctypes.c_uint32(0)
    _call_noalloc(lib, Xd.data_ptr(), dims, [u.data_ptr() for u in Ud], C, 0, outs[0].data_ptr(), o,
                  ctypes.byref(bits), stream)       # set-up call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        for n in range(4):
            outs[n].fill_(float("nan"))
            st = _call_noalloc(lib, Xd.data_ptr(), dims, [u.data_ptr() for u in Ud], C, n,
                               outs[n].data_ptr(), o, ctypes.byref(bits), stream)
            assert st == L.MTK_OK and bits.value == 0, (n, L.status_string(st))
            assert rel_fro(outs[n].double().cpu().numpy(), refs[n]) < TOL, n
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


@pytest.mark.gpu
def test_noalloc_oversize_leaves_output(torch_cuda):
    torch = torch_cuda
    lib = L.load()
    dims, C = [64, 64, 64, 64], 16
    Xd, Ud = _inputs(torch, dims, C, 3)
    o = L.opts(algo=L.ALGO_MATERIALIZED, precision=L.PREC_FP32)
    assert lib.mtk_mttkrp_workspace(L.dims_arr(dims), 4, C, 0, ctypes.byref(o)) > 16 << 20
    M = torch.full((dims[0], C), 7.0, device="cuda")
    st = _call_noalloc(lib, Xd.data_ptr(), dims, [u.data_ptr() for u in Ud], C, 0, M.data_ptr(), o,
                       None, torch.cuda.current_stream().cuda_stream)
    assert st == L.MTK_EWORKSPACE
    torch.cuda.synchronize()
    assert bool((M == 7.0).all())
