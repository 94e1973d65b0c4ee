"""The timeout path of the tensor-core contraction kernels, through the C ABI.

Every device-side wait of those kernels is bounded.  A wait that runs out sets
MTK_ETIMEOUT in the status word; every role of the CTA then stops, waits for the
copies and MMAs it has already started (with a limit that the abort does not
shorten) and the CTA frees its TMEM and returns.  These tests make one wait run
out on purpose: mtk_opts.test_stall makes the MMA issuer first wait on a barrier
that nothing completes, and mtk_opts.wait_us sets a short limit.  Nothing faults
or hangs: the call returns, the status word reports the timeout, the output of a
single-CTA planes launch stays as it was, and the next normal call on the same
context gives the oracle's result."""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import rel_fro
from paper_1708_08976_gb300 import _lib as L

pytestmark = pytest.mark.gpu

WAIT_US = 2000          # 2 ms: the stalled wait gives up long before the default 1 s


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()
    return torch


def _inputs(dims, C, seed):
    g = np.random.default_rng(seed)
    X = g.uniform(-1.0, 1.0, int(np.prod(dims))).astype(np.float32)
    U = [g.uniform(-1.0, 1.0, (d, C)).astype(np.float32) for d in dims]
    return X, U


def _ws(torch, nbytes):
    return torch.zeros(max(int(nbytes), 256), dtype=torch.uint8, device="cuda")


def _status(lib, ws, stream):
    bits = ctypes.c_uint32(0)
    st = lib.mtk_read_status(ws.data_ptr(), stream, ctypes.byref(bits))
    return st, bits.value


@pytest.mark.parametrize("splits", [1, 0])
def test_planes_timeout_reported(torch_cuda, splits):
    """mtk_mttkrp_split on a shape the planes kernel takes (64 x 48 x 40, C = 8, every
    mode).  splits = 1 runs one CTA and no slab reduce, so the output must be left
    untouched; splits = 0 runs one CTA per SM with a slab reduce, which skips its
    writes when the status word holds a timeout."""
    torch = torch_cuda
    lib = L.load()
    stream = torch.cuda.current_stream().cuda_stream
    dims, C = [64, 48, 40], 8
    X, U = _inputs(dims, C, 5)
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in U]
    d = L.dims_arr(dims)
    Xs = torch.empty(lib.mtk_split_bytes(d, 3) // 2, dtype=torch.int16, device="cuda")
    sws = _ws(torch, lib.mtk_split_workspace(d, 3))
    assert lib.mtk_split_tensor(Xd.data_ptr(), d, 3, Xs.data_ptr(), None, sws.data_ptr(), sws.numel(), stream) == 0
    Xr = X.astype(np.float64)
    Ur = [u.astype(np.float64) for u in U]
    for n in range(3):
        stall = L.opts(splits=splits, wait_us=WAIT_US, test_stall=1)
        need = lib.mtk_mttkrp_split_workspace(L.dims_arr(dims), 3, C, n, ctypes.byref(stall))
        assert need > 0
        ws = _ws(torch, need)
        M = torch.full((dims[n], C), 7.0, dtype=torch.float32, device="cuda")
        st = lib.mtk_mttkrp_split(Xs.data_ptr(), None, L.dims_arr(dims), 3, L.ptr_arr([u.data_ptr() for u in Ud]),
                                  C, n, M.data_ptr(), ws.data_ptr(), need, ctypes.byref(stall), stream)
        assert st == L.MTK_OK                         # nothing wrong on the host side
        st, bits = _status(lib, ws, stream)
        assert st == L.MTK_ETIMEOUT and bits == (1 << L.MTK_ETIMEOUT), (n, st, bits)
        assert bool((M == 7.0).all()), n             # no partial result was written
        # the context is still usable: the same call without the stall is exact
        ok = L.opts(splits=splits)
        lib.mtk_clear_status(ws.data_ptr(), stream)
        st = lib.mtk_mttkrp_split(Xs.data_ptr(), None, L.dims_arr(dims), 3, L.ptr_arr([u.data_ptr() for u in Ud]),
                                  C, n, M.data_ptr(), ws.data_ptr(), need, ctypes.byref(ok), stream)
        assert st == L.MTK_OK
        assert _status(lib, ws, stream) == (L.MTK_OK, 0)
        ref = oracle.mttkrp(Xr, dims, Ur, n)
        assert rel_fro(M.double().cpu().numpy(), ref) < 1e-5, n


@pytest.mark.parametrize("prec", [L.PREC_BF16X2, L.PREC_BF16X3])
def test_fp32_tensor_tc_timeout_reported(torch_cuda, prec):
    """mtk_mttkrp on the FP32 tensor with the tcgen05 kernel (64 x 48 x 40, C = 8, every
    mode): the stalled wait is reported, and the next normal call is exact."""
    torch = torch_cuda
    lib = L.load()
    stream = torch.cuda.current_stream().cuda_stream
    dims, C = [64, 48, 40], 8
    X, U = _inputs(dims, C, 6)
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in U]
    Xr = X.astype(np.float64)
    Ur = [u.astype(np.float64) for u in U]
    for n in range(3):
        stall = L.opts(algo=L.ALGO_FUSED, precision=prec, wait_us=WAIT_US, test_stall=1)
        need = lib.mtk_mttkrp_workspace(L.dims_arr(dims), 3, C, n, ctypes.byref(stall))
        ws = _ws(torch, need)
        M = torch.zeros((dims[n], C), dtype=torch.float32, device="cuda")
        st = lib.mtk_mttkrp(Xd.data_ptr(), L.dims_arr(dims), 3, L.ptr_arr([u.data_ptr() for u in Ud]), C, n,
                            M.data_ptr(), ws.data_ptr(), need, ctypes.byref(stall), stream)
        assert st == L.MTK_OK
        st, bits = _status(lib, ws, stream)
        assert st == L.MTK_ETIMEOUT and bits == (1 << L.MTK_ETIMEOUT), (n, st, bits)
        ok = L.opts(algo=L.ALGO_FUSED, precision=prec)
        lib.mtk_clear_status(ws.data_ptr(), stream)
        st = lib.mtk_mttkrp(Xd.data_ptr(), L.dims_arr(dims), 3, L.ptr_arr([u.data_ptr() for u in Ud]), C, n,
                            M.data_ptr(), ws.data_ptr(), need, ctypes.byref(ok), stream)
        assert st == L.MTK_OK
        assert _status(lib, ws, stream) == (L.MTK_OK, 0)
        ref = oracle.mttkrp(Xr, dims, Ur, n)
        assert rel_fro(M.double().cpu().numpy(), ref) < 1e-5, n
