"""CPU-only checks of the C ABI: the library loads and exports every symbol that
include/mttkrp.h declares, and host-side argument checks reject bad calls
before any launch (no GPU needed: nothing here reaches the device)."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from paper_1708_08976_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "mttkrp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(mtk_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_header_symbol():
    lib = L.load()
    names = header_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
        assert name in L.SIGNATURES, f"binding lacks a signature for {name}"


def test_status_strings():
    lib = L.load()
    assert lib.mtk_status_string(L.MTK_OK) == b"ok"
    assert b"positive definite" in lib.mtk_status_string(L.MTK_ENOTPD)
    assert lib.mtk_version() >= 100


def test_workspace_queries_and_bad_shapes():
    lib = L.load()
    d = L.dims_arr([60, 50, 40])
    o = L.opts()
    for n in range(3):
        assert lib.mtk_mttkrp_workspace(d, 3, 8, n, ctypes.byref(o)) >= 256
    assert lib.mtk_mttkrp_workspace(d, 3, 8, 3, ctypes.byref(o)) == 0      # n out of range
    assert lib.mtk_mttkrp_workspace(d, 3, 0, 0, ctypes.byref(o)) == 0      # C < 1
    assert lib.mtk_mttkrp_workspace(d, 3, 257, 0, ctypes.byref(o)) == 0    # C > 256
    assert lib.mtk_mttkrp_workspace(d, 1, 8, 0, ctypes.byref(o)) == 0      # N < 2
    bad = L.dims_arr([60, 0, 40])
    assert lib.mtk_mttkrp_workspace(bad, 3, 8, 0, ctypes.byref(o)) == 0    # zero dim
    huge = L.dims_arr([1 << 31, 1 << 31, 4])
    assert lib.mtk_mttkrp_workspace(huge, 3, 8, 0, ctypes.byref(o)) == 0   # overflow
    for algo in (L.ALGO_FUSED, L.ALGO_MATERIALIZED, L.ALGO_TWO_STEP):
        oa = L.opts(algo=algo)
        assert lib.mtk_mttkrp_workspace(d, 3, 8, 1, ctypes.byref(oa)) >= 256
    assert lib.mtk_cp_als_workspace(d, 3, 8, None) >= 256


def test_null_and_misaligned_pointers_rejected_before_launch():
    lib = L.load()
    d = L.dims_arr([4, 5, 6])
    fake = 0x10000
    U = L.ptr_arr([fake, fake, fake])
    # null X / M / ws
    assert lib.mtk_mttkrp(None, d, 3, U, 2, 0, fake, fake, 1 << 20, None, None) == L.MTK_EINVAL
    assert lib.mtk_mttkrp(fake, d, 3, U, 2, 0, None, fake, 1 << 20, None, None) == L.MTK_EINVAL
    assert lib.mtk_mttkrp(fake, d, 3, U, 2, 0, fake, None, 1 << 20, None, None) == L.MTK_EINVAL
    # misaligned X
    assert lib.mtk_mttkrp(fake + 2, d, 3, U, 2, 0, fake, fake, 1 << 20, None, None) == L.MTK_EINVAL
    # a null factor other than U[n]
    U2 = L.ptr_arr([fake, None, fake])
    assert lib.mtk_mttkrp(fake, d, 3, U2, 2, 0, fake, fake, 1 << 20, None, None) == L.MTK_EINVAL
    # workspace too small
    assert lib.mtk_mttkrp(fake, d, 3, U, 2, 0, fake, fake, 16, None, None) == L.MTK_EWORKSPACE
    # bad precision
    o = L.opts(precision=9)
    assert lib.mtk_mttkrp(fake, d, 3, U, 2, 0, fake, fake, 1 << 20, ctypes.byref(o), None) == L.MTK_EINVAL
    # KRP with a zero-row operand / bad Z
    assert lib.mtk_khatri_rao(U, L.dims_arr([3, 0]), 2, 2, fake, 1, None) == L.MTK_EINVAL
    assert lib.mtk_khatri_rao(U, L.dims_arr([3]), 0, 2, fake, 1, None) == L.MTK_EINVAL
    # fit requested without ||X||^2
    assert lib.mtk_cp_als_sweep(fake, d, 3, U, 2, None, fake, fake, 1 << 30, None, None) == L.MTK_EINVAL
    # the column normalisation: 0 or 1, and only where the one-launch update runs (C <= 64)
    o = L.opts(normalize=2)
    assert lib.mtk_cp_als_sweep(fake, d, 3, U, 2, None, None, fake, 1 << 30, ctypes.byref(o), None) == L.MTK_EINVAL
    o = L.opts(normalize=1)
    assert lib.mtk_cp_als_sweep(fake, d, 3, U, 65, None, None, fake, 1 << 30, ctypes.byref(o),
                                None) == L.MTK_EUNSUPPORTED
    # solve with n out of range
    G = L.ptr_arr([fake, fake, fake])
    assert lib.mtk_gram_hadamard_solve(G, 3, 2, 3, fake, 4, fake, None, fake, 1 << 20, None) == L.MTK_EINVAL


def test_split_and_batched_calls_rejected_before_launch():
    """The planes entry points and the batched entry point check their arguments on the
    host (these calls all fail before any launch)."""
    lib = L.load()
    fake = 0x10000
    d = L.dims_arr([64, 48, 40])
    U = L.ptr_arr([fake, fake, fake])
    # split: mode 0 padded to a multiple of 8, pitch and sizes; bad dims; null / misaligned planes
    assert [lib.mtk_split_rows0(v) for v in (0, 1, 8, 60, 165, 200)] == [0, 8, 8, 64, 168, 200]
    d1 = L.dims_arr([100])
    assert lib.mtk_split_pitch(d1, 1) == 128
    d5 = L.dims_arr([5, 7, 3])
    assert lib.mtk_split_pitch(d5, 3) == 192                      # 8 x 21 = 168 padded entries
    assert lib.mtk_split_bytes(d5, 3) == 4 * 192
    assert lib.mtk_split_pitch(d, 3) == 64 * 48 * 40
    assert lib.mtk_split_workspace(L.dims_arr([0, 4]), 2) == 0
    assert lib.mtk_split_bytes(L.dims_arr([4, 4]), 0) == 0
    assert lib.mtk_split_tensor(fake, d5, 3, None, None, fake, 1 << 20, None) == L.MTK_EINVAL
    assert lib.mtk_split_tensor(fake, d5, 3, fake + 8, None, fake, 1 << 20, None) == L.MTK_EINVAL
    assert lib.mtk_split_tensor(fake, L.dims_arr([5, -1]), 2, fake, None, fake, 1 << 20, None) == L.MTK_EINVAL
    assert lib.mtk_split_tensor(fake, d5, 3, fake, None, fake, 8, None) == L.MTK_EWORKSPACE
    # MTTKRP on the planes: options other than AUTO/BF16X2 and AUTO/FUSED are refused
    for o in (L.opts(precision=L.PREC_FP32), L.opts(precision=L.PREC_BF16X3), L.opts(algo=L.ALGO_TWO_STEP)):
        assert lib.mtk_mttkrp_split_workspace(d, 3, 8, 0, ctypes.byref(o)) == 0
        assert lib.mtk_mttkrp_split(fake, fake, d, 3, U, 8, 0, fake, fake, 1 << 20, ctypes.byref(o),
                                    None) == L.MTK_EINVAL
    assert lib.mtk_mttkrp_split_workspace(d, 3, 8, 0, None) >= 256
    assert lib.mtk_mttkrp_split(None, fake, d, 3, U, 8, 0, fake, fake, 1 << 20, None, None) == L.MTK_EINVAL
    assert lib.mtk_mttkrp_split(fake + 4, fake, d, 3, U, 8, 0, fake, fake, 1 << 20, None, None) == L.MTK_EINVAL
    assert lib.mtk_mttkrp_split(fake, fake, d, 3, U, 8, 0, fake, fake, 16, None, None) == L.MTK_EWORKSPACE
    assert lib.mtk_cp_als_sweep_split(None, fake, d, 3, U, 8, None, None, fake, 1 << 30, None, None) == L.MTK_EINVAL
    # batched: rank, order, count and contraction-length limits
    def prob(dims, n, C, X=fake, M=fake):
        p = L.MtkBatchProblem()
        p.X, p.M, p.N, p.n, p.C = X, M, len(dims), n, C
        for k, dk in enumerate(dims):
            p.dims[k] = dk
            p.U[k] = fake
        return p
    arr = (L.MtkBatchProblem * 1)(prob([8, 9, 10], 1, 16))
    assert lib.mtk_mttkrp_batched_workspace(arr, 1, None) >= 256
    for bad in (prob([8, 9, 10], 1, 33), prob([8, 9, 10], 3, 8), prob([8, 9], 0, 8, X=None),
                prob([8, 9, 10], 0, 8, M=fake + 2), prob([1 << 16, 1 << 16, 2], 2, 8)):
        a1 = (L.MtkBatchProblem * 1)(bad)
        assert lib.mtk_mttkrp_batched_workspace(a1, 1, None) == 0
        assert lib.mtk_mttkrp_batched(a1, 1, fake, 1 << 30, None, None) == L.MTK_EINVAL
    big = (L.MtkBatchProblem * (L.BATCH_MAXP + 1))(*[prob([4, 4, 4], 0, 4) for _ in range(L.BATCH_MAXP + 1)])
    assert lib.mtk_mttkrp_batched(big, L.BATCH_MAXP + 1, fake, 1 << 30, None, None) == L.MTK_EINVAL
    assert lib.mtk_mttkrp_batched(arr, 1, fake, 16, None, None) == L.MTK_EWORKSPACE


def test_partial_split_rejected_before_launch():
    """mtk_partial_mttkrp_split checks the side, the pointers, the options and the
    workspace on the host; shapes the planes kernel does not take return
    MTK_EUNSUPPORTED.  None of these calls reaches the device."""
    lib = L.load()
    fake = 0x10000
    d = L.dims_arr([16, 24, 40, 8])
    U = L.ptr_arr([fake, fake, fake, fake])
    # a contracted side exists: right needs n < N-1, left needs n > 0
    assert lib.mtk_partial_mttkrp_split_workspace(d, 4, 8, 3, 1, None) == 0
    assert lib.mtk_partial_mttkrp_split_workspace(d, 4, 8, 0, 0, None) == 0
    assert lib.mtk_partial_mttkrp_split(fake, d, 4, U, 8, 3, 1, fake, fake, 1 << 30, None, None) == L.MTK_EINVAL
    assert lib.mtk_partial_mttkrp_split(fake, d, 4, U, 8, 0, 0, fake, fake, 1 << 30, None, None) == L.MTK_EINVAL
    for n, right in ((0, 1), (1, 1), (2, 1), (1, 0), (2, 0), (3, 0)):
        need = lib.mtk_partial_mttkrp_split_workspace(d, 4, 8, n, right, None)
        assert need >= 512, (n, right)
        assert lib.mtk_partial_mttkrp_split(fake, d, 4, U, 8, n, right, fake, fake, need - 1, None,
                                            None) == L.MTK_EWORKSPACE
    # null or misaligned planes, null output, a missing factor on the contracted side
    assert lib.mtk_partial_mttkrp_split(None, d, 4, U, 8, 1, 1, fake, fake, 1 << 30, None, None) == L.MTK_EINVAL
    assert lib.mtk_partial_mttkrp_split(fake + 8, d, 4, U, 8, 1, 1, fake, fake, 1 << 30, None, None) == L.MTK_EINVAL
    assert lib.mtk_partial_mttkrp_split(fake, d, 4, U, 8, 1, 1, None, fake, 1 << 30, None, None) == L.MTK_EINVAL
    U_no3 = L.ptr_arr([fake, fake, fake, None])
    assert lib.mtk_partial_mttkrp_split(fake, d, 4, U_no3, 8, 1, 1, fake, fake, 1 << 30, None, None) == L.MTK_EINVAL
    # the factors on the other side are not read (may be NULL)
    U_left_only = L.ptr_arr([fake, None, None, None])
    assert lib.mtk_partial_mttkrp_split(fake, d, 4, U_left_only, 8, 1, 0, fake, fake, 16, None,
                                        None) == L.MTK_EWORKSPACE
    # options other than AUTO/BF16X2 precision and AUTO/FUSED algorithm
    for o in (L.opts(precision=L.PREC_FP32), L.opts(algo=L.ALGO_TWO_STEP)):
        assert lib.mtk_partial_mttkrp_split_workspace(d, 4, 8, 1, 1, ctypes.byref(o)) == 0
        assert lib.mtk_partial_mttkrp_split(fake, d, 4, U, 8, 1, 1, fake, fake, 1 << 30, ctypes.byref(o),
                                            None) == L.MTK_EINVAL
    # shapes outside the planes kernel: C > 64 (I_0 = 6 is taken: the planes pad mode 0 to 8)
    assert lib.mtk_partial_mttkrp_split_workspace(d, 4, 65, 1, 1, None) == 0
    assert lib.mtk_partial_mttkrp_split(fake, d, 4, U, 65, 1, 1, fake, fake, 1 << 30, None,
                                        None) == L.MTK_EUNSUPPORTED
    d_odd = L.dims_arr([6, 5, 3, 3])
    for n in range(1, 4):
        assert lib.mtk_partial_mttkrp_split_workspace(d_odd, 4, 8, n, 0, None) > 0
    for n in range(3):
        assert lib.mtk_partial_mttkrp_split_workspace(d_odd, 4, 8, n, 1, None) > 0


@pytest.mark.parametrize("dims,C", [((200, 200, 300, 40), 25), ((24, 16, 20, 8), 8), ((32, 24, 40), 12),
                                    ((40, 16, 24, 10), 25), ((200, 200, 12, 5), 25), ((64, 48, 40, 8), 64)])
def test_sweep_workspace_covers_tree_partials(dims, C):
    """The CP-ALS workspace query (every sweep form) is at least what the dimension tree
    carves: each partial contraction's own workspace plus the partial tensors it keeps,
    and at least every per-mode planes MTTKRP's workspace (host-side sizes, no launch).
    A sweep runs its planes contractions on one CTA per SM but one (151 on the 152-SM
    GB300 the host-side sizes assume): that SM takes the factorisation overlapped with
    the contraction."""
    lib = L.load()
    N = len(dims)
    d = L.dims_arr(list(dims))
    o = L.opts(algo=L.ALGO_TWO_STEP)
    ws = lib.mtk_cp_als_workspace(d, N, C, ctypes.byref(o))
    assert ws > 0
    parts = 4 * dims[0] * dims[1] * C + (4 * dims[2] * dims[3] * C if N == 4 else 0)
    so = L.opts(splits=151)
    wr = lib.mtk_partial_mttkrp_split_workspace(d, N, C, 1, 1, ctypes.byref(so))
    wl = lib.mtk_partial_mttkrp_split_workspace(d, N, C, 2, 0, ctypes.byref(so)) if N == 4 else 0
    assert wr > 0 and (N == 3 or wl > 0)
    assert ws >= max(wr, wl) + parts
    for n in range(N):
        assert ws >= lib.mtk_mttkrp_split_workspace(d, N, C, n, ctypes.byref(so))


def test_noalloc_scratch_covers_the_benchmark_shapes():
    """The fixed scratch of mtk_mttkrp_noalloc (MTK_NOALLOC_SCRATCH_BYTES, 16 MiB) covers
    the fused and two-step MTTKRPs of the 200x200x300x40 and 60x50x40 workloads in every
    precision, and the fused ones of 512^3.  The two-step form of 512^3 at mode 1 keeps a
    512 x 512 x 32 partial tensor (32 MiB): that call is one the fixed scratch refuses."""
    lib = L.load()
    limit = 16 << 20
    for dims, C, algos in (((200, 200, 300, 40), 25, (L.ALGO_FUSED, L.ALGO_TWO_STEP)),
                           ((60, 50, 40), 8, (L.ALGO_FUSED, L.ALGO_TWO_STEP)),
                           ((512, 512, 512), 32, (L.ALGO_FUSED,))):
        d = L.dims_arr(list(dims))
        for algo in algos:
            for prec in (L.PREC_FP32, L.PREC_BF16X2, L.PREC_BF16X3):
                o = L.opts(algo=algo, precision=prec)
                for n in range(len(dims)):
                    need = lib.mtk_mttkrp_workspace(d, len(dims), C, n, ctypes.byref(o))
                    assert 0 < need <= limit, (dims, algo, prec, n, need)
    d = L.dims_arr([512, 512, 512])
    o = L.opts(algo=L.ALGO_TWO_STEP, precision=L.PREC_FP32)
    assert lib.mtk_mttkrp_workspace(d, 3, 32, 1, ctypes.byref(o)) > limit


def test_symmetric_packed_sizes_and_shapes():
    """Packed rows: n0 (n0 + 1) / 2 (with diagonal) or n0 (n0 - 1) / 2 (without: 200 ->
    19,900 -> 19,904) rounded up to 8; the symmetric MTTKRP takes every mode of the
    200x200x300x40 workload and of small 3- to 5-way shapes, and refuses unequal modes 0/1,
    N = 2 and a diag other than 0/1 (workspace 0) and bad pointers before a launch."""
    lib = L.load()
    assert [lib.mtk_sym_packed_rows(n, 1) for n in (1, 2, 3, 4, 12, 200)] == [8, 8, 8, 16, 80, 20160]
    assert [lib.mtk_sym_packed_rows(n, 0) for n in (1, 2, 3, 5, 12, 200)] == [0, 8, 8, 16, 72, 19904]
    assert lib.mtk_sym_packed_rows(12, 2) == 0
    # from 2048 rows on, a multiple of 64: 63 * 64 / 2 = 2016 rows -> 2016, 64 * 65 / 2 = 2080 -> 2112
    assert [lib.mtk_sym_packed_rows(n, 1) for n in (62, 63, 64)] == [1960, 2016, 2112]
    o = L.opts()
    for dims, C in (((200, 200, 300, 40), 25), ((12, 12, 40), 8), ((13, 13, 24, 5), 16), ((10, 10, 8, 6, 3), 7)):
        d = L.dims_arr(list(dims))
        for diag in (0, 1):
            for n in range(len(dims)):
                assert lib.mtk_mttkrp_sym_split_workspace(d, len(dims), diag, C, n, ctypes.byref(o)) > 0, (dims, n)
    assert lib.mtk_mttkrp_sym_split_workspace(L.dims_arr([12, 13, 40]), 3, 1, 8, 0, ctypes.byref(o)) == 0
    assert lib.mtk_mttkrp_sym_split_workspace(L.dims_arr([12, 12]), 2, 1, 8, 0, ctypes.byref(o)) == 0
    assert lib.mtk_mttkrp_sym_split_workspace(L.dims_arr([12, 12, 40]), 3, 2, 8, 0, ctypes.byref(o)) == 0
    fake = ctypes.c_void_p(1 << 20)
    d = L.dims_arr([12, 12, 40])
    assert lib.mtk_pack_symmetric(None, d, 3, 1, fake, None) == L.MTK_EINVAL
    assert lib.mtk_pack_symmetric(fake, L.dims_arr([12, 13, 40]), 3, 1, fake, None) == L.MTK_EINVAL
    assert lib.mtk_pack_symmetric(fake, d, 3, 2, fake, None) == L.MTK_EINVAL
    for ptrs, n in (([None, 1 << 20, 1 << 20], 2), ([1 << 20, None, None], 0), ([None, 1 << 20, 1 << 20], 1)):
        st = lib.mtk_mttkrp_sym_split(fake, d, 3, 1, L.ptr_arr(ptrs), 8, n, fake, fake, 1 << 30, ctypes.byref(o),
                                      None)
        assert st == L.MTK_EINVAL, (ptrs, n)


def test_corr4_generator_is_exactly_symmetric():
    """The correlation-shaped generator gives X(a, b, ...) == X(b, a, ...) bit for bit."""
    X, dims, _ = synth.corr4(dims=(20, 20, 6, 3))
    Xn = synth.as_natural(X, dims)
    assert np.array_equal(Xn, Xn.swapaxes(0, 1))


def test_ffma_probe_rejects_bad_arguments():
    lib = L.load()
    fake = ctypes.c_void_p(1 << 20)
    assert lib.mtk_ffma_probe_out_floats(0) == 0 and lib.mtk_ffma_probe_out_floats(65) == 0
    assert lib.mtk_ffma_probe_out_floats(1) % 256 == 0
    for cps, iters, out in ((0, 16, fake), (65, 16, fake), (1, 0, fake), (1, (1 << 24) + 1, fake), (1, 16, None),
                            (1, 16, ctypes.c_void_p((1 << 20) + 2))):
        assert lib.mtk_ffma_probe(cps, iters, out, None, None) == L.MTK_EINVAL


def test_norm_and_split_partials_bounded():
    """||X||^2 (mtk_norm2, the split) is summed over at most 1216 fixed chunks of at least
    4096 entries (whatever the device), so the workspace of the partial sums stays small and
    a 134 MB tensor is not left to a few CTAs."""
    lib = L.load()
    status = 256
    cap = status + (1216 * 8 + 255) // 256 * 256
    for I in (1, 4095, 4096, 4097, 1 << 20, 33554432, 480000000, 3 << 30):
        w = lib.mtk_norm2_workspace(I)
        assert status + 256 <= w <= cap, (I, w)
    # a 32^5 tensor (33.5 M entries) gets the full 1216-way split, not 32 chunks of 1 M
    assert lib.mtk_norm2_workspace(33554432) == cap
    assert lib.mtk_norm2_workspace(0) == 0
    for dims in ((200, 200, 300, 40), (900, 900, 900), (5,)):
        w = lib.mtk_split_workspace(L.dims_arr(list(dims)), len(dims))
        assert status + 256 <= w <= cap, (dims, w)
