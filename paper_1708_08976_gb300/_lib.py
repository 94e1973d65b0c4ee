"""ctypes loader for libmttkrp.so with the signatures of include/mttkrp.h.

The library is built in-tree by ``_build.build()``.  Loading fails loudly if it
is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

_lib = None

P = ctypes.c_void_p
I32 = ctypes.c_int
I64 = ctypes.c_int64
SZ = ctypes.c_size_t
U32P = ctypes.POINTER(ctypes.c_uint32)

MTK_OK, MTK_EINVAL, MTK_ECUDA, MTK_ENOTPD, MTK_ETIMEOUT, MTK_EUNSUPPORTED, MTK_EWORKSPACE = 0, 1, 3, 4, 5, 6, 7
ALGO_AUTO, ALGO_FUSED, ALGO_MATERIALIZED, ALGO_TWO_STEP = 0, 1, 2, 3
PREC_AUTO, PREC_FP32, PREC_BF16X2, PREC_BF16X3 = 0, 1, 2, 3


class MtkOpts(ctypes.Structure):
    _fields_ = [("algo", I32), ("precision", I32), ("splits", I32), ("wait_us", I32), ("test_stall", I32),
                ("normalize", I32), ("reserved", I32 * 2)]


OPTS_P = ctypes.POINTER(MtkOpts)

BATCH_MAXN = 4
BATCH_MAXP = 192


class MtkBatchProblem(ctypes.Structure):
    """mtk_batch_problem of include/mttkrp.h."""
    _fields_ = [("X", P), ("U", P * BATCH_MAXN), ("dims", I64 * BATCH_MAXN), ("N", I32), ("n", I32),
                ("C", I32), ("M", P)]


BATCH_P = ctypes.POINTER(MtkBatchProblem)

# name -> (restype, argtypes); mirrors include/mttkrp.h
SIGNATURES = {
    "mtk_status_string": (ctypes.c_char_p, [I32]),
    "mtk_version": (I32, []),
    "mtk_launch_count": (ctypes.c_uint64, []),
    "mtk_clear_status": (I32, [P, P]),
    "mtk_read_status": (I32, [P, P, U32P]),
    "mtk_khatri_rao": (I32, [P, P, I32, I32, P, I32, P]),
    "mtk_mttkrp_workspace": (SZ, [P, I32, I32, I32, OPTS_P]),
    "mtk_mttkrp": (I32, [P, P, I32, P, I32, I32, P, P, SZ, OPTS_P, P]),
    "mtk_mttkrp_noalloc": (I32, [P, P, I32, P, I32, I32, P, OPTS_P, U32P, P]),
    "mtk_split_rows0": (I64, [I64]),
    "mtk_split_pitch": (I64, [P, I32]),
    "mtk_split_bytes": (SZ, [P, I32]),
    "mtk_split_workspace": (SZ, [P, I32]),
    "mtk_split_tensor": (I32, [P, P, I32, P, P, P, SZ, P]),
    "mtk_mttkrp_split_workspace": (SZ, [P, I32, I32, I32, OPTS_P]),
    "mtk_mttkrp_split": (I32, [P, P, P, I32, P, I32, I32, P, P, SZ, OPTS_P, P]),
    "mtk_mttkrp_all_split_workspace": (SZ, [P, I32, I32, OPTS_P]),
    "mtk_mttkrp_all_split": (I32, [P, P, I32, P, I32, P, P, SZ, OPTS_P, P]),
    "mtk_ffma_probe_out_floats": (I64, [I32]),
    "mtk_ffma_probe": (I32, [I32, I32, P, P, P]),
    "mtk_sym_packed_rows": (I64, [I64, I32]),
    "mtk_pack_symmetric": (I32, [P, P, I32, I32, P, P]),
    "mtk_mttkrp_sym_split_workspace": (SZ, [P, I32, I32, I32, I32, OPTS_P]),
    "mtk_mttkrp_sym_split": (I32, [P, P, I32, I32, P, I32, I32, P, P, SZ, OPTS_P, P]),
    "mtk_mttkrp_batched_workspace": (SZ, [BATCH_P, I32, OPTS_P]),
    "mtk_mttkrp_batched": (I32, [BATCH_P, I32, P, SZ, OPTS_P, P]),
    "mtk_partial_mttkrp_workspace": (SZ, [P, I32, I32, I32, I32, OPTS_P]),
    "mtk_partial_mttkrp": (I32, [P, P, I32, P, I32, I32, I32, P, P, SZ, OPTS_P, P]),
    "mtk_partial_mttkrp_split_workspace": (SZ, [P, I32, I32, I32, I32, OPTS_P]),
    "mtk_partial_mttkrp_split": (I32, [P, P, I32, P, I32, I32, I32, P, P, SZ, OPTS_P, P]),
    "mtk_multi_ttv": (I32, [P, P, I32, P, I32, I32, I32, P, P]),
    "mtk_gram_workspace": (SZ, [I64, I32]),
    "mtk_gram": (I32, [P, I64, I32, P, P, SZ, P]),
    "mtk_solve_workspace": (SZ, [I64, I32]),
    "mtk_gram_hadamard_solve": (I32, [P, I32, I32, I32, P, I64, P, P, P, SZ, P]),
    "mtk_norm2_workspace": (SZ, [I64]),
    "mtk_norm2": (I32, [P, I64, P, P, SZ, P]),
    "mtk_cp_als_workspace": (SZ, [P, I32, I32, OPTS_P]),
    "mtk_cp_als_sweep": (I32, [P, P, I32, P, I32, P, P, P, SZ, OPTS_P, P]),
    "mtk_cp_als_sweep_split": (I32, [P, P, P, I32, P, I32, P, P, P, SZ, OPTS_P, P]),
    "mtk_cp_residual": (I32, [P, P, P, I64, P, I32, I32, P, P, P]),
    "mtk_cp_loss": (I32, [P, P, P, I64, P, I32, I32, P, P]),
    "mtk_cp_gradient": (I32, [P, P, P, I32, I32, I32, I64, P, P, P]),
}


class MtkError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmttkrp.so (building it first if needed).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"libmttkrp.so not built at {_build.LIB}")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(st: int) -> str:
    return load().mtk_status_string(int(st)).decode()


def check(st: int, what: str) -> None:
    if st != MTK_OK:
        raise MtkError(st, what)


def opts(algo=ALGO_AUTO, precision=PREC_AUTO, splits=0, wait_us=0, test_stall=0, normalize=0):
    o = MtkOpts()
    o.algo = int(algo)
    o.precision = int(precision)
    o.splits = int(splits)
    o.wait_us = int(wait_us)
    o.test_stall = int(test_stall)
    o.normalize = int(normalize)
    return o


def dims_arr(dims):
    return (I64 * len(dims))(*[int(d) for d in dims])


def ptr_arr(ptrs):
    arr = (P * len(ptrs))()
    for k, p in enumerate(ptrs):
        arr[k] = None if p is None else int(p)
    return arr
