"""FP64 CPU oracle for dense MTTKRP and CP-ALS -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over
fixed chunks so results do not depend on the thread count); this module only
compiles it (``build()``) and marshals numpy arrays.  All tensors are flat
numpy arrays in the natural linearization (mode 0 fastest, Section 2.1 of the
paper); factor matrices are ``I_k x C`` row-major.

Parity: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle.py`` (brute force, closed forms, special cases, finite
differences, hand-derived integer fixtures).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, EINVAL, ENOMEM, ENOTPD = 0, 1, 2, 4


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP, no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "oracle_mttkrp": (i32, [P, P, i32, P, i32, i32, P]),
        "oracle_mttkrp_range": (i32, [P, P, i32, P, i32, i32, i64, i64, P]),
        "oracle_mttkrp_rows_f32": (i32, [P, P, i32, P, i32, i32, P, i32, P]),
        "oracle_mttkrp_brute": (i32, [P, P, i32, P, i32, i32, P]),
        "oracle_krp": (i32, [P, P, i32, i32, P]),
        "oracle_partial_mttkrp": (i32, [P, P, i32, P, i32, i32, i32, P]),
        "oracle_multi_ttv": (i32, [P, P, i32, P, i32, i32, i32, P]),
        "oracle_gram": (i32, [P, i64, i32, P]),
        "oracle_gram_hadamard": (i32, [P, i32, P, i32, i32, P]),
        "oracle_cholesky": (i32, [P, i32, P]),
        "oracle_chol_solve": (i32, [P, i32, P, i64, P]),
        "oracle_norm2": (dbl, [P, i64]),
        "oracle_residual2_explicit": (dbl, [P, P, i32, P, i32]),
        "oracle_residual2_identity": (dbl, [dbl, P, P, i64, P, i32, P, i32]),
        "oracle_als_sweep": (i32, [P, P, i32, P, i32, P]),
        "oracle_als_sweep_opt": (i32, [P, P, i32, P, i32, i32, P]),
        "oracle_normalize_columns": (None, [P, i64, i32, P]),
        "oracle_grad": (i32, [P, P, i32, P, i32, i32, P]),
        "oracle_num_threads": (i32, []),
        "oracle_set_num_threads": (None, [i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


# ----------------------------------------------------------------- marshalling
def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dims(dims: Sequence[int]) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(list(dims), dtype=np.int64))


def _ptrs(mats):
    """array of pointers to the given contiguous float64 matrices (None -> NULL)"""
    arr = (ctypes.c_void_p * len(mats))()
    for k, m in enumerate(mats):
        arr[k] = None if m is None else m.ctypes.data
    return arr


def _check(st, what):
    if st != OK:
        raise OracleError(f"{what} failed with status {st}")


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(t: int) -> None:
    _load().oracle_set_num_threads(int(t))


def _rank(U) -> int:
    """number of columns C of the factor matrices (any non-None one)"""
    for u in U:
        if u is not None:
            return int(np.asarray(u).shape[-1])
    raise OracleError("no factor matrix given")


def _factors(U, dims, C):
    Us = []
    for k, u in enumerate(U):
        if u is None:
            Us.append(None)
            continue
        u = _f64(u).reshape(int(dims[k]), C)
        Us.append(u)
    return Us


def mttkrp(X, dims, U, n) -> np.ndarray:
    """Mode-n MTTKRP by the element-wise definition (Section 2.2). Returns I_n x C."""
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = _factors(U, d, C)
    X = _f64(X).ravel()
    M = np.zeros((int(d[n]), C))
    _check(lib.oracle_mttkrp(X.ctypes.data, d.ctypes.data, len(d), _ptrs(Us), C, n, M.ctypes.data), "mttkrp")
    return M


def mttkrp_range(X_slice, l_begin, l_end, dims, U, n) -> np.ndarray:
    """Contribution of the entries with linear index in [l_begin, l_end) to the
    mode-n MTTKRP; X_slice holds exactly those entries."""
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = _factors(U, d, C)
    Xs = _f64(X_slice).ravel()
    assert Xs.size == l_end - l_begin
    M = np.zeros((int(d[n]), C))
    _check(lib.oracle_mttkrp_range(Xs.ctypes.data, d.ctypes.data, len(d), _ptrs(Us), C, n,
                                   int(l_begin), int(l_end), M.ctypes.data), "mttkrp_range")
    return M


def mttkrp_rows_f32(X32, dims, U, n, rows) -> np.ndarray:
    """Selected rows of the mode-n MTTKRP of an FP32 tensor (entries promoted
    exactly to double). Returns len(rows) x C."""
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = _factors(U, d, C)
    X32 = np.ascontiguousarray(X32, dtype=np.float32).ravel()
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((r.size, C))
    _check(lib.oracle_mttkrp_rows_f32(X32.ctypes.data, d.ctypes.data, len(d), _ptrs(Us), C, n,
                                      r.ctypes.data, int(r.size), out.ctypes.data), "mttkrp_rows_f32")
    return out


def mttkrp_brute(X, dims, U, n) -> np.ndarray:
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = _factors(U, d, C)
    X = _f64(X).ravel()
    M = np.zeros((int(d[n]), C))
    _check(lib.oracle_mttkrp_brute(X.ctypes.data, d.ctypes.data, len(d), _ptrs(Us), C, n, M.ctypes.data), "mttkrp_brute")
    return M


def krp(U) -> np.ndarray:
    """K = U_0 kr ... kr U_{Z-1}, last operand's row index fastest (Section 4.1)."""
    lib = _load()
    Us = [_f64(u) for u in U]
    C = Us[0].shape[1]
    rows = _dims([u.shape[0] for u in Us])
    J = int(np.prod(rows))
    K = np.zeros((J, C))
    _check(lib.oracle_krp(_ptrs(Us), rows.ctypes.data, len(Us), C, K.ctypes.data), "krp")
    return K


def partial_mttkrp(X, dims, U, n, right: bool) -> np.ndarray:
    """First step of Algorithm 4. right: R[l + IL*i + IL*In*c]; left: L[i + In*r + In*IR*c]."""
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = _factors(U, d, C)
    IL = int(np.prod(d[:n])); In = int(d[n]); IR = int(np.prod(d[n + 1:]))
    out = np.zeros((IL * In * C) if right else (In * IR * C))
    X = _f64(X).ravel()
    _check(lib.oracle_partial_mttkrp(X.ctypes.data, d.ctypes.data, len(d), _ptrs(Us), C, n,
                                     1 if right else 0, out.ctypes.data), "partial_mttkrp")
    return out


def multi_ttv(T, dims, U, n, right: bool) -> np.ndarray:
    """Second step of Algorithm 4 on the output of partial_mttkrp."""
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = _factors(U, d, C)
    T = _f64(T).ravel()
    M = np.zeros((int(d[n]), C))
    _check(lib.oracle_multi_ttv(T.ctypes.data, d.ctypes.data, len(d), _ptrs(Us), C, n,
                                1 if right else 0, M.ctypes.data), "multi_ttv")
    return M


def gram(U) -> np.ndarray:
    lib = _load()
    U = _f64(U)
    I, C = U.shape
    G = np.zeros((C, C))
    _check(lib.oracle_gram(U.ctypes.data, I, C, G.ctypes.data), "gram")
    return G


def gram_hadamard(dims, U, n) -> np.ndarray:
    """H = Hadamard over k != n of U_k^T U_k; n = -1 takes every mode."""
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = _factors(U, d, C)
    H = np.zeros((C, C))
    _check(lib.oracle_gram_hadamard(d.ctypes.data, len(d), _ptrs(Us), C, n, H.ctypes.data), "gram_hadamard")
    return H


def cholesky(H) -> np.ndarray:
    lib = _load()
    H = _f64(H)
    C = H.shape[0]
    L = np.zeros((C, C))
    _check(lib.oracle_cholesky(H.ctypes.data, C, L.ctypes.data), "cholesky")
    return L


def chol_solve(L, M) -> np.ndarray:
    lib = _load()
    L = _f64(L); M = _f64(M)
    I, C = M.shape
    U = np.zeros((I, C))
    _check(lib.oracle_chol_solve(L.ctypes.data, C, M.ctypes.data, I, U.ctypes.data), "chol_solve")
    return U


def norm2(X) -> float:
    X = _f64(X).ravel()
    return float(_load().oracle_norm2(X.ctypes.data, X.size))


def residual2_explicit(X, dims, U) -> float:
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = _factors(U, d, C)
    X = _f64(X).ravel()
    return float(lib.oracle_residual2_explicit(X.ctypes.data, d.ctypes.data, len(d), _ptrs(Us), C))


def residual2_identity(normX2, Mm, Um, dims, U) -> float:
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = _factors(U, d, C)
    Mm = _f64(Mm); Um = _f64(Um)
    return float(lib.oracle_residual2_identity(float(normX2), Mm.ctypes.data, Um.ctypes.data,
                                               Mm.shape[0], d.ctypes.data, len(d), _ptrs(Us), C))


def als_sweep(X, dims, U, normalize=False):
    """One CP-ALS sweep (Section 2.2). Returns (new factor list, fit).  normalize: every
    factor but the last scaled to unit column norms after its update (an optional step
    the paper does not have; the last factor carries the weights)."""
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = [u.copy() for u in _factors(U, d, C)]
    X = _f64(X).ravel()
    fit = ctypes.c_double(0.0)
    if normalize:
        _check(lib.oracle_als_sweep_opt(X.ctypes.data, d.ctypes.data, len(d), _ptrs(Us), C, 1,
                                        ctypes.byref(fit)), "als_sweep")
    else:
        _check(lib.oracle_als_sweep(X.ctypes.data, d.ctypes.data, len(d), _ptrs(Us), C,
                                    ctypes.byref(fit)), "als_sweep")
    return Us, fit.value


def normalize_columns(U):
    """(U with unit 2-norm columns, the C norms); zero columns stay zero."""
    lib = _load()
    Un = np.ascontiguousarray(np.array(U, dtype=np.float64))
    lam = np.zeros(Un.shape[1])
    lib.oracle_normalize_columns(Un.ctypes.data, Un.shape[0], Un.shape[1], lam.ctypes.data)
    return Un, lam


def grad(X, dims, U, n) -> np.ndarray:
    """d/dU_n of 0.5 ||X - [[U]]||^2 = U_n H_n - M_n."""
    lib = _load()
    d = _dims(dims)
    C = _rank(U)
    Us = _factors(U, d, C)
    X = _f64(X).ravel()
    G = np.zeros((int(d[n]), C))
    _check(lib.oracle_grad(X.ctypes.data, d.ctypes.data, len(d), _ptrs(Us), C, n, G.ctypes.data), "grad")
    return G


def loss_explicit(X, dims, U) -> float:
    """0.5 ||X - [[U]]||^2 by explicit reconstruction (tiny inputs)."""
    return 0.5 * residual2_explicit(X, dims, U)
