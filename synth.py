"""Seeded synthetic inputs for dense MTTKRP / CP-ALS workloads.

This module only draws numbers: it holds none of the MTTKRP, KRP or CP-ALS
arithmetic, and both the FP64 oracle side and the CUDA side of every test and
benchmark take their inputs from here.  Generators are numpy ``PCG64`` streams
(``numpy.random.default_rng(seed)``), drawn in a fixed order.

Tensors are returned as flat arrays in the natural linearization of the
paper (Section 2.1): entry (i_0, ..., i_{N-1}) sits at
l = sum_k i_k * prod_{j<k} I_j, mode 0 fastest.  A C-ordered numpy array of
shape ``dims[::-1]`` has exactly that memory order, which is how the
structured tensors below are assembled.  Factor matrices are ``I_k x C``
row-major.

Workloads (shapes from the paper's experiments, Section 5; the paper's fMRI
data is not available, a synthetic tensor of its shape stands in for it):

* ``tiny3``     60x50x40 FP64 uniform[0,1) (seed 0), rank 8 factors uniform[0,1) (seed 1)
* ``cube512``   512^3 FP32 N(0,1) (seed 2), rank 32 factors N(0,1)/sqrt(32) (seed 3)
* ``corr4``     200x200x300x40 FP32 correlation-shaped: rank-10 CP with factors
                uniform[-1,1], modes 0/1 sharing one factor, its FP32 values
                symmetrised, plus N(0, 0.05^2) noise symmetrised in modes 0/1,
                clipped to [-1,1] (seed 4): exactly symmetric in modes 0/1;
                rank 25 ALS factors uniform[0,1) (seed 5)
* ``cube32x5``  32^5 FP32 rank-16 CP with factors uniform[-1,1] plus N(0, 0.01^2)
                noise (seed 6); rank 16
* ``fd5``       6x5x4x3x2 FP64 N(0,1), rank 3 factors uniform[-1,1] (seed 7)
* ``batch64``   64 3-way FP32 N(0,1) tensors, dims uniform integers in [64, 384],
                ranks from {8, 16, 32} (seed 8)
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def numel(dims) -> int:
    n = 1
    for d in dims:
        n *= int(d)
    return n


def as_natural(X: np.ndarray, dims) -> np.ndarray:
    """View a flat natural-order tensor as an N-d numpy array indexed [i_0, ..., i_{N-1}]."""
    return X.reshape(tuple(int(d) for d in dims), order="F")


def uniform_tensor(dims, seed, dtype=np.float64, lo=0.0, hi=1.0) -> np.ndarray:
    g = rng(seed)
    x = g.random(numel(dims), dtype=np.float64 if dtype == np.float64 else np.float32)
    if lo != 0.0 or hi != 1.0:
        x = x * (hi - lo) + lo
    return x.astype(dtype, copy=False)


def normal_tensor(dims, seed, dtype=np.float32, scale=1.0) -> np.ndarray:
    g = rng(seed)
    x = g.standard_normal(numel(dims), dtype=np.float32 if dtype == np.float32 else np.float64)
    if scale != 1.0:
        x *= scale
    return x.astype(dtype, copy=False)


def uniform_factors(dims, C, seed, dtype=np.float64, lo=0.0, hi=1.0):
    """One stream, factors drawn in mode order."""
    g = rng(seed)
    out = []
    for d in dims:
        u = g.random((int(d), C)) * (hi - lo) + lo
        out.append(u.astype(dtype))
    return out


def normal_factors(dims, C, seed, dtype=np.float32, scale=1.0):
    g = rng(seed)
    return [(g.standard_normal((int(d), C)) * scale).astype(dtype) for d in dims]


def _outer_sum(factors, dtype):
    """sum_a outer(factors[0][:, a], ..., factors[N-1][:, a]) as a flat natural-order
    tensor.  Built as (rows over modes 1..N-1) x (mode 0) with numpy broadcasting
    and one matrix product, which is the memory order of the natural layout."""
    dims = [f.shape[0] for f in factors]
    R = factors[0].shape[1]
    # P[(i_{N-1}, ..., i_1), a] = prod_{k>=1} f_k[i_k, a], i_1 fastest
    P = np.ones((1, R), dtype=np.float64)
    for f in factors[1:]:
        P = (f.astype(np.float64)[:, None, :] * P[None, :, :]).reshape(-1, R)
    X = (P.astype(dtype) @ factors[0].astype(dtype).T)   # rows: modes >= 1, cols: mode 0
    return np.ascontiguousarray(X).reshape(-1), dims


# ---------------------------------------------------------------- workloads
def tiny3():
    dims = (60, 50, 40)
    X = uniform_tensor(dims, 0, np.float64)
    U = uniform_factors(dims, 8, 1, np.float64)
    return X, dims, U


def cube512():
    dims = (512, 512, 512)
    X = normal_tensor(dims, 2, np.float32)
    U = normal_factors(dims, 32, 3, np.float32, scale=1.0 / np.sqrt(32.0))
    return X, dims, U


def corr4(dims=(200, 200, 300, 40), rank_true=10, C=25, seed_x=4, seed_u=5,
          noise=0.05):
    """Correlation-shaped 4-way tensor (regions x regions x time windows x subjects)."""
    assert dims[0] == dims[1]
    g = rng(seed_x)
    A = g.random((dims[0], rank_true)) * 2.0 - 1.0          # shared by modes 0 and 1
    A2 = g.random((dims[2], rank_true)) * 2.0 - 1.0
    A3 = g.random((dims[3], rank_true)) * 2.0 - 1.0
    X, _ = _outer_sum([A, A, A2, A3], np.float32)
    X = X.reshape(dims[3], dims[2], dims[1], dims[0])        # C-order view [i3, i2, i1, i0]
    for i3 in range(dims[3]):
        E = g.standard_normal((dims[2], dims[1], dims[0]), dtype=np.float32) * np.float32(noise)
        E = (E + E.transpose(0, 2, 1)) * np.float32(0.5)     # symmetric in modes 0/1
        blk = X[i3]
        S = blk + blk.transpose(0, 2, 1)                     # the rounded CP part, made
        S *= np.float32(0.5)                                 # exactly symmetric as well
        S += E
        np.clip(S, -1.0, 1.0, out=blk)
    X = X.reshape(-1)
    U = uniform_factors(dims, C, seed_u, np.float32)
    return X, tuple(dims), U


def cube32x5(dims=(32, 32, 32, 32, 32), rank_true=16, C=16, seed=6, noise=0.01):
    g = rng(seed)
    F = [g.random((d, rank_true)) * 2.0 - 1.0 for d in dims]
    X, _ = _outer_sum(F, np.float32)
    X = X + g.standard_normal(X.size, dtype=np.float32) * np.float32(noise)
    U = [g.random((d, C)).astype(np.float32) * 2.0 - 1.0 for d in dims]
    return X.astype(np.float32), tuple(dims), [u.astype(np.float32) for u in U]


def fd5():
    dims = (6, 5, 4, 3, 2)
    g = rng(7)
    X = g.standard_normal(numel(dims))
    U = [g.random((d, 3)) * 2.0 - 1.0 for d in dims]
    return X, dims, U


def batch64(count=64, lo=64, hi=384, ranks=(8, 16, 32), seed=8):
    """List of (X, dims, U) for independent 3-way tensors of uneven sizes."""
    g = rng(seed)
    out = []
    for _ in range(count):
        dims = tuple(int(v) for v in g.integers(lo, hi + 1, size=3))
        C = int(ranks[int(g.integers(0, len(ranks)))])
        X = g.standard_normal(numel(dims), dtype=np.float32)
        U = [g.standard_normal((d, C), dtype=np.float32) / np.float32(np.sqrt(C)) for d in dims]
        out.append((X, dims, U))
    return out


def random_case(dims, C, seed, dtype=np.float64, dist="normal"):
    """Generic small case for parity sweeps: X and factors from one stream."""
    g = rng(seed)
    if dist == "normal":
        X = g.standard_normal(numel(dims))
        U = [g.standard_normal((int(d), C)) for d in dims]
    else:
        X = g.random(numel(dims))
        U = [g.random((int(d), C)) for d in dims]
    return X.astype(dtype), tuple(int(d) for d in dims), [u.astype(dtype) for u in U]


# The paper's synthetic sweep: for N = 3..6 every mode has the same dimension, chosen so
# that the tensor has about 750 million entries, and the rank is 25.  The entry values are
# not stated there; these are uniform in [-1, 1) (FP32 draws), the factors N(0, 1) / sqrt(C).
PAPER_EQUAL_DIMS = {3: 900, 4: 165, 5: 60, 6: 30}


def paper_equal(N, C=25, seed=9):
    dims = (PAPER_EQUAL_DIMS[N],) * N
    X = rng(seed + N).random(numel(dims), dtype=np.float32)
    X *= np.float32(2.0)
    X -= np.float32(1.0)
    U = normal_factors(dims, C, seed + 10 + N, np.float32, scale=1.0 / np.sqrt(C))
    return X, dims, U


# The paper's KRP experiment: Z = 2, 3 or 4 operands with equal row counts whose product
# is about 2e7 output rows, C = 25 or 50, entries uniform in [0, 1).
KRP_ROWS = {2: 4472, 3: 271, 4: 67}


def krp_case(Z, C, seed=20):
    g = rng(seed + 10 * Z + C)
    return [g.random((KRP_ROWS[Z], C), dtype=np.float32) for _ in range(Z)]
