"""CP-ALS sweeps with the optional column normalisation, and sweeps recorded in a CUDA
graph, through the C ABI.

* normalize: every factor but the last scaled to unit columns after its update.  Three
  sweeps against the FP64 oracle's normalised sweeps (factors and fit), on the FP32 tensor
  (per-mode sweep) and on the planes (per mode and the dimension tree); the scaled factors
  have unit columns; the model [[U]] is the one of the plain sweeps (ALS is equivariant
  under column scaling, pinned on the oracle).
* capture/replay: a sweep replayed from a CUDA graph gives bit for bit the factors and fit
  of the same sweeps launched one by one.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import f32_round, factors_dev, rel_fro, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08976_gb300 as mtk  # noqa: E402
from paper_1708_08976_gb300 import _lib as L  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mtk.load()


FORMS = [
    # (dims, C, ALS keyword arguments)
    ((30, 24, 20), 8, {}),                                   # FP32 tensor, per mode
    ((24, 16, 20, 8), 6, {}),
    ((64, 48, 40), 8, {"presplit": True}),                   # planes, per mode
    ((64, 48, 40), 8, {"presplit": True, "algo": "two_step"}),         # planes, dimension tree
    ((24, 16, 20, 8), 25, {"presplit": True, "algo": "two_step"}),
]


@pytest.mark.parametrize("dims,C,kw", FORMS)
def test_normalized_sweeps_match_oracle(dims, C, kw):
    X, dims, U = synth.random_case(dims, C, seed=101 + C + len(dims), dist="uniform")
    Xr = X.astype(np.float32).astype(np.float64)
    ref = f32_round(U)
    plain = f32_round(U)
    Ud = factors_dev(U, torch)
    als = mtk.ALS(to_dev(X, torch), dims, Ud, normalize=True, **kw)
    N = len(dims)
    for it in range(3):
        ref, ref_fit = oracle.als_sweep(Xr, dims, ref, normalize=True)
        plain, plain_fit = oracle.als_sweep(Xr, dims, plain)
        als.sweep()
        assert als.status() == 0
        got = [u.double().cpu().numpy() for u in Ud]
        for k in range(N):
            err = rel_fro(got[k], ref[k])
            assert err < 5e-5, (dims, kw, it, k, err)
        for k in range(N - 1):
            np.testing.assert_allclose(np.linalg.norm(got[k], axis=0), 1.0, rtol=2e-6)
        assert abs(als.fit.item() - ref_fit) < 1e-5
        assert abs(ref_fit - plain_fit) < 1e-10


def test_normalize_refused_above_c64():
    X, dims, U = synth.random_case((8, 6, 5), 65, seed=3, dist="uniform")
    Ud = factors_dev(U, torch)
    als = mtk.ALS(to_dev(X, torch), dims, Ud, normalize=True)
    with pytest.raises(L.MtkError) as e:
        als.sweep()
    assert e.value.status == L.MTK_EUNSUPPORTED


@pytest.mark.parametrize("dims,C,kw", FORMS + [((64, 48, 40), 8, {"presplit": True, "algo": "two_step",
                                                                  "normalize": True})])
def test_graph_replay_bitwise(dims, C, kw):
    X, dims, U = synth.random_case(dims, C, seed=7 + C, dist="uniform")
    Xd = to_dev(X, torch)
    Ua = factors_dev(U, torch)
    Ub = factors_dev(U, torch)
    a = mtk.ALS(Xd, dims, Ua, **kw)
    b = mtk.ALS(Xd, dims, Ub, **kw)
    b.capture()
    fits_a, fits_b = [], []
    for _ in range(3):
        a.sweep()
        fits_a.append(a.fit.item())
        b.replay()
        fits_b.append(b.fit.item())
    torch.cuda.synchronize()
    assert a.status() == 0 and b.status() == 0
    for k in range(len(dims)):
        assert torch.equal(Ua[k], Ub[k]), (dims, kw, k)
    assert fits_a == fits_b
