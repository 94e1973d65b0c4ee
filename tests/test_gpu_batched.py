"""GPU parity of the batched MTTKRP (mtk_mttkrp_batched: many independent problems in one
persistent launch) against the FP64 oracle.

The batched kernel is the FP32 CUDA-core form (FP32 products and accumulation), so it is
held to the FP32 bound of test_gpu_parity.py: 2e-6 relative Frobenius error on the
FP32-rounded inputs.  Cases: uneven 3-way tensors (all modes), N = 2 and N = 4
problems, ranks 1..32 (8-, 16- and 32-column blocks), ragged row tiles and k-chunks,
every autotuner candidate, determinism, CUDA-graph replay, more than one launch's worth
of problems, rejected inputs, and the 64-tensor workload on sampled rows against the
sequential per-problem launches.
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

TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mtk.load()


def make_problems(cases, seed):
    """cases: list of (dims, C); every mode of every tensor becomes a problem."""
    probs, refs = [], []
    for t, (dims, C) in enumerate(cases):
        X, dims, U = synth.random_case(dims, C, seed=seed + 31 * t)
        Xd = to_dev(X, torch)
        Ud = factors_dev(U, torch)
        Xr = X.astype(np.float32).astype(np.float64)
        Ur = f32_round(U)
        for n in range(len(dims)):
            out = torch.empty((dims[n], C), dtype=torch.float32, device="cuda")
            probs.append((Xd, dims, Ud, n, out))
            refs.append(oracle.mttkrp(Xr, dims, Ur, n))
    return probs, refs


CASES = [((17, 33, 9), 1), ((64, 5, 130), 8), ((7, 300, 11), 16), ((40, 41, 42), 25), ((129, 3, 70), 32),
         ((600, 9), 12), ((6, 5, 4, 3), 30), ((1, 50, 20), 7)]


def check(probs, refs, tol=TOL):
    for (X, dims, U, n, out), ref in zip(probs, refs):
        err = rel_fro(out.double().cpu().numpy(), ref)
        assert err < tol, (dims, n, int(out.shape[1]), err)


def test_batched_parity():
    probs, refs = make_problems(CASES, seed=3)
    mtk.mttkrp_batched(probs)
    torch.cuda.synchronize()
    check(probs, refs)


@pytest.mark.parametrize("splits", [16, 64, 1000, 4096, 1 << 20])
def test_batched_chunk_sizes(splits):
    """Every k-extent of the work units gives the same result within the bound (16: many
    ragged chunks; 1 << 20: one chunk per problem, written without the reduce)."""
    probs, refs = make_problems(CASES[:5], seed=5)
    mtk.mttkrp_batched(probs, splits=splits)
    torch.cuda.synchronize()
    check(probs, refs)


def test_batched_deterministic_and_graph_replay():
    probs, refs = make_problems(CASES, seed=7)
    plan = mtk.BatchedMTTKRP(probs)
    plan.run()
    torch.cuda.synchronize()
    first = [p[4].clone() for p in probs]
    check(probs, refs)
    for p in probs:
        p[4].zero_()
    plan.capture()
    plan.replay()
    torch.cuda.synchronize()
    for a, p in zip(first, probs):
        assert torch.equal(a, p[4])
    for p in probs:
        p[4].fill_(float("nan"))
    plan.replay()
    torch.cuda.synchronize()
    for a, p in zip(first, probs):
        assert torch.equal(a, p[4])


def test_batched_autotuner_picks_a_candidate():
    probs, refs = make_problems(CASES[:4], seed=9)
    plan = mtk.BatchedMTTKRP(probs)
    choice = plan.tune(reps=2)
    assert choice in mtk.BatchedMTTKRP.CANDIDATES
    plan.run()
    torch.cuda.synchronize()
    check(probs, refs)


def test_batched_more_problems_than_one_launch():
    cases = [((9 + t % 7, 8 + t % 5, 6 + t % 3), 4 + t % 5) for t in range(70)]   # 210 problems
    probs, refs = make_problems(cases, seed=11)
    assert len(probs) > L.BATCH_MAXP
    plan = mtk.BatchedMTTKRP(probs)
    plan.run()
    torch.cuda.synchronize()
    check(probs, refs)


def test_batched_rejects_bad_problems():
    X, dims, U = synth.random_case((8, 9, 10), 40, seed=1)     # C > 32
    out = torch.empty((8, 40), device="cuda")
    with pytest.raises(ValueError):
        mtk.mttkrp_batched([(to_dev(X, torch), dims, factors_dev(U, torch), 0, out)])
    X, dims, U = synth.random_case((2, 3, 2, 2, 2), 4, seed=1)  # N > 4
    out = torch.empty((2, 4), device="cuda")
    with pytest.raises(ValueError):
        mtk.mttkrp_batched([(to_dev(X, torch), dims, factors_dev(U, torch), 0, out)])


def test_batch64_workload_against_sequential_launches():
    """64 uneven 3-way tensors (dims in [64, 384], C in {8, 16, 32}): all 192 MTTKRPs in one
    graph-replayed launch, against the FP32 per-problem mtk_mttkrp launches and, on sampled
    rows, the FP64 oracle."""
    batch = synth.batch64()
    probs, seq = [], []
    for X, dims, U in batch:
        Xd = torch.from_numpy(X).cuda()
        Ud = [torch.from_numpy(u).cuda() for u in U]
        C = U[0].shape[1]
        for n in range(3):
            probs.append((Xd, dims, Ud, n, torch.empty((dims[n], C), device="cuda")))
    plan = mtk.BatchedMTTKRP(probs)
    plan.tune(reps=2)
    plan.capture()
    plan.replay()
    torch.cuda.synchronize()
    g = np.random.default_rng(64)
    for t, (X, dims, U) in enumerate(batch):
        U64 = [u.astype(np.float64) for u in U]
        for n in range(3):
            out = probs[3 * t + n][4]
            ref_seq = mtk.mttkrp(probs[3 * t + n][0], dims, probs[3 * t + n][2], n, precision="fp32")
            assert rel_fro(out.double().cpu().numpy(), ref_seq.double().cpu().numpy()) < 4e-6
            if t % 8 == 0:
                rows = np.unique(np.concatenate([[0, dims[n] - 1], g.integers(0, dims[n], 4)]))
                ref = oracle.mttkrp_rows_f32(X, dims, U64, n, rows)
                got = out[torch.as_tensor(rows, device="cuda")].double().cpu().numpy()
                assert rel_fro(got, ref) < TOL, (t, n)
