"""GPU parity of the MTTKRP on a tensor stored as two BF16 planes (mtk_split_tensor,
mtk_mttkrp_split, mtk_cp_als_sweep_split) against the FP64 oracle.

* The split itself is checked bit for bit against its definition: hi = bf16_rn(x),
  lo = bf16_rn(x - hi), with the rounding done by torch on the CPU, at i0 + I0p r with
  mode 0 padded to I0p = the next multiple of 8 and zeros in the padding; ||X||^2 against
  the oracle.
* The contraction carries each tensor entry as hi + lo (error <= 2^-16 |x|) and each
  KRP entry as three BF16 pieces, so it is held to the bf16x2 bound derived in
  test_gpu_tc.py: 3x the expected representation error plus 2e-6 for FP32
  accumulation.
The shapes cover each branch of the planes kernel: K-major CTA tiles of up to 128 rows or
of up to 256 rows as two MMA tiles (one or several per mode, ragged last tile), K-major with
the head inside the modes left of n (several runs per row), runs packed into the MMA rows for
small I_n, MN-major (mode 0) with one to four 64-row boxes per CTA or packed runs, ranks
C = 1..64 (one to four 16-column chunks), N = 2..6, heads shorter than one 64-k stage,
several tail factors, explicit CTA counts, and I_0 not a multiple of 8 (the planes pad
mode 0 to the next multiple of 8: U_0's missing rows count as zero, mode 0 and the right
partial drop the padding rows of their output).
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


def bf16x2_bound(Xr, dims, Ur, n, ref):
    M2 = oracle.mttkrp(Xr * Xr, dims, [u * u for u in Ur], n)
    rho = np.sqrt(max(M2.sum(), 0.0)) / max(np.linalg.norm(ref), 1e-300)
    return 3.0 * 2.0 ** -16 / np.sqrt(3.0) * rho + 2e-6


def planes_ref(X32: torch.Tensor):
    """hi, lo by their definition, BF16 round-to-nearest-even on the CPU (torch)."""
    x = X32.cpu()
    hi = x.to(torch.bfloat16)
    lo = (x - hi.to(torch.float32)).to(torch.bfloat16)
    return hi.view(torch.int16), lo.view(torch.int16)


@pytest.mark.parametrize("dims", [(1,), (7,), (64,), (1000,), (4099,), (262147,), (8, 9), (5, 7, 3),
                                  (13, 40), (60, 50, 40), (1, 9, 2), (165, 31, 7), (30, 30, 30, 4)])
def test_split_planes_bits_and_norm(dims):
    n_entries = int(np.prod(dims))
    g = np.random.default_rng(n_entries)
    X = (g.standard_normal(n_entries) * np.exp(g.uniform(-20, 20, n_entries))).astype(np.float32)
    X[::13] = 0.0
    Xd = torch.from_numpy(X).cuda()
    Xs, nx2 = mtk.split_tensor(Xd, dims)
    torch.cuda.synchronize()
    lib = L.load()
    I0 = dims[0]
    I0p = (I0 + 7) // 8 * 8
    assert lib.mtk_split_rows0(I0) == I0p
    rest = n_entries // I0
    pitch = lib.mtk_split_pitch(L.dims_arr(list(dims)), len(dims))
    assert pitch % 64 == 0 and pitch >= I0p * rest
    hi, lo = planes_ref(Xd)
    got = Xs.cpu()
    idx = (torch.arange(I0).view(1, I0) + I0p * torch.arange(rest).view(rest, 1)).reshape(-1)
    assert torch.equal(got[idx], hi)
    assert torch.equal(got[pitch + idx], lo)
    pad = torch.ones(pitch, dtype=torch.bool)
    pad[idx] = False
    pad[I0p * rest:] = False                         # beyond the padded tensor: not written
    assert bool((got[:pitch][pad] == 0).all()) and bool((got[pitch:][pad] == 0).all())
    ref = oracle.norm2(X.astype(np.float64))
    assert abs(nx2.item() - ref) <= 1e-12 * ref


def test_split_special_values():
    """The rounding of the split against torch's round-to-nearest-even on the CPU, bit for
    bit, at the edges: signed zeros, subnormals, ties to even in the normal and subnormal
    ranges, the largest finite numbers (rounding up to infinity), infinities and NaN; both
    the 4-wide path (I_0 % 8 == 0) and the padded one."""
    f = np.float32
    tiny = np.float32(2.0 ** -149)
    vals = [0.0, -0.0, tiny, -tiny, 3 * tiny, 2.0 ** -126, -(2.0 ** -126) * (1 + 2.0 ** -8),
            2.0 ** -133 * (1 + 2.0 ** -8), 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8),
            1 + 2.0 ** -8 + 2.0 ** -20, 1 - 2.0 ** -24, np.finfo(f).max, -np.finfo(f).max,
            3.3895314e38, 3.3961514e38, np.inf, -np.inf, np.nan, 65504.0, 1e-30, -7.0e-39]
    base = np.array(vals, dtype=f)
    g = np.random.default_rng(3)
    for I0 in (8, 13):
        n = I0 * 24
        X = (g.standard_normal(n) * np.exp(g.uniform(-80, 80, n))).astype(f)
        X[: base.size * 5: 5] = base
        dims = (I0, 24)
        Xd = torch.from_numpy(X).cuda()
        Xs, _ = mtk.split_tensor(Xd, dims)
        torch.cuda.synchronize()
        lib = L.load()
        I0p = lib.mtk_split_rows0(I0)
        pitch = lib.mtk_split_pitch(L.dims_arr(list(dims)), 2)
        hi, lo = planes_ref(Xd)
        got = Xs.cpu()
        idx = (torch.arange(I0).view(1, I0) + I0p * torch.arange(24).view(24, 1)).reshape(-1)
        for a, b in ((got[idx], hi), (got[pitch + idx], lo)):
            # NaN encodings differ between implementations: NaN where torch has NaN, the
            # same bits everywhere else
            na, nb = bf16_isnan(a), bf16_isnan(b)
            assert torch.equal(na, nb), I0
            assert torch.equal(a[~na], b[~nb]), I0


def bf16_isnan(v: torch.Tensor) -> torch.Tensor:
    w = v.to(torch.int32) & 0xFFFF
    return ((w & 0x7F80) == 0x7F80) & ((w & 0x7F) != 0)


@pytest.mark.parametrize("dims", [(165, 31, 7), (64, 48, 40), (1000,)])
def test_split_from_pinned_host_memory(dims):
    """The split reads a pinned host tensor in place: the same planes and the same ||X||^2,
    bit for bit, as from the device copy; pageable host memory is refused before any launch."""
    n_entries = int(np.prod(dims))
    X = np.random.default_rng(7 + n_entries).standard_normal(n_entries).astype(np.float32)
    Xh = torch.from_numpy(X).pin_memory()
    Xs_d, nx_d = mtk.split_tensor(Xh.cuda(), dims)
    Xs_h, nx_h = mtk.split_tensor(Xh, dims, device="cuda")
    torch.cuda.synchronize()
    lib = L.load()
    d = L.dims_arr(list(dims))
    nxp = lib.mtk_split_rows0(dims[0]) * (n_entries // dims[0])
    pitch = lib.mtk_split_pitch(d, len(dims))
    assert Xs_h.is_cuda
    for a in (0, pitch):                             # the written entries of hi and lo
        assert torch.equal(Xs_h[a:a + nxp], Xs_d[a:a + nxp])
    assert nx_h.item() == nx_d.item()
    ws = torch.zeros(lib.mtk_split_workspace(d, len(dims)), dtype=torch.uint8, device="cuda")
    st = lib.mtk_split_tensor(X.ctypes.data, d, len(dims), Xs_h.data_ptr(), None, ws.data_ptr(), ws.numel(),
                              torch.cuda.current_stream().cuda_stream)
    assert st == L.MTK_EINVAL


def run_split(X, dims, U, n, C, splits=0, with_x=True):
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    Xs, _ = mtk.split_tensor(Xd, dims)
    M = mtk.mttkrp(Xd if with_x else None, dims, Ud, n, Xs=Xs, splits=splits)
    torch.cuda.synchronize()
    return M.double().cpu().numpy()


SHAPES = [
    # (dims, C): comment = what the modes exercise
    ((64, 48, 40), 8),            # MN 64 rows; K-major L=64; 5-D map (head U_0 inside I^L=3072), packed I=40
    ((200, 64, 30), 25),          # MN two tiles (72-row tail, two boxes); K-major packed 64 -> U=2
    ((160, 40, 48), 17),          # MN ragged last tile of 32 rows (one box); heads of 40 rows (< one stage)
    ((32, 64, 16), 16),           # MN packed (I_0 = 32, U = 2 runs); K-major I=64
    ((32, 300, 20), 32),          # K-major three tiles of 104 rows over I = 300, head of 32 rows
    ((256, 200), 33),             # N = 2: MN with one run; K-major with no tail
    ((40, 40, 30, 8), 25),        # two tail factors; packed I = 8 (U = 16)
    ((64, 16, 24, 40), 48),       # 5-D map with Lq = 384, packed U = 3
    ((8, 8, 8, 8, 8), 64),        # N = 5, C = 64 (four chunks), packed U = 16
    ((24, 136, 72), 1),           # C = 1; K-major two tiles (72 + 64 rows)
    ((512, 8, 24), 16),           # MN two CTA tiles of 256 rows (two MMA tiles each)
    ((16, 456, 12), 32),          # K-major CTA tiles of 232 + 224 rows (two MMA tiles, ragged)
    ((200, 200, 8), 25),          # K-major 200 rows in one CTA; head of 200 rows: padding k-steps skipped
    ((60, 50, 40), 8),            # I_0 = 60 padded to 64: mode 0 drops 4 rows, U_0 rows 60..63 zero
    ((165, 9, 20), 25),           # I_0 = 165 -> 168; mode 0 three tiles (the last ragged)
    ((5, 24, 40, 8), 16),         # I_0 = 5 -> 8: heads of mostly padding
    ((30, 30, 30, 4), 12),        # 30 -> 32 with a short head
    ((7, 6, 5, 4, 3, 2), 9),      # N = 6, every mode
    ((64, 65, 32, 3), 16),        # mode 2: 65 runs per row packed 8 at a time in row-local groups (the
                                  # last of each row has one run), no divisor of 65 near 8
]


# Shapes whose I^L (natural layout) is not a multiple of 8 at some mode: with mode 0 padded
# in the planes every row is aligned.  (dims, C, modes the planes kernel must take without
# the FP32 tensor)
UNALIGNED_SHAPES = [
    ((12, 6, 10), 8, (0, 1, 2)),          # I_0 = 12 -> 16
    ((20, 10, 7, 8), 25, (0, 1, 2, 3)),   # 20 -> 24, packed runs
    ((6, 4, 10, 5), 12, (0, 1, 2, 3)),    # 6 -> 8
    ((5, 8, 9), 8, (0, 1, 2)),            # 5 -> 8
    ((3, 16, 11, 2), 16, (0, 1, 2, 3)),   # 3 -> 8: heads of 3 real rows in 8
    ((100, 3000, 3), 25, (0, 1, 2)),      # 100 -> 104; mode 1: 3000 rows (12 tiles); mode 2: head
                                          # of 104 rows (the 312000-row one exceeds the image budget)
    ((30, 30, 4, 6), 33, (0, 1, 2, 3)),   # 30 -> 32; C = 33 (three chunks)
]


@pytest.mark.parametrize("dims,C,modes", UNALIGNED_SHAPES)
def test_mttkrp_split_unaligned(dims, C, modes):
    """The planes kernel on shapes whose natural rows are not 16-byte aligned, against the
    oracle, without the FP32 tensor to fall back to."""
    X, dims, U = synth.random_case(dims, C, seed=13 * sum(dims) + C)
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    for n in modes:
        ref = oracle.mttkrp(Xr, dims, Ur, n)
        got = run_split(X, dims, U, n, C, with_x=False)
        err = rel_fro(got, ref)
        tol = bf16x2_bound(Xr, dims, Ur, n, ref)
        assert err < tol, (dims, C, n, err, tol)


@pytest.mark.parametrize("dims,C", SHAPES)
def test_mttkrp_split_parity(dims, C):
    X, dims, U = synth.random_case(dims, C, seed=11 * sum(dims) + C)
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    for n in range(len(dims)):
        ref = oracle.mttkrp(Xr, dims, Ur, n)
        got = run_split(X, dims, U, n, C)
        err = rel_fro(got, ref)
        tol = bf16x2_bound(Xr, dims, Ur, n, ref)
        assert err < tol, (dims, C, n, err, tol)


def test_mttkrp_split_without_fp32_tensor():
    """Shapes the planes kernel takes need no FP32 tensor (60x50x40: I_0 = 60 padded to 64
    in the planes); others (C > 64) report EUNSUPPORTED, and run the FP32-input path when
    the FP32 tensor is given."""
    for shape in ((64, 48, 40), (60, 50, 40)):
        X, dims, U = synth.random_case(shape, 8, seed=5)
        Xr = X.astype(np.float32).astype(np.float64)
        Ur = f32_round(U)
        for n in range(3):
            ref = oracle.mttkrp(Xr, dims, Ur, n)
            got = run_split(X, dims, U, n, 8, with_x=False)
            assert rel_fro(got, ref) < bf16x2_bound(Xr, dims, Ur, n, ref), (shape, n)
    X, dims, U = synth.random_case((24, 20, 16), 80, seed=6)
    Xd = to_dev(X, torch)
    Xs, _ = mtk.split_tensor(Xd, dims)
    with pytest.raises(mtk.MtkError) as ei:
        mtk.mttkrp(None, dims, factors_dev(U, torch), 0, Xs=Xs)
    assert ei.value.status == L.MTK_EUNSUPPORTED
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    ref = oracle.mttkrp(Xr, dims, Ur, 0)
    got = run_split(X, dims, U, 0, 80)
    assert rel_fro(got, ref) < bf16x2_bound(Xr, dims, Ur, 0, ref)


@pytest.mark.parametrize("splits", [1, 3, 500])
def test_mttkrp_split_cta_counts(splits):
    """One CTA, a few, and a request for more CTAs than the plan allows (capped at four
    stages per CTA)."""
    X, dims, U = synth.random_case((48, 96, 24), 16, seed=splits)
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    for n in range(3):
        ref = oracle.mttkrp(Xr, dims, Ur, n)
        got = run_split(X, dims, U, n, 16, splits=splits)
        assert rel_fro(got, ref) < bf16x2_bound(Xr, dims, Ur, n, ref), (splits, n)


def test_mttkrp_split_deterministic():
    X, dims, U = synth.random_case((72, 64, 50), 25, seed=3)
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    Xs, _ = mtk.split_tensor(Xd, dims)
    for n in range(3):
        a = mtk.mttkrp(Xd, dims, Ud, n, Xs=Xs).clone()
        b = mtk.mttkrp(Xd, dims, Ud, n, Xs=Xs)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_split_rejects_bad_options():
    X, dims, U = synth.random_case((64, 48, 40), 8, seed=5)
    Xd = to_dev(X, torch)
    Xs, _ = mtk.split_tensor(Xd, dims)
    for kw in ({"precision": "fp32"}, {"precision": "bf16x3"}, {"algo": "two_step"}):
        with pytest.raises(ValueError):
            mtk.mttkrp(Xd, dims, factors_dev(U, torch), 0, Xs=Xs, **kw)


@pytest.mark.parametrize("case", ["tiny3", "all_planes", "tiny3_host", "all_planes_host"])
def test_als_sweep_split(case):
    """One CP-ALS sweep on the planes against the oracle's sweep (tiny3 has a mode that
    falls back to the FP32 tensor).  *_host: X is a pinned host tensor, split in place and
    (tiny3) read in place by the fallback mode."""
    host = case.endswith("_host")
    case = case.replace("_host", "")
    if case == "tiny3":
        X, dims, U = synth.tiny3()
    else:
        X, dims, U = synth.random_case((64, 48, 40), 8, seed=9, dist="uniform")
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    ref_U, ref_fit = oracle.als_sweep(Xr, dims, Ur)
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).pin_memory() if host else to_dev(X, torch)
    Ud = factors_dev(U, torch)
    als = mtk.ALS(Xd, dims, Ud, presplit=True)
    als.sweep()
    assert als.status() == 0
    for k in range(len(dims)):
        err = rel_fro(Ud[k].double().cpu().numpy(), ref_U[k])
        assert err < 2e-5, (case, k, err)
    assert abs(als.fit.item() - ref_fit) < 2e-6
    assert abs(als.normX2.item() - oracle.norm2(Xr)) <= 1e-12 * oracle.norm2(Xr)


def test_corr4_split_full_M():
    """Every mode of the 200x200x300x40 workload in the benchmark's configuration (one
    CTA per SM), the whole M against the FP64 oracle: <= 1e-5 and within the bound."""
    X, dims, U = synth.corr4()
    X64 = X.astype(np.float64)
    U64 = [u.astype(np.float64) for u in U]
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in U]
    Xs, nx2 = mtk.split_tensor(Xd, dims)
    assert abs(nx2.item() - oracle.norm2(X64)) <= 1e-12 * oracle.norm2(X64)
    for n in range(4):
        ref = oracle.mttkrp(X64, dims, U64, n)
        got = mtk.mttkrp(None, dims, Ud, n, Xs=Xs).double().cpu().numpy()
        err = rel_fro(got, ref)
        assert err < 1e-5, (n, err)
        tol = bf16x2_bound(X64, dims, U64, n, ref)
        assert err < tol, (n, err, tol)


@pytest.mark.parametrize("dims,C", [((24, 16, 20, 8), 8), ((32, 24, 40), 12), ((40, 16, 24, 10), 25),
                                    ((30, 20, 12, 7), 8), ((13, 31, 9), 10)])
def test_als_sweep_dimension_tree(dims, C):
    """The dimension-tree sweep (algo two_step on the planes: partials over modes >= 2 and
    over modes 0, 1 shared by two updates each) against the oracle's Gauss-Seidel sweep,
    and against the per-mode sweep on the same planes."""
    X, dims, U = synth.random_case(dims, C, seed=sum(dims) + C, dist="uniform")
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    ref_U, ref_fit = oracle.als_sweep(Xr, dims, Ur)
    Xd = to_dev(X, torch)
    Ut = factors_dev(U, torch)
    tree = mtk.ALS(Xd, dims, Ut, presplit=True, algo="two_step")
    tree.sweep()
    assert tree.status() == 0
    Up = factors_dev(U, torch)
    per = mtk.ALS(Xd, dims, Up, presplit=True)
    per.sweep()
    for k in range(len(dims)):
        err = rel_fro(Ut[k].double().cpu().numpy(), ref_U[k])
        assert err < 5e-5, (dims, k, err)
        assert rel_fro(Ut[k].double().cpu().numpy(), Up[k].double().cpu().numpy()) < 5e-5
    assert abs(tree.fit.item() - ref_fit) < 1e-5


def partial_bound(Xr, dims, Ur, n, right, ref):
    """The bf16x2 bound of bf16x2_bound, with the partial MTTKRP of the squared inputs
    in place of the MTTKRP (the same sums, over one side of n only)."""
    T2 = oracle.partial_mttkrp(Xr * Xr, dims, [u * u for u in Ur], n, right)
    rho = np.sqrt(max(T2.sum(), 0.0)) / max(np.linalg.norm(ref), 1e-300)
    return 3.0 * 2.0 ** -16 / np.sqrt(3.0) * rho + 2e-6


PARTIAL_SHAPES = [
    # (dims, C): every (n, side) with a contracted side that the planes kernel takes
    ((24, 16, 20, 8), 8),         # the 4-way tree shape; I^L = 24 at n = 1 (left), 384 at n = 2
    ((32, 24, 40), 12),           # 3-way; left at n = 2 is the mode-2 MTTKRP's view
    ((40, 16, 24, 10), 25),       # C = 25 (two 16-column chunks)
    ((8, 6, 5, 4, 3), 5),         # N = 5: several factors on each side
    ((64, 48, 40), 33),           # C = 33 (three chunks); MN view of 64 rows (n = 0, right)
    ((200, 200, 12, 5), 25),      # tall right view at n = 1: 40000 rows, many CTAs
    ((5, 24, 40, 8), 8),          # I_0 = 5 (8 in the planes): right partials drop the padding rows
    ((6, 5, 8, 3), 8),            # I_0 = 6: left views over the padded I^L = 8 and 40
]


@pytest.mark.parametrize("dims,C", PARTIAL_SHAPES)
def test_partial_split_parity(dims, C):
    """First step of Algorithm 4 on the planes (mtk_partial_mttkrp_split) against the
    oracle's partial MTTKRP by its element-wise definition, for every mode and side."""
    X, dims, U = synth.random_case(dims, C, seed=7 * sum(dims) + C)
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    Xs, _ = mtk.split_tensor(Xd, dims)
    N = len(dims)
    ran = 0
    for n in range(N):
        for right in (True, False):
            if (right and n == N - 1) or (not right and n == 0):
                continue
            got = mtk.partial_mttkrp_split(Xs, dims, Ud, n, right)
            torch.cuda.synchronize()
            ref = oracle.partial_mttkrp(Xr, dims, Ur, n, right)
            err = rel_fro(got.double().cpu().numpy(), ref.reshape(-1))
            tol = partial_bound(Xr, dims, Ur, n, right, ref)
            assert err < tol, (dims, C, n, right, err, tol)
            ran += 1
    assert ran == 2 * (N - 1)


def test_partial_split_factors_off_side_unused_and_repeatable():
    """Only the factors on the contracted side are read (the others may be None), the
    output is overwritten, and two calls give the same bits (fixed-order reduction)."""
    X, dims, U = synth.random_case((24, 16, 20, 8), 8, seed=3)
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    Xs, _ = mtk.split_tensor(Xd, dims)
    a = mtk.partial_mttkrp_split(Xs, dims, [None, None, Ud[2], Ud[3]], 1, True)
    b = torch.full_like(a, float("nan"))
    mtk.partial_mttkrp_split(Xs, dims, Ud, 1, True, out=b)
    c = mtk.partial_mttkrp_split(Xs, dims, [Ud[0], Ud[1], None, None], 2, False)
    d = mtk.partial_mttkrp_split(Xs, dims, Ud, 2, False)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(c, d)
    assert mtk.default_workspace(Xd.device).status() == 0


def test_corr4_tree_partials_full():
    """The two partials of the dimension tree on the 200x200x300x40 workload in the
    benchmark's launch configuration (modes >= 2 at n = 1, 40000 x 25; modes 0, 1 at
    n = 2, 12000 x 25), whole outputs against the FP64 oracle."""
    X, dims, U = synth.corr4()
    X64 = X.astype(np.float64)
    U64 = [u.astype(np.float64) for u in U]
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in U]
    Xs, _ = mtk.split_tensor(Xd, dims)
    del Xd
    for n, right in ((1, True), (2, False)):
        got = mtk.partial_mttkrp_split(Xs, dims, Ud, n, right).double().cpu().numpy()
        ref = oracle.partial_mttkrp(X64, dims, U64, n, right).reshape(-1)
        err = rel_fro(got, ref)
        assert err < 1e-5, (n, right, err)
        tol = partial_bound(X64, dims, U64, n, right, ref)
        assert err < tol, (n, right, err, tol)


@pytest.mark.parametrize("splits", [1, 5, 7])
def test_partial_split_units_back_to_back(splits):
    """Views with more units (tile, slab) than CTAs: each CTA runs several units back to
    back, with its rings, barrier phases and accumulator buffers carried over.  One CTA,
    and CTA counts that do not divide the units, on an MN-major view (n = 1, right:
    3072 rows, 256-row tiles) and a K-major one (n = 2, left: 320 rows)."""
    X, dims, U = synth.random_case((64, 48, 40, 8), 16, seed=100 + splits)
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    Xs, _ = mtk.split_tensor(Xd, dims)
    for n, right in ((1, True), (2, False)):
        got = mtk.partial_mttkrp_split(Xs, dims, Ud, n, right, splits=splits)
        ref = oracle.partial_mttkrp(Xr, dims, Ur, n, right)
        err = rel_fro(got.double().cpu().numpy(), ref.reshape(-1))
        tol = partial_bound(Xr, dims, Ur, n, right, ref)
        assert err < tol, (splits, n, right, err, tol)
        again = mtk.partial_mttkrp_split(Xs, dims, Ud, n, right, splits=splits)
        assert torch.equal(got, again)


@pytest.mark.parametrize("dims,C", [((24, 16, 20, 8), 8), ((30, 20, 12, 7), 16), ((13, 31, 9), 10),
                                    ((8, 6, 5, 4, 3), 5), ((7, 6, 5, 4, 3, 2), 9), ((12, 10, 9, 8, 7), 33)])
@pytest.mark.parametrize("algo", ["auto", "fused"])
def test_mttkrp_all_split(dims, C, algo):
    """Every mode's MTTKRP with the same factors (mtk_mttkrp_all_split): the dimension tree
    (algo auto: N = 3, 4, and N = 5, 6 with one-mode contractions of the left partial;
    C = 33 > I_0 I_1 / 4 keeps N = 5 on per-mode MTTKRPs) or N planes MTTKRPs, each against
    the oracle."""
    X, dims, U = synth.random_case(dims, C, seed=11 * sum(dims) + C)
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    Xd = to_dev(X, torch)
    Ud = factors_dev(U, torch)
    Xs, _ = mtk.split_tensor(Xd, dims)
    Ms = mtk.mttkrp_all(Xs, dims, Ud, algo=algo)
    torch.cuda.synchronize()
    for n in range(len(dims)):
        ref = oracle.mttkrp(Xr, dims, Ur, n)
        err = rel_fro(Ms[n].double().cpu().numpy(), ref)
        assert err < bf16x2_bound(Xr, dims, Ur, n, ref), (dims, algo, n, err)


@pytest.mark.parametrize("dims,C", [((24, 16, 20, 8), 8), ((13, 31, 9), 6)])
def test_cp_loss_gradient_on_planes(dims, C):
    """The CP loss and its gradient with the MTTKRPs on the planes (the backward through
    mttkrp_all: the dimension tree) against the oracle's FP64 gradient.  The factors are
    random, far from a fixed point, so the gradient U_n H_n - M_n does not cancel: it
    carries the MTTKRP's bf16x2 error, held to 2e-5."""
    X, dims, U = synth.random_case(dims, C, seed=5 * sum(dims) + C)
    Xr = X.astype(np.float32).astype(np.float64)
    Ur = f32_round(U)
    Xd = to_dev(X, torch)
    Xs, _ = mtk.split_tensor(Xd, dims)
    Ud = [u.requires_grad_(True) for u in factors_dev(U, torch)]
    loss = mtk.cp_loss(Xd, dims, Ud, Xs=Xs)
    loss.backward()
    np.testing.assert_allclose(loss.item(), oracle.loss_explicit(Xr, dims, Ur), rtol=2e-5)
    for n in range(len(dims)):
        ref = oracle.grad(Xr, dims, Ur, n)
        assert rel_fro(Ud[n].grad.double().cpu().numpy(), ref) < 2e-5, n
    # ||X||^2 passed in (from the split), and only one factor's gradient wanted (the forward
    # then takes the last mode's MTTKRP alone and the backward mode 0's): the same numbers
    _, nx2 = mtk.split_tensor(Xd, dims)
    Uo = [u.detach().clone() for u in Ud]
    Uo[0].requires_grad_(True)
    loss1 = mtk.cp_loss(Xd, dims, Uo, Xs=Xs, normX2=nx2)
    loss1.backward()
    np.testing.assert_allclose(loss1.item(), oracle.loss_explicit(Xr, dims, Ur), rtol=2e-5)
    assert rel_fro(Uo[0].grad.double().cpu().numpy(), oracle.grad(Xr, dims, Ur, 0)) < 2e-5
    assert all(u.grad is None for u in Uo[1:])
