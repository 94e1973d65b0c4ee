#!/usr/bin/env python3
"""Benchmark: dense MTTKRP throughput inside CP-ALS on one GB300.

Workload (default): the correlation-shaped 4-way FP32 tensor 200x200x300x40
(regions x regions x time windows x subjects, 480M entries, 1.92 GB), rank
C = 25.  One step = one CP-ALS sweep through the C ABI: for each of the 4 modes
the MTTKRP, the FP64 factor update and the Gram of the new factor, then the fit.
The tensor is split once into its two BF16 planes (timed apart, and inside every
e2e step, where the split reads the step's tensor from pinned host memory); the sweep runs on the planes either with per-mode MTTKRPs or with the
dimension tree (two partial contractions shared by two modes each), the tree
also replayed from a CUDA graph of the whole sweep, and the fastest form is
reported.  Metric = useful MTTKRP flops (4 modes x 2*I*C) per
second of the whole sweep.

Roofline: the dominant kernel is timed alone with CUDA events on its launch
stream (the tree's partial contractions, or the per-mode MTTKRPs); achieved =
its algorithmic bytes (the tensor once, the factors read, the output written)
over that time, against the measured HBM copy bandwidth.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Dense MTTKRP TFLOP/s & roofline %, mixed-precision vs FP32 at stated rel err"

# DRAM bytes (read + write) per launch of the planes contraction on the full
# 200x200x300x40 workload, from ncu dram__bytes_read.sum + dram__bytes_write.sum on the
# 200x200x30x40 case (the same plan shapes, a tensor 10x smaller): reads scaled by 10;
# writes (the output and the partial slabs of tiles split between CTAs, a few MB) taken
# as measured.
#   tree: mean of the two partials (n = 1 right: 192.32 MB read, 3.86 MB written;
#         n = 2 left: 204.49 MB read, 0.09 MB written) -> 1.9271e9 and 2.0450e9 per
#         full launch, 1.002x and 1.065x their algorithmic bytes.
#   planes (per-mode MTTKRPs): None (the bench's dominant kernel is the tree's).
NCU_TRAFFIC_PER_LAUNCH = {"planes": None, "tree": 1.9861e9}
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="corr4",
                    choices=["corr4", "cube512", "corr4-small", "corr4-mid", "paper-synth", "krp", "corr4-sym",
                             "dims", "cube512-forms", "cube32x5-grad"],
                    help="paper-synth: the paper's equal-dimension tensors (N = 3..6, ~7.3e8 entries, "
                         "C = 25), every mode's MTTKRP timed and checked on sampled rows; krp: the "
                         "Khatri-Rao product with and without reuse (Z = 2..4, ~2e7 rows, C = 25, 50); "
                         "corr4-sym: corr4 stored packed in its symmetric modes 0/1, every mode's MTTKRP "
                         "from the packed planes, and a CP-ALS sweep of the packed 3-way tensor; "
                         "each prints its own line")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only run every mode's MTTKRP W+K times (for profiler captures)")
    ap.add_argument("--dims", default="165,165,165,8",
                    help="--workload dims: the tensor's dims (entries uniform[-1,1), factors N(0,1)/sqrt(C))")
    ap.add_argument("--rank", type=int, default=25, help="--workload dims: the rank C")
    ap.add_argument("--modes", default="", help="--kernel-only: the modes to run (default: all)")
    ap.add_argument("--precision", default="best", help="fp32 | bf16x2 | bf16x3 | planes | best")
    ap.add_argument("--algo", default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-tensor batched measurement")
    ap.add_argument("--sweep", default="best", choices=["best", "per-mode", "tree"],
                    help="CP-ALS sweep form on the planes: per-mode MTTKRPs or the dimension tree")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


def workload(name):
    if name == "corr4":
        X, dims, U = synth.corr4()
        desc = "corr4: 200x200x300x40 FP32 correlation-shaped (rank-10 CP, modes 0/1 symmetric, N(0,0.05^2) noise, clipped), rank C=25, factors uniform[0,1)"
    elif name == "corr4-small":
        X, dims, U = synth.corr4(dims=(200, 200, 30, 40))
        desc = "corr4-small: 200x200x30x40 FP32 correlation-shaped (same per-mode I_n as corr4, 1/10 of the entries), rank C=25"
    elif name == "corr4-mid":
        X, dims, U = synth.corr4(dims=(200, 200, 300, 12))
        desc = "corr4-mid: 200x200x300x12 FP32 correlation-shaped (the mode-2 view of corr4 with 12 subjects), rank C=25"
    elif name == "dims":
        dims = tuple(int(v) for v in ARGS.dims.split(","))
        X = synth.uniform_tensor(dims, 31, np.float32, -1.0, 1.0)
        U = synth.normal_factors(dims, ARGS.rank, 32, np.float32, scale=1.0 / np.sqrt(ARGS.rank))
        desc = f"dims: {'x'.join(map(str, dims))} FP32 uniform[-1,1), rank C={ARGS.rank}"
    else:
        X, dims, U = synth.cube512()
        desc = "cube512: 512^3 FP32 N(0,1), rank C=32, factors N(0,1)/sqrt(32)"
    return X, tuple(dims), U, desc


def ffma_peak(mtk, torch):
    """The device's FP32 FMA throughput (TFLOP/s) from the library's FMA probe: the best
    of three CUDA-event timings of one launch (8 CTAs of 256 threads per SM, 8 independent
    chains per thread)."""
    mtk.ffma_probe(8, 256)
    best = 0.0
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        flops = mtk.ffma_probe(8, 65536)
        b.record()
        b.synchronize()
        best = max(best, flops / (a.elapsed_time(b) * 1e-3) / 1e12)
    return best


def time_calls(fn, reps, warm=2, stream=None):
    """Average device time of one fn() call: `reps` calls back to back between two CUDA
    events (the host enqueues faster than the GPU runs them, so host-side launch work
    does not show up as GPU time)."""
    import torch
    for _ in range(warm):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) * 1e-3 / reps


def tree_partials(N):
    """(n, right) of the partial contractions in a dimension-tree sweep of an N-way
    tensor: modes >= 2 at n = 1 (right), and for N = 4 modes 0, 1 at n = 2 (left)."""
    return [(1, True), (2, False)] if N == 4 else [(1, True)]


def partial_bytes(dims, C, n, right):
    """Algorithmic bytes of one partial contraction on the planes: the tensor once
    (4 B per entry over both planes), the factors on the contracted side, the output."""
    I = 1
    for d in dims:
        I *= d
    side = range(n + 1, len(dims)) if right else range(0, n)
    rows = I
    for k in side:
        rows //= dims[k]
    return 4.0 * I + 4.0 * C * sum(dims[k] for k in side) + 4.0 * rows * C


def max_over_ranks(t, world, device):
    """The job's time per step: the slowest rank's (an all-reduce MAX over the replicas of
    the process group; the tensor lives on `device`, a GPU under NCCL, the CPU under gloo)."""
    if world == 1:
        return float(t)
    import torch
    import torch.distributed as dist
    x = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def job_value(flops_step, world, t_max):
    """Whole-job TFLOP/s: every replica does flops_step per step, the job takes t_max."""
    return world * flops_step / t_max / 1e12


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(X, dims, U, C, budget_s=12.0):
    """The FP64 oracle, as it stands, on a bounded prefix of the tensor for every mode."""
    import oracle
    Ud = [u.astype(np.float64) for u in U]
    N = len(dims)
    # calibrate on a small prefix, then size the sample to the time budget
    n0 = 1 << 18
    t0 = time.perf_counter()
    for n in range(N):
        oracle.mttkrp_range(X[:n0].astype(np.float64), 0, n0, dims, Ud, n)
    dt = time.perf_counter() - t0
    n_s = int(min(X.size, max(n0, n0 * budget_s / max(dt, 1e-6))))
    n_s -= n_s % 1024
    Xs = X[:n_s].astype(np.float64)
    t0 = time.perf_counter()
    for n in range(N):
        oracle.mttkrp_range(Xs, 0, n_s, dims, Ud, n)
    dt = time.perf_counter() - t0
    flops = N * 2.0 * n_s * C
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {n_s} of {X.size} entries (natural order), all {N} modes, FP64 definition loop, {dt:.1f} s"}


def batch_measure(mtk, torch, dev, hbm_peak):
    """The 64-tensor batch (dims uniform in [64, 384], C in {8, 16, 32}): all 3 modes of
    every tensor (192 MTTKRPs) as one graph-replayed persistent launch, against the same
    192 MTTKRPs as sequential per-problem launches of the FP32 path."""
    batch = synth.batch64()
    probs = []
    flops = 0.0
    nbytes = 0.0
    for X, dims, U in batch:
        Xd = torch.from_numpy(X).to(dev)
        Ud = [torch.from_numpy(u).to(dev) for u in U]
        C = U[0].shape[1]
        for n in range(3):
            probs.append((Xd, dims, Ud, n, torch.empty((dims[n], C), dtype=torch.float32, device=dev)))
            flops += 2.0 * X.size * C
            nbytes += 4.0 * X.size + 4.0 * C * (sum(dims) - dims[n]) + 4.0 * dims[n] * C
    plan = mtk.BatchedMTTKRP(probs)
    choice = plan.tune()
    plan.capture()
    t_batch = time_calls(plan.replay, 10)
    outs = [p[4].clone() for p in probs]

    def seq():
        for X, dims, U, n, out in probs:
            mtk.mttkrp(X, dims, U, n, precision="fp32", out=out)
    t_seq = time_calls(seq, 3, warm=1)
    diff = max(float(torch.linalg.norm(a - p[4]) / torch.linalg.norm(p[4])) for a, p in zip(outs, probs))
    return {"workload": "64 3-way FP32 tensors, dims uniform in [64,384], C in {8,16,32}, N(0,1) (seed 8); "
                        "all 3 modes (192 MTTKRPs)",
            "batched_graph_us": t_batch * 1e6, "batched_tflops": flops / t_batch / 1e12,
            "batched_hbm_frac": nbytes / t_batch / 1e9 / hbm_peak,
            "sequential_us": t_seq * 1e6, "sequential_tflops": flops / t_seq / 1e12,
            "speedup": t_seq / t_batch, "autotuned_k_per_unit": choice,
            "max_rel_diff_vs_sequential": diff, "launches_per_batch": 2,
            "arith": "FP32 FMA on CUDA cores, FP32 accumulation (both forms)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    X, dims, U, desc = workload(args.workload)
    C = U[0].shape[1]
    import oracle
    Ud = [u.astype(np.float64) for u in U]
    N = len(dims)
    n_s = min(X.size, 1 << 22)
    Xs = X[:n_s].astype(np.float64)
    for _ in range(args.warmup):
        oracle.mttkrp_range(Xs, 0, n_s, dims, Ud, 0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for n in range(N):
            oracle.mttkrp_range(Xs, 0, n_s, dims, Ud, n)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = N * 2.0 * n_s * C / t / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "sample_entries": n_s},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"first {n_s} entries, all {N} modes per step"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_krp(args, mtk, torch, dev, hbm_peak):
    """The Khatri-Rao product of Z = 2, 3, 4 equal operands with about 2e7 output rows, at
    C = 25 and 50, with the reuse of Algorithm 1 and without it (every row from scratch).
    Both are bound by the HBM write of K: roofline time = (K bytes + operand bytes) over the
    measured copy bandwidth.  Sampled rows are checked against the oracle's KRP of the
    same operand rows (exact FP64 products, compared with the FP32 result)."""
    import oracle
    out = []
    for Z in (2, 3, 4):
        for C in (25, 50):
            U = synth.krp_case(Z, C)
            Ud = [torch.from_numpy(u).to(dev) for u in U]
            J = 1
            for u in U:
                J *= u.shape[0]
            K = torch.empty((J, C), dtype=torch.float32, device=dev)
            nbytes = 4.0 * J * C + sum(4.0 * u.size for u in U)
            row = {"Z": Z, "C": C, "rows": J, "bytes": nbytes}
            g = np.random.default_rng(Z * 100 + C)
            for reuse in (True, False):
                fn = lambda: mtk.khatri_rao(Ud, reuse=reuse, out=K)
                t = time_calls(fn, max(args.steps, 3), warm=max(args.warmup, 1))
                fn()
                js = np.unique(np.concatenate([[0, J - 1], g.integers(0, J, 6)]))
                got = K[torch.as_tensor(js, device=dev)].double().cpu().numpy()
                err = 0.0
                for q, j in enumerate(js):
                    rem, sel = int(j), []
                    for u in reversed(U):                    # the last operand's index is fastest
                        sel.append(u[rem % u.shape[0]: rem % u.shape[0] + 1])
                        rem //= u.shape[0]
                    ref = oracle.krp(sel[::-1])[0]
                    err = max(err, float(np.max(np.abs(got[q] - ref) / np.maximum(np.abs(ref), 1e-30))))
                key = "reuse" if reuse else "naive"
                row[key] = {"us": t * 1e6, "gbs": nbytes / t / 1e9, "roofline_frac": nbytes / t / 1e9 / hbm_peak,
                            "max_rel_err_sampled_rows": err}
            row["reuse_speedup"] = row["naive"]["us"] / row["reuse"]["us"]
            out.append(row)
            del Ud, K
            torch.cuda.empty_cache()
    print(json.dumps({"workload": "krp: Z equal operands of uniform[0,1) FP32 entries, prod of rows ~2e7, "
                      "C in {25, 50}; reuse (Algorithm 1) vs every row from scratch", "hbm_peak_gbs": hbm_peak,
                      "cases": out}), flush=True)
    return 0


def run_paper_synth(args, mtk, torch, dev, hbm_peak):
    """Every mode's MTTKRP of the paper's equal-dimension tensors (900^3, 165^4, 60^5, 30^6,
    C = 25): the fused contraction on the BF16 planes where the planes kernel takes the
    mode, else the FP32-input path at bf16x2 (tensor cores, or CUDA cores for shapes the
    tensor-core kernel does not take).  Each result is checked against the FP64 oracle on
    sampled rows; times are CUDA events over back-to-back calls (inputs > L2)."""
    import oracle
    from paper_1708_08976_gb300 import _lib as L
    out = []
    for N in (3, 4, 5, 6):
        X, dims, U = synth.paper_equal(N)
        C = U[0].shape[1]
        I = X.size
        U64 = [u.astype(np.float64) for u in U]
        Xd = torch.from_numpy(X).to(dev)
        Ud = [torch.from_numpy(u).to(dev) for u in U]
        Xs, _ = mtk.split_tensor(Xd, dims)
        M = torch.empty((dims[0], C), dtype=torch.float32, device=dev)
        g = np.random.default_rng(1000 + N)
        modes = []
        for n in range(N):
            path = "planes"
            fn = lambda: mtk.mttkrp(None, dims, Ud, n, Xs=Xs, out=M)
            try:
                fn()
            except mtk.MtkError as e:
                if e.status != L.MTK_EUNSUPPORTED:
                    raise
                path = "bf16x2 on the FP32 tensor"
                fn = lambda: mtk.mttkrp(Xd, dims, Ud, n, precision="bf16x2", out=M)
            t = time_calls(fn, max(args.steps, 3), warm=max(args.warmup, 1))
            fn()
            rows = np.unique(np.concatenate([[0, dims[n] - 1], g.integers(0, dims[n], 2)]))
            ref = oracle.mttkrp_rows_f32(X, dims, U64, n, rows)
            got = M[torch.as_tensor(rows, device=dev)].double().cpu().numpy()
            err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            b = 4.0 * I + 4.0 * C * (sum(dims) - dims[n]) + 4.0 * dims[n] * C
            modes.append({"n": n, "path": path, "us": t * 1e6, "tflops": 2.0 * I * C / t / 1e12,
                          "roofline_frac": (b / hbm_peak / 1e9) / t, "rel_err_sampled_rows": err})
        out.append({"dims": list(dims), "entries": I, "rank": C, "modes": modes})
        del Xd, Xs, Ud, M
        torch.cuda.empty_cache()
    print(json.dumps({"workload": "paper-synth: equal-dimension tensors of the paper's synthetic sweep, "
                      "entries uniform[-1,1), factors N(0,1)/sqrt(25)", "hbm_peak_gbs": hbm_peak,
                      "tensors": out}), flush=True)
    return 0


def run_sym(args, mtk, torch, dev, hbm_peak):
    """corr4 (200x200x300x40, exactly symmetric in modes 0/1) stored packed: the 20,100
    entries a >= b of each 200 x 200 slice (20,104 rows with padding), about half the
    bytes.  Every mode's MTTKRP of the full tensor is computed from the BF16 planes of the
    packed tensor (mtk_mttkrp_sym_split) and checked on sampled rows against the FP64
    oracle on the full tensor; the same MTTKRPs on the full tensor's planes are timed
    beside it.  Roofline: the packed planes (4 B per packed entry) + factors + output over
    the measured copy bandwidth.  Then the paper's 3-D variant: the 19,900 entries a > b
    as one mode of a 3-way tensor (19,904 x 300 x 40 with padding), one CP-ALS sweep on
    its planes (C = 25)."""
    import oracle
    from paper_1708_08976_gb300 import _lib as L
    lib = L.load()
    X, dims, U = synth.corr4()
    N, C, I = len(dims), U[0].shape[1], X.size
    U64 = [u.astype(np.float64) for u in U]
    Xd = torch.from_numpy(X).to(dev)
    Ud = [torch.from_numpy(u).to(dev) for u in U]
    Xs, _ = mtk.split_tensor(Xd, dims)
    Xp = mtk.pack_symmetric(Xd, dims)
    Pp = lib.mtk_sym_packed_rows(dims[0], 1)
    rest = I // (dims[0] * dims[1])
    Xps, _ = mtk.split_tensor(Xp, mtk.sym_packed_dims(dims))
    del Xp
    torch.cuda.synchronize()
    pack_us = time_calls(lambda: mtk.pack_symmetric(Xd, dims), 3) * 1e6
    M = torch.empty((max(dims), C), dtype=torch.float32, device=dev)
    g = np.random.default_rng(77)
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    modes = []
    l0 = lib.mtk_launch_count()
    reps = max(args.steps, 5)
    for n in range(N):
        out = M[: dims[n]]
        fn_sym = lambda: mtk.mttkrp_sym(Xps, dims, Ud, n, out=out)
        fn_full = lambda: mtk.mttkrp(None, dims, Ud, n, Xs=Xs, out=out)
        t_full = time_calls(fn_full, reps, warm=max(args.warmup, 1))
        t_sym = time_calls(fn_sym, reps, warm=max(args.warmup, 1))
        fn_sym()
        rows = np.unique(np.concatenate([[0, dims[n] - 1], g.integers(0, dims[n], 6)]))
        ref = oracle.mttkrp_rows_f32(X, dims, U64, n, rows)
        got = out[torch.as_tensor(rows, device=dev)].double().cpu().numpy()
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        b = 4.0 * Pp * rest + 4.0 * C * (sum(dims) - dims[n]) + 4.0 * dims[n] * C
        modes.append({"n": n, "us_packed": t_sym * 1e6, "us_full_planes": t_full * 1e6,
                      "speedup_vs_full": t_full / t_sym, "bytes_packed": b,
                      "roofline_frac": (b / hbm_peak / 1e9) / t_sym, "rel_err_sampled_rows": err})
    launches = lib.mtk_launch_count() - l0
    # the paper's 3-D variant: CP-ALS on the packed 3-way tensor without the diagonal
    Xp3 = mtk.pack_symmetric(Xd, dims, diag=False)
    del Xd, Xs, Xps
    torch.cuda.empty_cache()
    d3 = (lib.mtk_sym_packed_rows(dims[0], 0), dims[2], dims[3])
    U3 = [torch.from_numpy(u).to(dev) for u in synth.uniform_factors(d3, C, 5, np.float32)]
    als = mtk.ALS(Xp3, d3, U3, presplit=True)
    for _ in range(max(args.warmup, 3)):
        als.sweep()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        als.sweep()
    e1.record()
    torch.cuda.synchronize()
    sweep3_ms = e0.elapsed_time(e1) / args.steps
    clocks = sampler.stop()
    t_step = sum(m["us_packed"] for m in modes) * 1e-6
    bsum = sum(m["bytes_packed"] for m in modes)
    achieved = bsum / t_step / 1e9
    print(json.dumps({
        "metric": "Dense MTTKRP of a tensor symmetric in modes 0/1 from packed storage, every mode",
        "value": N * 2.0 * I * C / t_step / 1e12, "unit": "TFLOP/s (full-tensor MTTKRP flops 2 I C per mode)",
        "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "dtype": "bf16x2 split products (packed tensor pre-split into BF16 hi/lo planes), f32 accumulate",
        "data": "synthetic",
        "config": {"workload": "corr4-sym: corr4 (200x200x300x40, exactly symmetric in modes 0/1) packed as "
                               f"{Pp} x 300 x 40 (a >= b), rank C=25", "dims": list(dims), "packed_rows": Pp,
                   "step": "the 4 MTTKRPs of the full tensor from the packed planes", "pack_us": pack_us,
                   "l2": "packed planes (0.96 GB) larger than L2; no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": None,
                     "kernel": "mtk_mttkrp_sym_split per mode (pair products or triangle walk + planes contraction)"},
        "modes": modes,
        "paper_3d_variant": {"dims": list(d3), "packed_rows_without_diagonal": dims[0] * (dims[0] - 1) // 2,
                             "sweep_ms": sweep3_ms, "fit": float(als.fit.item()),
                             "tflops": 3 * 2.0 * d3[0] * d3[1] * d3[2] * C / (sweep3_ms * 1e-3) / 1e12},
        "clocks": clocks, "gpu_launches": int(launches)}), flush=True)
    return 0


ARGS = None


def run_forms(args, mtk, torch, dev, hbm_peak):
    """cube512 (512^3 FP32 N(0,1), C = 32): every mode's MTTKRP in every algorithm
    (fused, materialised KRP, two-step) and precision form (FP32, bf16x2, bf16x3 on the
    FP32 tensor; the planes), timed with CUDA events over back-to-back calls (the tensor,
    512 MiB, is larger than L2) against the HBM roofline, each checked on sampled rows
    against the FP64 oracle.  The N(0,1) entries cancel heavily in every sum, so the
    relative error of the split forms is larger here than on the correlation workload."""
    import oracle
    X, dims, U = synth.cube512()
    N, C, I = 3, U[0].shape[1], X.size
    U64 = [u.astype(np.float64) for u in U]
    Xd = torch.from_numpy(X).to(dev)
    Ud = [torch.from_numpy(u).to(dev) for u in U]
    Xs, _ = mtk.split_tensor(Xd, dims)
    M = torch.empty((max(dims), C), dtype=torch.float32, device=dev)
    g = np.random.default_rng(512)
    rows = [np.unique(np.concatenate([[0, dims[n] - 1], g.integers(0, dims[n], 6)])) for n in range(N)]
    refs = [oracle.mttkrp_rows_f32(X, dims, U64, n, rows[n]) for n in range(N)]
    ffma = ffma_peak(mtk, torch)
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    out = []
    forms = [(a, p) for a in ("fused", "materialized", "two_step") for p in ("fp32", "bf16x2", "bf16x3")]
    forms.append(("fused", "planes"))
    for algo, prec in forms:
        modes = []
        for n in range(N):
            o = M[: dims[n]]
            if prec == "planes":
                fn = lambda: mtk.mttkrp(None, dims, Ud, n, Xs=Xs, out=o)
            else:
                fn = lambda: mtk.mttkrp(Xd, dims, Ud, n, algo=algo, precision=prec, out=o)
            t = time_calls(fn, max(args.steps, 3), warm=max(args.warmup, 1))
            fn()
            got = o[torch.as_tensor(rows[n], device=dev)].double().cpu().numpy()
            err = float(np.linalg.norm(got - refs[n]) / np.linalg.norm(refs[n]))
            b = 4.0 * I + 4.0 * C * (sum(dims) - dims[n]) + 4.0 * dims[n] * C
            row = {"n": n, "us": t * 1e6, "tflops": 2.0 * I * C / t / 1e12, "roofline_frac": (b / hbm_peak / 1e9) / t,
                   "rel_err_sampled_rows": err, "within_1e-5": err <= 1e-5}
            if prec == "fp32":
                row["ffma_frac"] = 2.0 * I * C / t / 1e12 / ffma
            modes.append(row)
        out.append({"algo": algo, "precision": prec, "modes": modes})
    clocks = sampler.stop()
    print(json.dumps({"workload": "cube512-forms: 512^3 FP32 N(0,1), rank C=32, factors N(0,1)/sqrt(32); "
                      "every algorithm x precision form, per mode", "hbm_peak_gbs": hbm_peak, "ffma_peak_tflops": ffma,
                      "forms": out, "clocks": clocks}), flush=True)
    return 0


def run_grad(args, mtk, torch, dev, hbm_peak):
    """The CP loss and its gradient on 32^5 (rank-16 CP plus noise, C = 16): forward (the
    mode-4 MTTKRP, the Grams, the loss) and hand-written backward (every mode's MTTKRP and
    U_n H_n - M_n) through torch.autograd, timed with CUDA events over back-to-back steps.
    Forms: on the planes with every mode's MTTKRP from the dimension tree, in the forward
    (two passes over the tensor), also replayed from a CUDA graph; on the planes one MTTKRP
    per mode; and on the FP32 tensor (FP32 and bf16x2).  ||X||^2 is computed once, with the
    planes, and passed to the loss.  The flops counted are the definition's, (N + 1) x 2 I C
    per step; roofline_frac_definition is the HBM time of (N + 1) passes over the 4-byte
    tensor (the definition) over the step time, roofline_frac_read that of the passes the
    form makes (2 for the tree, N per mode).  Each form's gradient is checked against the
    FP64 oracle's at mode 0."""
    import oracle
    X, dims, U = synth.cube32x5()
    N, C, I = len(dims), U[0].shape[1], X.size
    Xd = torch.from_numpy(X).to(dev)
    # the planes and ||X||^2, once per tensor (X is a constant of the loss)
    Xs, nx2 = mtk.split_tensor(Xd, dims)
    ref0 = oracle.grad(X.astype(np.float64), dims, [u.astype(np.float64) for u in U], 0)
    forms = {"planes-tree": {"Xs": Xs, "normX2": nx2}, "planes-tree-graph": {"Xs": Xs, "normX2": nx2},
             "planes-per-mode": {"Xs": Xs, "algo": "fused", "normX2": nx2},
             "fp32": {"precision": "fp32", "normX2": nx2}, "bf16x2": {"precision": "bf16x2", "normX2": nx2}}
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    out = {}
    for name, opts in forms.items():
        Ud = [torch.from_numpy(u).to(dev).requires_grad_(True) for u in U]

        def step():
            for u in Ud:
                u.grad = None
            mtk.cp_loss(Xd, dims, Ud, **opts).backward()
        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        if name.endswith("graph"):
            # forward and backward recorded once (the gradients land in the .grad tensors
            # allocated during the capture); each step replays the graph
            g_ = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream(dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            for u in Ud:
                u.grad = None
            with torch.cuda.graph(g_, stream=side, capture_error_mode="thread_local"):
                mtk.cp_loss(Xd, dims, Ud, **opts).backward()
            torch.cuda.current_stream(dev).wait_stream(side)
            step = g_.replay
            for _ in range(3):
                step()
            torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(args.steps, 5)
        torch.cuda.nvtx.range_push("grad_" + name)
        e0.record()
        for _ in range(reps):
            step()
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        t = e0.elapsed_time(e1) * 1e-3 / reps
        step()
        err = float(np.linalg.norm(Ud[0].grad.double().cpu().numpy() - ref0) / np.linalg.norm(ref0))
        # passes over the tensor per step: the tree's two partial contractions, or one
        # MTTKRP per mode (the forward's last-mode MTTKRP serves the backward too)
        passes = 2 if name.startswith("planes-tree") else N
        out[name] = {"ms_per_step": t * 1e3, "tflops": (N + 1) * 2.0 * I * C / t / 1e12,
                     "tensor_passes": passes,
                     "roofline_frac_definition": ((N + 1) * 4.0 * I / hbm_peak / 1e9) / t,
                     "roofline_frac_read": (passes * 4.0 * I / hbm_peak / 1e9) / t,
                     "grad_rel_err_mode0": err}
    clocks = sampler.stop()
    print(json.dumps({"workload": "cube32x5-grad: 32^5 FP32 rank-16 CP plus N(0,0.01^2), C=16; CP loss forward + "
                      "hand-written backward (all-mode MTTKRP) per step", "hbm_peak_gbs": hbm_peak,
                      "forms": out, "clocks": clocks}), flush=True)
    return 0


def main():
    global ARGS
    args = parse()
    ARGS = args
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_1708_08976_gb300 as mtk
    lib = mtk.load()
    hbm_peak, bf16_peak, peak_kind = peaks()

    if args.workload == "paper-synth":
        return run_paper_synth(args, mtk, torch, dev, hbm_peak)
    if args.workload == "krp":
        return run_krp(args, mtk, torch, dev, hbm_peak)
    if args.workload == "corr4-sym":
        return run_sym(args, mtk, torch, dev, hbm_peak)
    if args.workload == "cube512-forms":
        return run_forms(args, mtk, torch, dev, hbm_peak)
    if args.workload == "cube32x5-grad":
        return run_grad(args, mtk, torch, dev, hbm_peak)
    X, dims, U, desc = workload(args.workload)
    N = len(dims)
    C = U[0].shape[1]
    I = X.size
    flops_step = N * 2.0 * I * C
    Xd = torch.from_numpy(X).to(dev)
    U0 = [torch.from_numpy(u).to(dev) for u in U]
    if args.kernel_only:
        prec = "planes" if args.precision == "best" else args.precision
        Xs = mtk.split_tensor(Xd, dims)[0] if prec == "planes" else None
        ts = []
        if Xs is not None and args.sweep == "tree":
            # the two partial contractions of the dimension tree (n = 1 right, n = 2 left)
            for n, right in tree_partials(N):
                fn = lambda: mtk.partial_mttkrp_split(Xs, dims, U0, n, right)
                if args.steps > 0:
                    ts.append((f"{n}{'R' if right else 'L'}", time_calls(fn, args.steps, warm=args.warmup) * 1e6))
                else:
                    for _ in range(args.warmup):
                        fn()
            torch.cuda.synchronize()
            print(json.dumps({"kernel_only": True, "workload": desc, "precision": prec, "tree_partials": True,
                              "us": [[n, round(t, 1)] for n, t in ts]}), flush=True)
            return 0
        modes = [int(v) for v in args.modes.split(",")] if args.modes else range(N)
        for n in modes:
            if Xs is not None:
                fn = lambda: mtk.mttkrp(Xd, dims, U0, n, Xs=Xs)
            else:
                fn = lambda: mtk.mttkrp(Xd, dims, U0, n, precision=prec, algo=args.algo)
            if args.steps > 0:
                ts.append((n, time_calls(fn, args.steps, warm=args.warmup) * 1e6))
            else:
                for _ in range(args.warmup):
                    fn()
        torch.cuda.synchronize()
        print(json.dumps({"kernel_only": True, "workload": desc, "precision": prec,
                          "us": [[n, round(t, 1)] for n, t in ts]}), flush=True)
        return 0

    # accuracy of each precision form on every mode (vs the FP64 oracle on sampled rows)
    import oracle
    Ud64 = [u.astype(np.float64) for u in U]
    g = np.random.default_rng(123)
    forms = {}
    ffma = ffma_peak(mtk, torch)
    # the tensor split once into its BF16 planes (with ||X||^2 from the same pass)
    Xs, _ = mtk.split_tensor(Xd, dims)
    torch.cuda.synchronize()
    split_us = time_calls(lambda: mtk.split_tensor(Xd, dims, out=Xs), 3) * 1e6

    def call(prec, n, out=None):
        if prec == "planes":
            return mtk.mttkrp(Xd, dims, U0, n, Xs=Xs, out=out)
        return mtk.mttkrp(Xd, dims, U0, n, precision=prec, out=out)

    for prec in ("fp32", "bf16x2", "bf16x3", "planes"):
        try:
            errs, times = [], []
            for n in range(N):
                M = call(prec, n)
                rows = np.unique(np.concatenate([[0, dims[n] - 1], g.integers(0, dims[n], 6)]))
                ref = oracle.mttkrp_rows_f32(X, dims, Ud64, n, rows)
                got = M[torch.as_tensor(rows, device=dev)].double().cpu().numpy()
                errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
                times.append(time_calls(lambda: call(prec, n, out=M), 5))
            forms[prec] = {"rel_err_per_mode": errs, "mttkrp_us_per_mode": [t * 1e6 for t in times],
                           "tflops_per_mode": [2.0 * I * C / t / 1e12 for t in times]}
            if prec == "fp32":
                # the plain-FP32 form runs on the CUDA cores (one FFMA per multiply-add): its
                # ceiling is the measured FMA throughput, or the HBM read of the tensor
                forms[prec]["ffma_peak_tflops"] = ffma
                forms[prec]["ffma_frac_per_mode"] = [2.0 * I * C / t / 1e12 / ffma for t in times]
                forms[prec]["hbm_frac_per_mode"] = [
                    (4.0 * I + 4.0 * C * (sum(dims) - dims[n]) + 4.0 * dims[n] * C) / t / 1e9 / hbm_peak
                    for n, t in enumerate(times)]
        except mtk.MtkError as e:
            forms[prec] = {"unavailable": str(e)}
    if args.precision == "best":
        ok = {p: v for p, v in forms.items() if "unavailable" not in v and max(v["rel_err_per_mode"]) <= 1e-5}
        prec = min(ok, key=lambda p: sum(ok[p]["mttkrp_us_per_mode"])) if ok else "fp32"
    else:
        prec = args.precision

    planes = prec == "planes"
    stream = torch.cuda.current_stream(dev)
    # the sweep forms to time: per-mode MTTKRPs, and on the planes the dimension tree
    # (the partial contraction over modes >= 2 shared by the updates of U_0 and U_1, the
    # one over modes 0, 1 by those of U_2 and U_3: the tensor is read twice per sweep)
    # "tree-graph": the same tree sweep recorded once in a CUDA graph and replayed
    forms_sweep = ["per-mode"]
    if planes and len(dims) in (3, 4) and args.sweep in ("best", "tree"):
        forms_sweep = ["tree", "tree-graph"] if args.sweep == "tree" else ["per-mode", "tree", "tree-graph"]
    sweeps = {}
    graph_launches = 0
    for fs in forms_sweep:
        Uw = [u.clone() for u in U0]
        algo = "two_step" if fs.startswith("tree") else args.algo
        a_ = mtk.ALS(Xd, dims, Uw, algo=algo, precision="auto" if planes else prec, presplit=planes)
        for _ in range(args.warmup):
            a_.sweep()
        torch.cuda.synchronize()
        if a_.status() != 0:
            raise RuntimeError(f"device status {a_.status()} after warm-up ({fs})")
        if fs.endswith("graph"):
            l0 = lib.mtk_launch_count()
            a_.capture()
            graph_launches = lib.mtk_launch_count() - l0      # kernels in one replay
            for _ in range(args.warmup):
                a_.replay()
            torch.cuda.synchronize()
            if a_.status() != 0:
                raise RuntimeError(f"device status {a_.status()} after warm-up ({fs})")
        for a, b in zip(Uw, U0):
            a.copy_(b)
        sweeps[fs] = (a_, Uw)
    torch.cuda.synchronize()

    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    sweep_ms = {}
    launches_by = {}
    for fs, (a_, Uw) in sweeps.items():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = lib.mtk_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_sweeps" if fs == forms_sweep[-1] else "timed_sweeps_" + fs)
        run = a_.replay if fs.endswith("graph") else a_.sweep
        e0.record(stream)
        for _ in range(args.steps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        launches_by[fs] = lib.mtk_launch_count() - l0 + (graph_launches * args.steps if fs.endswith("graph") else 0)
        if world > 1:
            torch.distributed.barrier()
        sweep_ms[fs] = e0.elapsed_time(e1) / args.steps
    best_form = min(sweep_ms, key=sweep_ms.get)
    als = sweeps[best_form][0]
    launches = launches_by[best_form]
    t_step = sweep_ms[best_form] * 1e-3

    # per-launch duration of the dominant kernel (the MTTKRP contraction of every mode,
    # timed on its launch stream; inputs 1.92 GB > L2)
    per_mode = []
    M = torch.empty((max(dims), C), dtype=torch.float32, device=dev)
    for n in range(N):
        out = M[: dims[n]]
        if planes:
            fn = lambda: mtk.mttkrp(Xd, dims, U0, n, Xs=als.Xs, out=out)
        else:
            fn = lambda: mtk.mttkrp(Xd, dims, U0, n, precision=prec, algo=args.algo, out=out)
        per_mode.append(time_calls(fn, max(args.steps, 5), stream=stream))
    # with the dimension tree the step's dominant kernel is the partial contraction on
    # the planes (each call: prep, contraction, slab reduce), timed the same way
    partials = []
    if best_form.startswith("tree"):
        for n, right in tree_partials(N):
            fn = lambda: mtk.partial_mttkrp_split(als.Xs, dims, U0, n, right)
            partials.append((n, right, time_calls(fn, max(args.steps, 5), stream=stream)))
    clocks = sampler.stop()

    t_max = max_over_ranks(t_step, world, dev)
    value = job_value(flops_step, world, t_max)

    # e2e: host buffers, H2D of the tensor + factors and D2H of factors + fit inside the region
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(X).pin_memory()
        Uh = [torch.from_numpy(u).pin_memory() for u in U]
        Uo = [torch.empty_like(u).pin_memory() for u in Uh]
        fit_h = torch.empty((), dtype=torch.float64).pin_memory()
        Ue = [torch.empty_like(u) for u in U0]
        # planes: the split reads the pinned host tensor in place (the host-to-device
        # transfer of X and its split are one pass; X never occupies device memory);
        # otherwise X is copied to the device and its norm taken there
        Xe = Xh if planes else torch.empty_like(Xd)
        alse = mtk.ALS(Xe, dims, Ue, algo="two_step" if best_form.startswith("tree") else args.algo,
                       precision="auto" if planes else prec, presplit=planes)
        ksteps = max(3, min(args.steps, 5))
        for it in range(ksteps + 1):
            if it == 1:
                torch.cuda.synchronize()
                a = time.perf_counter()
            if not planes:
                Xe.copy_(Xh, non_blocking=True)
            for d_, h_ in zip(Ue, Uh):
                d_.copy_(h_, non_blocking=True)
            if planes:
                alse.resplit(Xh)    # this step's tensor: BF16 planes and ||X||^2 from host memory
            else:
                alse.resplit()      # ||X||^2 of this step's tensor
            alse.sweep()
            for h_, d_ in zip(Uo, Ue):
                h_.copy_(d_, non_blocking=True)
            fit_h.copy_(alse.fit, non_blocking=True)
            torch.cuda.synchronize()
        te = (time.perf_counter() - a) / ksteps
        h2d = X.nbytes + sum(u.nbytes for u in U)
        d2h = sum(u.nbytes for u in U) + 8
        e2e = {"value": world * flops_step / te / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": te * 1e3,
               "tensor_transfer": ("read in place from pinned host memory by the split kernel "
                                   "(mtk_split_tensor on the host pointer)") if planes else
                                  "cudaMemcpyAsync from pinned host memory"}

    batch = None
    if not args.no_batch:
        batch = batch_measure(mtk, torch, dev, hbm_peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(X, dims, U, C)

    bytes_mode = [4.0 * I + 4.0 * C * (sum(dims) - dims[n]) + 4.0 * dims[n] * C for n in range(N)]
    tree_rows = []
    if partials:
        pbytes = [partial_bytes(dims, C, n, r) for n, r, _ in partials]
        achieved = sum(pbytes) / sum(t for _, _, t in partials) / 1e9
        kernel = ("planes partial contraction of the dimension tree (mtk_partial_mttkrp_split at "
                  + ", ".join(f"n={n} {'right' if r else 'left'}" for n, r, _ in partials)
                  + "; each call = prep + contraction + slab reduce)")
        traffic = NCU_TRAFFIC_PER_LAUNCH.get("tree")
        tree_rows = [{"n": n, "side": "right" if r else "left", "us": t * 1e6, "bytes": b,
                      "frac": (b / hbm_peak / 1e9) / t} for (n, r, t), b in zip(partials, pbytes)]
    else:
        achieved = sum(bytes_mode) / sum(per_mode) / 1e9
        kernel = "MTTKRP contraction (mtk_mttkrp per mode, incl. split reduce)"
        traffic = NCU_TRAFFIC_PER_LAUNCH.get(prec)
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "planes": "bf16x2 split products (tensor pre-split into BF16 hi/lo planes), f32 accumulate"}.get(
            prec, f"{prec} split products, f32 accumulate"),
        "data": "synthetic",
        "config": {"workload": desc, "dims": list(dims), "rank": C,
                   "step": "one CP-ALS sweep (4 MTTKRPs + FP64 solves + Grams + fit)",
                   "sweep_form": best_form, "sweep_ms_by_form": sweep_ms,
                   "flops_counted": "4 x 2 I C per sweep (the definition of the 4 MTTKRPs); the dimension tree "
                                    "computes them with 2 passes over the tensor",
                   "precision": prec, "algo": args.algo, "l2": "inputs (1.92 GB) larger than L2; no flush",
                   "tensor_split_us": split_us,
                   "tensor_split": ("the BF16 planes and ||X||^2 are made once per CP-ALS run, outside the timed sweeps "
                                    "(inside every e2e step)") if planes else "not used",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "traffic_unit": "DRAM bytes per launch of the contraction (ncu, scaled from the 200x200x30x40 "
                                     "capture by the tensor entries)",
                     "kernel": kernel, "peak_kind": peak_kind},
        "tree_partials": tree_rows,
        "mttkrp_us_per_mode": [t * 1e6 for t in per_mode],
        "roofline_frac_per_mode": [(b / hbm_peak / 1e9) / t for b, t in zip(bytes_mode, per_mode)],
        "precision_forms": forms,
        "fit_after_timed_sweeps": float(als.fit.item()),
        "clocks": clocks,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "batch64": batch,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
