"""Shared test utilities (no method arithmetic here)."""
import numpy as np


def rel_fro(got, ref) -> float:
    """||got - ref||_F / ||ref||_F (0 if both are zero)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    num = np.linalg.norm(got - ref)
    if den == 0.0:
        return float(num)
    return float(num / den)


def to_dev(a, torch, dtype=None):
    dtype = dtype or torch.float32
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dtype).cuda().contiguous()


def factors_dev(U, torch):
    return [to_dev(u, torch) for u in U]


def f32_round(U):
    """The FP32 rounding of FP64 inputs, back in FP64 (what the GPU sees)."""
    return [np.asarray(u, dtype=np.float32).astype(np.float64) for u in U]
