"""Shared test helpers: error metrics and GPU runs through the C-ABI."""
from __future__ import annotations

import numpy as np
import torch

FP32_TOL = 1e-5  # per-signal relative L2 against the FP64 oracle


def rel_l2_per_signal(got, ref) -> np.ndarray:
    """||got - ref|| / ||ref|| per row (absolute error where ||ref|| == 0)."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    num = np.linalg.norm(got - ref, axis=-1)
    den = np.linalg.norm(ref, axis=-1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def max_rel_l2(got, ref) -> float:
    e = rel_l2_per_signal(got, ref)
    return float(e.max()) if e.size else 0.0


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.complex128)
