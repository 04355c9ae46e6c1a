"""Helpers for the GPU parity tests (comparison logic only; no method
arithmetic)."""
from __future__ import annotations

import numpy as np


def rel_rms(a: np.ndarray, ref: np.ndarray) -> float:
    den = float((ref ** 2).sum())
    num = float(((a - ref) ** 2).sum())
    if den == 0.0:
        return float(np.sqrt(num))
    return float(np.sqrt(num / den))


def min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def dense_cluster_state(seed: int = 3):
    """A dilute lattice gas (rho 0.1) holding a compressed blob (rho 2.2):
    cells with more than 32 particles and stencil windows larger than the
    force kernel's shared-memory staging capacity."""
    from paper_0709_3225_gb300 import inputs
    x, L = inputs.jittered_fcc(6, 0.1, 0.1, seed)
    blob, _ = inputs.fcc(6, 2.2)          # 864 sites, nearest distance ~0.86
    blob = blob + np.array([3.0, 4.0, 5.0])
    keep = np.ones(x.shape[0], bool)
    lo, hi = blob.min(0) - 1.0, blob.max(0) + 1.0
    inside = np.all((x > lo) & (x < hi), axis=1)
    keep &= ~inside
    xx = np.concatenate([x[keep], blob])
    return np.ascontiguousarray(xx), L
