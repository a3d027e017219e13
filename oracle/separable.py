"""The separable canonical-row design of the large-scale experiment (§6.3), FP64 oracle side.

Test infrastructure: only the tests, the smoke check and the bench's CPU baseline use
this module; the CUDA path shares no code with it.

Every row of A is a canonical vector e_{c_i}, so ‖A·x − b‖₁ = Σ_j Σ_{i: c_i = j} |x_j − b_i|
splits into one scalar problem per coordinate, and the minimisers of Σ_i |x_j − b_i| over
a group of m values are exactly the points between the group's lower median (order
statistic ⌈m/2⌉ counting from 1) and its upper median (order statistic ⌊m/2⌋ + 1): the
optimum of the whole problem is that box, a single point where every group is odd.
"""
from __future__ import annotations

import numpy as np


def canonical_optimum(cols: np.ndarray, b: np.ndarray, d: int):
    """(lo, hi): the box [lo_j, hi_j] of minimisers of ‖A·x − b‖₁ for A with rows
    e_{cols_i} (FP64, per-coordinate lower and upper medians of b; NaN for an empty group)."""
    cols = np.asarray(cols, dtype=np.int64)
    b = np.asarray(b, dtype=np.float64)
    lo = np.full(d, np.nan)
    hi = np.full(d, np.nan)
    for j in range(d):
        v = np.sort(b[cols == j])
        m = v.size
        if m == 0:
            continue
        lo[j] = v[(m + 1) // 2 - 1]
        hi[j] = v[m // 2]
    return lo, hi


def box_distance(x: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Per-coordinate distance of x from the optimal box [lo, hi] (0 inside it)."""
    x = np.asarray(x, dtype=np.float64)
    return np.maximum(0.0, np.maximum(lo - x, x - hi))


def relative_errors(x: np.ndarray, lo: np.ndarray, hi: np.ndarray, x_ref: np.ndarray) -> dict:
    """‖e‖_p / ‖x_ref‖_p for p = 1, 2, ∞ (the three columns of the §6.3 error table), e the
    per-coordinate distance of x from the optimal box and x_ref the reference optimum."""
    e = box_distance(x, lo, hi)
    x_ref = np.asarray(x_ref, dtype=np.float64)
    return {
        "l1": float(np.sum(e) / np.sum(np.abs(x_ref))),
        "l2": float(np.sqrt(np.sum(e * e)) / np.sqrt(np.sum(x_ref * x_ref))),
        "linf": float(np.max(e) / np.max(np.abs(x_ref))),
    }
