"""Conditioning quality of an ℓ1 basis, FP64 oracle side (§6.1).

Test infrastructure: only the tests and the bench's validation leg use this module;
the CUDA path shares no code with it.

U ∈ R^{n×d} is (α, β)-conditioned when ‖U‖₁ ≤ α (the entrywise ℓ1 norm) and
‖z‖_∞ ≤ β·‖U·z‖₁ for every z (the definition of (α, β, p)-conditioning the paper
takes from Dasgupta et al., with p = 1 and its dual q = ∞); κ̄₁(U) is the smallest
α·β: α = ‖U‖₁ and β = 1 / min_{‖z‖_∞ = 1} ‖U·z‖₁, which §6.1 computes with d linear
programs.  Here the d programs are ℓ1 regressions: a minimiser z of ‖U·z‖₁ on
‖z‖_∞ = 1 has |z_j| = 1 at its largest coordinate, so
    min_{‖z‖_∞=1} ‖U·z‖₁ = min_j min_y ‖U_{:,j} + U_{:,−j}·y‖₁
(if the unconstrained minimiser for the best j had a coordinate above 1 in magnitude,
dividing by it would give a feasible z with a smaller value).  Each is solved exactly as
an LP (oracle.solve.lad_lp).
"""
from __future__ import annotations

import numpy as np

from . import solve


def min_l1_on_unit_box(U: np.ndarray) -> float:
    """min_{‖z‖_∞ = 1} ‖U·z‖₁ as the smallest of d unconstrained ℓ1 regressions."""
    U = np.asarray(U, dtype=np.float64)
    n, d = U.shape
    best = np.inf
    for j in range(d):
        if d == 1:
            v = float(np.abs(U[:, 0]).sum())
        else:
            rest = np.delete(U, j, axis=1)
            _, v = solve.lad_lp(rest, -U[:, j])
        best = min(best, v)
    return best


def kappa_bar_1(U: np.ndarray) -> float:
    """κ̄₁(U) = ‖U‖₁ / min_{‖z‖_∞ = 1} ‖U·z‖₁ (§6.1)."""
    U = np.asarray(U, dtype=np.float64)
    return float(np.abs(U).sum()) / min_l1_on_unit_box(U)
