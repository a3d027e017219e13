"""Weighted ℓ1 regression on the coreset, FP64 oracle side (Figure 2, step 8).

Test infrastructure: only the tests, the smoke check and the bench's CPU
baseline use this module; the CUDA path shares no code with it.

min_x Σ_i w_i·|A_i·x − b_i| is the linear program
    min  Σ w_i (t⁺_i + t⁻_i)   s.t.  A·x − t⁺ + t⁻ = b,  t⁺, t⁻ ≥ 0,
solved here with HiGHS' dual simplex (scipy).  The LP optimum is attained at
a vertex where d residuals vanish; the oracle re-solves that d×d system
exactly (`polish`) and keeps whichever point has the smaller objective.
`lad_bruteforce` enumerates every vertex (tiny instances only) and
`weighted_median` is the closed form for a single all-ones column.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog


def weighted_objective(A: np.ndarray, b: np.ndarray, w: np.ndarray | None, x: np.ndarray) -> float:
    """Σ w_i·|A_i·x − b_i| in FP64 with a correctly rounded final sum."""
    r = np.asarray(A, dtype=np.float64) @ np.asarray(x, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    t = np.abs(r) if w is None else np.asarray(w, dtype=np.float64) * np.abs(r)
    return math.fsum(t.tolist())


def objective(A, b, x) -> float:
    """‖A·x − b‖₁ in FP64 (the problem statement's objective)."""
    return weighted_objective(A, b, None, x)


def _polish(A, b, w, x):
    d = A.shape[1]
    r = np.abs(A @ x - b)
    basis = np.argsort(r, kind="stable")[:d]
    try:
        xp = np.linalg.solve(A[basis], b[basis])
    except np.linalg.LinAlgError:
        return x
    return xp if weighted_objective(A, b, w, xp) <= weighted_objective(A, b, w, x) else x


def lad_lp(A: np.ndarray, b: np.ndarray, w: np.ndarray | None = None):
    """Exact weighted LAD solution by linear programming; returns (x, objective)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, d = A.shape
    w = np.ones(m) if w is None else np.asarray(w, dtype=np.float64)
    cost = np.concatenate([np.zeros(d), w, w])
    a_eq = sp.hstack([sp.csr_matrix(A), -sp.identity(m, format="csr"),
                      sp.identity(m, format="csr")], format="csr")
    bounds = [(None, None)] * d + [(0, None)] * (2 * m)
    res = linprog(cost, A_eq=a_eq, b_eq=b, bounds=bounds, method="highs-ds",
                  options={"primal_feasibility_tolerance": 1e-10,
                           "dual_feasibility_tolerance": 1e-10})
    if res.status != 0:
        raise RuntimeError(f"LP failed: {res.message}")
    x = _polish(A, b, w, res.x[:d])
    return x, weighted_objective(A, b, w, x)


def lad_bruteforce(A: np.ndarray, b: np.ndarray, w: np.ndarray | None = None):
    """Minimum over all vertices (every nonsingular d-row subset solved exactly)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, d = A.shape
    best = (None, math.inf)
    for rows in itertools.combinations(range(m), d):
        sub = A[list(rows)]
        if abs(np.linalg.det(sub)) < 1e-12:
            continue
        x = np.linalg.solve(sub, b[list(rows)])
        f = weighted_objective(A, b, w, x)
        if f < best[1]:
            best = (x, f)
    return best


def weighted_median(values: np.ndarray, weights: np.ndarray) -> float:
    """A minimizer of Σ w_i |v_i − x|: the smallest v whose cumulative weight reaches half."""
    order = np.argsort(values, kind="stable")
    v = np.asarray(values, dtype=np.float64)[order]
    cw = np.cumsum(np.asarray(weights, dtype=np.float64)[order])
    return float(v[np.searchsorted(cw, 0.5 * cw[-1])])
