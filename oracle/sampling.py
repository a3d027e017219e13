"""Coreset sampling, FP64 oracle side (Figure 2, steps 6-7; ℓ1 sampling lemma, §2).

Test infrastructure: only the tests, the smoke check and the bench's CPU
baseline use this module; the CUDA path shares no code with it.

p̂_i = min{1, m_s·λ_i / Σ_j λ_j}, evaluated in FP64 as τ = m_s / Σλ (one
division) followed by p̂_i = min(1, τ·λ_i); D_ii = 1/p̂_i with probability p̂_i,
else 0, decided by u_i < p̂_i with the 53-bit uniform of row i.  Kept indices
are returned in ascending order.  Σλ is the correctly rounded FP64 sum.
"""
from __future__ import annotations

import math

import numpy as np


def lambda_total(lam: np.ndarray) -> float:
    return math.fsum(np.asarray(lam, dtype=np.float64).tolist())


def probabilities(lam: np.ndarray, coreset: float, total: float | None = None):
    lam = np.asarray(lam, dtype=np.float64)
    if total is None:
        total = lambda_total(lam)
    if not (total > 0.0) or not math.isfinite(total):
        raise ValueError("Σλ must be positive and finite")
    tau = float(coreset) / total
    return np.minimum(1.0, tau * lam), tau, total


def probabilities_scaled(lam: np.ndarray, scale: float):
    """p̂_i = min{1, s·λ̂_i} with the sampling size s given (Figure "mainOpt", step 7):
    OptimizedFastCauchyRegression does not normalise by Σλ."""
    lam = np.asarray(lam, dtype=np.float64)
    return np.minimum(1.0, float(scale) * lam)


def bernoulli_sample(p: np.ndarray, u: np.ndarray):
    """Indices i with u_i < p_i (ascending) and their weights 1/p_i."""
    p = np.asarray(p, dtype=np.float64)
    keep = np.asarray(u, dtype=np.float64) < p
    idx = np.flatnonzero(keep)
    return idx, 1.0 / p[idx]


def sample_with_replacement(lam: np.ndarray, m: int, u: np.ndarray):
    """Exactly m rows drawn independently with replacement, p̂_i = λ_i/Σλ (the alternative
    to step 6-7 that the caption of Figure 2 allows).  Draw t takes the row i with
    C_{i−1} ≤ u_t·Σλ < C_i, C the running FP64 sum of λ (C_{−1} = 0, Σλ = C_{n−1}); its
    weight is 1/(m·p̂_i) = Σλ/(m·λ_i).  Returns (rows in draw order, weights, C)."""
    lam = np.asarray(lam, dtype=np.float64)
    cdf = np.cumsum(lam)
    total = float(cdf[-1])
    if not (total > 0.0) or not math.isfinite(total):
        raise ValueError("Σλ must be positive and finite")
    target = np.asarray(u, dtype=np.float64)[:m] * total
    idx = np.searchsorted(cdf, target, side="right")
    return idx, total / (m * lam[idx]), cdf
