"""Conditioning step, FP64 oracle side (Figure 1 / Figure 2, steps 2-3).

Test infrastructure: only the tests, the smoke check and the bench's CPU
baseline use this module; the CUDA path shares no code with it.

Π1·X = Q·R with R upper triangular; the oracle takes LAPACK's Householder QR
(numpy) and flips signs so that diag(R) > 0, which makes R unique for a full
column rank Π1·X.  R⁻¹ comes from a triangular solve, and the product that
phase 2 needs is formed in the order the paper's running-time argument uses
(proof of the fast ℓ1 regression theorem, Appendix): first M = R⁻¹·Π2
(q × r2), never U = X·R⁻¹.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

RANK_TOL = 1e-5


class RankDeficient(ValueError):
    pass


def qr_positive(pix: np.ndarray):
    """(Q, R) with Π1X = Q·R, QᵀQ = I, R upper triangular with positive diagonal."""
    q_mat, r_mat = np.linalg.qr(np.asarray(pix, dtype=np.float64), mode="reduced")
    sgn = np.sign(np.diag(r_mat))
    sgn[sgn == 0] = 1.0
    return q_mat * sgn[None, :], r_mat * sgn[:, None]


def check_rank(r_mat: np.ndarray, tol: float = RANK_TOL) -> None:
    """Full column rank (§2 assumes it) to the precision Π1·X is formed in: column k of
    Π1X = QR has norm ‖R_{:k,k}‖₂, and it is dependent on the columns before it when
    |R_kk| ≤ tol·‖R_{:k,k}‖₂ (1e-5: Π1·X is accumulated in FP32 on the GPU)."""
    dg = np.abs(np.diag(r_mat))
    coln = np.linalg.norm(np.triu(r_mat), axis=0)
    if dg.size == 0 or not np.all(np.isfinite(r_mat)) or np.any(dg <= tol * coln):
        raise RankDeficient("Π1·X is numerically rank deficient")


def r_inverse(r_mat: np.ndarray) -> np.ndarray:
    return solve_triangular(r_mat, np.eye(r_mat.shape[0]), lower=False)


def m_matrix(r_mat: np.ndarray, pi2: np.ndarray) -> np.ndarray:
    """M = R⁻¹·Π2 by back substitution (q × r2)."""
    return solve_triangular(r_mat, pi2, lower=False)
