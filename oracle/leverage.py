"""ℓ1 row-norm estimates, FP64 oracle side (Figure 2, steps 4-5).

Test infrastructure: only the tests, the smoke check and the bench's CPU
baseline use this module; the CUDA path shares no code with it.

Λ = X·M with M = R⁻¹·Π2, and λ_i = median_j |Λ_ij|.  For an even number r2 of
columns the median is read as the lower median, the ((r2−1)//2)-th order
statistic counting from 0 (for r2 = 16: the 8th smallest).  The lemma on
medians of half-Cauchys (proof of the fast ℓ1 regression theorem) holds for
either middle element.  `exact_row_l1` is the quantity λ estimates: the row ℓ1
norm of U = X·R⁻¹.
"""
from __future__ import annotations

import numpy as np


def lower_median_index(r2: int) -> int:
    return (r2 - 1) // 2


def lambda_estimates(X: np.ndarray, M: np.ndarray, chunk: int = 1 << 20) -> np.ndarray:
    X = np.asarray(X)
    M = np.asarray(M, dtype=np.float64)
    k = lower_median_index(M.shape[1])
    out = np.empty(X.shape[0])
    for a in range(0, X.shape[0], chunk):
        lam = np.abs(X[a:a + chunk].astype(np.float64) @ M)
        out[a:a + chunk] = np.sort(lam, axis=1)[:, k]
    return out


def bf16_round(values: np.ndarray) -> np.ndarray:
    """Round to FP32 (nearest even), then to bfloat16 (nearest even, 8 significant bits), in FP64.

    This is the mixed-precision form of M: the tensor-core product uses M's first d rows
    rounded this way, the b column's row stays FP32.
    """
    f = np.ascontiguousarray(np.asarray(values, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def mixed_precision_m(M: np.ndarray) -> np.ndarray:
    """M as the mixed-precision λ uses it: rows 0..d−1 in BF16, row d (the b column) in FP32."""
    M = np.asarray(M, dtype=np.float64)
    out = np.empty_like(M)
    out[:-1] = bf16_round(M[:-1])
    out[-1] = M[-1].astype(np.float32).astype(np.float64)
    return out


def lambda_term_scale(X: np.ndarray, M: np.ndarray, chunk: int = 1 << 20) -> np.ndarray:
    """Per row, max_j Σ_k |X_ik|·|M_kj|: the magnitude that bounds the rounding of Λ_i·."""
    X = np.asarray(X)
    am = np.abs(np.asarray(M, dtype=np.float64))
    out = np.empty(X.shape[0])
    for a in range(0, X.shape[0], chunk):
        out[a:a + chunk] = (np.abs(X[a:a + chunk].astype(np.float64)) @ am).max(axis=1)
    return out


def exact_row_l1(X: np.ndarray, r_inv: np.ndarray) -> np.ndarray:
    """‖U_(i)‖₁ with U = X·R⁻¹ formed explicitly (Definition of ℓ1 leverage scores, §4.1)."""
    return np.abs(np.asarray(X, dtype=np.float64) @ r_inv).sum(axis=1)
