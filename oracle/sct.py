"""The slow Cauchy transform Π1·X = (4/r1)·C·X, FP64 oracle side.

Test infrastructure: only the tests, the smoke check and the bench's CPU
baseline use this module; the CUDA path shares no code with it.

C is an r1 × n matrix of i.i.d. standard Cauchy variables; by the theorem of
Sohler and Woodruff that the paper restates in §3 (its proof is in the
appendix), ‖y‖₁ ≤ (4/r1)‖C·y‖₁ ≤ κ'‖y‖₁ for every y in a fixed d-dimensional
subspace with high probability, when r1 = O(d log d).  The paper's large-scale
experiment (§6.3) conditions with this transform ("CT") instead of FCT1.  The
oracle forms the product directly from its definition, a row block at a time,
with the draws of `oracle.rng.sct_matrix`, and returns the per-entry sum of
|terms| that the FP32 tolerance refers to.
"""
from __future__ import annotations

import numpy as np

from .rng import sct_matrix


def sct_embed(X: np.ndarray, r1: int, seed: int = 0, problem_id: int = 0, row_offset: int = 0,
              block: int = 1 << 14):
    """(Π1X, T) with Π1X = (4/r1)·C·X ∈ R^{r1×q} and T = (4/r1)·|C|·|X|, in FP64."""
    X = np.asarray(X, dtype=np.float64)
    n, q = X.shape
    pix = np.zeros((r1, q))
    tsum = np.zeros((r1, q))
    for a in range(0, n, block):
        rows = row_offset + np.arange(a, min(n, a + block), dtype=np.int64)
        C = sct_matrix(seed, problem_id, rows, r1)             # r1 × block
        xb = X[a:a + rows.size]
        pix += C @ xb
        tsum += np.abs(C) @ np.abs(xb)
    scale = 4.0 / r1
    return scale * pix, scale * tsum
