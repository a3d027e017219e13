"""The FCT2 embedding (§3.2, FCT2 construction), FP64 oracle side.

Test infrastructure: only the tests, the smoke check and the bench's CPU baseline
use this module; the CUDA path shares no code with it.

Π1 = (8/r1)·√(πt/(2s))·C·H̃ with H̃ block diagonal, n/t copies of one s × t fast
Johnson–Lindenstrauss matrix G on its diagonal, and C an r1 × (ns/t) matrix of i.i.d.
standard Cauchy variables.  The paper leaves G's construction open (its experiments use
a subsampled randomized Hadamard transform as their FJLT, §6.1); here G is that
transform, G = √(t/s)·S·H_t·D: D a random ±1 diagonal, H_t the normalized Sylvester
Hadamard matrix of order t (a power of two) and S the selection of s of its rows, drawn
uniformly with replacement, so every entry of G is ±1/√s.  One G serves every block (the
construction repeats the same block).  X is extended by zero rows to a multiple of t.
Row k of H̃X takes column k of C: its entries come from the slow transform's generator
(`oracle.rng.sct_matrix`, stream 4) at row id k, with the global id of the block's first
row of H̃X equal to (global row offset / t)·s.  The oracle forms G densely from its
definition and the products directly, and returns the per-entry sum of |terms| that the
FP32 tolerance refers to.
"""
from __future__ import annotations

import math

import numpy as np

from . import rng
from .fct import sylvester_hadamard


def fjlt_matrix(seed: int, problem_id: int, t: int, s: int) -> np.ndarray:
    """G = √(t/s)·S·H_t·D (s × t), H_t normalized by 1/√t."""
    D, sel = rng.fjlt_draws(seed, problem_id, t, s)
    H = sylvester_hadamard(t) / math.sqrt(t)
    return math.sqrt(t / s) * H[sel] * D[None, :]


def fct2_scale(t: int, s: int, r1: int) -> float:
    return 8.0 / r1 * math.sqrt(math.pi * t / (2.0 * s))


def fct2_embed(X: np.ndarray, t: int, s: int, r1: int, seed: int = 0, problem_id: int = 0,
               row_offset: int = 0):
    """(Π1X, T) with Π1X ∈ R^{r1×q} in FP64 and T = scale·|C|·(|G|·|X| per block)."""
    X = np.asarray(X, dtype=np.float64)
    n, q = X.shape
    nb = -(-n // t)
    Xp = np.zeros((nb * t, q))
    Xp[:n] = X
    G = fjlt_matrix(seed, problem_id, t, s)
    Xb = Xp.reshape(nb, t, q)
    Y = np.einsum("rt,btq->brq", G, Xb).reshape(nb * s, q)
    Yabs = np.einsum("rt,btq->brq", np.abs(G), np.abs(Xb)).reshape(nb * s, q)
    ids = (row_offset // t) * s + np.arange(nb * s, dtype=np.int64)
    C = rng.sct_matrix(seed, problem_id, ids, r1)
    scale = fct2_scale(t, s, r1)
    return scale * (C @ Y), scale * (np.abs(C) @ Yabs)
