"""FCT1 embedding Π1·X, FP64 oracle side (§3.1, FCT1 construction).

Test infrastructure: only the tests, the smoke check and the bench's CPU
baseline use this module; the CUDA path shares no code with it.

Π1 = 4·B·C·H̃, applied here after the random ±1 diagonal D (sign_flip=True),
so the oracle computes Π1·X = 4·B·C·H̃·D·X for X = [A, −b]:

* H̃ ∈ R^{2n×n} is block-diagonal with n/s blocks G_s = [H_s; I_s], H_s the
  normalized Sylvester Hadamard matrix (H_s/√s of the recursion in §3.1);
* C ∈ R^{2n×2n} is diagonal with independent standard Cauchy entries;
* B ∈ R^{r1×2n} has one uniformly chosen standard basis vector per column.

Virtual-row convention (the paper orders rows only through H̃): within block
β the 2s virtual rows are the s rows of H_s·z_β then the s rows of z_β; the
Hadamard virtual row (β, ι) and the identity virtual row (β, ι) both take
their draws from input row β·s + ι (see `oracle.rng.fct_draws`).

When n is not a multiple of s, X is extended by zero rows to the next
multiple of s and Π1 acts on the padded matrix; the padded rows add nothing
through the identity half, but their Hadamard virtual rows carry values and
use the draws of their (out-of-range) row ids.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .rng import fct_draws


def sylvester_hadamard(s: int) -> np.ndarray:
    """Unnormalized Hadamard H_s from H_1 = [1], H_{2m} = [[H_m, H_m], [H_m, −H_m]] (§3.1)."""
    if s < 1 or (s & (s - 1)) != 0:
        raise ValueError("s must be a power of two")
    h = np.ones((1, 1))
    while h.shape[0] < s:
        h = np.block([[h, h], [h, -h]])
    return h


def _draws(seed, problem_id, n_pad, r1, row_offset, draws):
    if draws is not None:
        return draws
    rows = row_offset + np.arange(n_pad, dtype=np.int64)
    return fct_draws(seed, problem_id, rows, r1)


def padded_rows(n: int, s: int) -> int:
    return -(-n // s) * s


def fct1_embed(X: np.ndarray, s: int, r1: int, seed: int = 0, problem_id: int = 0,
               row_offset: int = 0, sign_flip: bool = True, draws: dict | None = None):
    """Π1·X in FP64, block by block, and the per-entry sum of |terms|.

    Returns (PiX, T): PiX ∈ R^{r1×q}, and T, the sum of |contributing terms| of
    each entry: (Π1X)_rc = Σ_k (Π1)_rk·X_kc expands, through H̃, into the terms
    4·c_v·(H̃)_vk·σ_k·X_kc over the virtual rows v hashed to r and the rows k of
    v's block, so T_rc = Σ_{v→r} 4|c_v|·Σ_k |(H̃)_vk|·|X_kc|, i.e. 4|c_v|·|z_vc|
    for an identity row and 4|c_v|·Σ_{k∈block}|z_kc|/√s for a Hadamard row.
    This is the scale the FP32 tolerance refers to.
    `draws` may replace the generated draws (tests use this to set C ≡ 1).
    """
    X = np.asarray(X, dtype=np.float64)
    n, q = X.shape
    n_pad = padded_rows(n, s)
    nb = n_pad // s
    dr = _draws(seed, problem_id, n_pad, r1, row_offset, draws)
    xp = np.zeros((n_pad, q))
    xp[:n] = X
    sigma = dr["sigma"][:n_pad] if sign_flip else np.ones(n_pad)
    z = sigma[:, None] * xp                                  # D·X
    h_s = sylvester_hadamard(s) / np.sqrt(s)                  # normalized H_s
    g_h = np.matmul(h_s[None, :, :], z.reshape(nb, s, q)).reshape(n_pad, q)   # H_s·z_β per block
    g_i = z                                                   # I_s·z_β per block
    t_h = 4.0 * dr["cauchy_h"][:n_pad, None] * g_h            # 4·C on the Hadamard half
    t_i = 4.0 * dr["cauchy_i"][:n_pad, None] * g_i            # 4·C on the identity half
    zabs = np.abs(z).reshape(nb, s, q).sum(axis=1) / np.sqrt(s)              # Σ_k |H_s,ιk|·|z_k| per block
    a_h = 4.0 * np.abs(dr["cauchy_h"][:n_pad, None]) * np.repeat(zabs, s, axis=0)
    a_i = np.abs(t_i)
    hh = dr["hash_h"][:n_pad]
    hi = dr["hash_i"][:n_pad]
    pix = np.zeros((r1, q))
    tsum = np.zeros((r1, q))
    for c in range(q):                                        # B: sum each virtual row into its bucket
        pix[:, c] = (np.bincount(hh, weights=t_h[:, c], minlength=r1)
                     + np.bincount(hi, weights=t_i[:, c], minlength=r1))
        tsum[:, c] = (np.bincount(hh, weights=a_h[:, c], minlength=r1)
                      + np.bincount(hi, weights=a_i[:, c], minlength=r1))
    return pix, tsum


def dense_pi1(n: int, s: int, r1: int, seed: int = 0, problem_id: int = 0,
              row_offset: int = 0, sign_flip: bool = True, draws: dict | None = None) -> np.ndarray:
    """Π1 formed explicitly as the product 4·B·C·H̃·D of the four factors (r1 × n_pad).

    Only for small n: this builds every factor as a matrix and multiplies them.
    """
    n_pad = padded_rows(n, s)
    nb = n_pad // s
    dr = _draws(seed, problem_id, n_pad, r1, row_offset, draws)
    g_s = np.vstack([sylvester_hadamard(s) / np.sqrt(s), np.eye(s)])       # G_s = [H_s; I_s]
    h_tilde = sp.block_diag([sp.csr_matrix(g_s)] * nb, format="csr")                    # 2n × n
    cdiag = np.empty(2 * n_pad)
    bcol = np.empty(2 * n_pad, dtype=np.int64)
    for beta in range(nb):
        rows = slice(beta * s, (beta + 1) * s)
        cdiag[2 * s * beta: 2 * s * beta + s] = dr["cauchy_h"][rows]
        cdiag[2 * s * beta + s: 2 * s * (beta + 1)] = dr["cauchy_i"][rows]
        bcol[2 * s * beta: 2 * s * beta + s] = dr["hash_h"][rows]
        bcol[2 * s * beta + s: 2 * s * (beta + 1)] = dr["hash_i"][rows]
    b_mat = np.zeros((r1, 2 * n_pad))
    b_mat[bcol, np.arange(2 * n_pad)] = 1.0
    c_mat = sp.diags(cdiag)
    sigma = dr["sigma"][:n_pad] if sign_flip else np.ones(n_pad)
    d_mat = sp.diags(sigma)
    right = (c_mat @ h_tilde @ d_mat).toarray()                             # C·H̃·D
    return 4.0 * b_mat @ right
