"""Helpers shared by the GPU parity tests: inputs on the device, the oracle on the host."""
from __future__ import annotations

import math

import numpy as np
import torch

import paper_1207_4684_gb300 as L
from oracle import fct, pipeline
from synth import make_problem
from synth.inputs import bf16_bits_to_f32

DEV = "cuda"

# Tolerance of an FP32 entry of Π1X against the FP64 oracle, relative to the sum of
# |contributing terms| of that entry.
PIX_REL = 1e-5


def to_device(pr: dict, lda: int | None = None):
    """A (float32, or bfloat16 from its bits) and b as device tensors; optional padded lda."""
    A = pr["A"]
    if A.dtype == np.uint16:
        t = torch.from_numpy(A.view(np.int16)).view(torch.bfloat16)
    else:
        t = torch.from_numpy(A)
    if lda is not None and lda > t.shape[1]:
        big = torch.zeros((t.shape[0], lda), dtype=t.dtype)
        big[:, : t.shape[1]] = t
        t = big.to(DEV)[:, : A.shape[1]]
    else:
        t = t.to(DEV)
    return t, torch.from_numpy(pr["b"]).to(DEV)


def host_x(pr: dict) -> np.ndarray:
    """X = [A, −b] in FP64 from exactly the stored values."""
    A = pr["A"]
    if A.dtype == np.uint16:
        A = bf16_bits_to_f32(A)
    return pipeline.form_x(A, pr["b"])


def problem(n: int, d: int, seed: int = 0, dtype: str = "f32", design: str = "gauss") -> dict:
    from dataclasses import replace

    from synth.inputs import Workload

    w = Workload(f"test_{n}_{d}", n, d, 64, 16, 100.0, dtype, design, "laplace_outliers", seed=seed)
    return make_problem(w)


def gpu_pix(A, b, prm, ws=None):
    n, d = A.shape
    if ws is None:
        ws = L.workspace(prm, n, d, L.BF16 if A.dtype == torch.bfloat16 else L.F32)
    pix = torch.empty((prm.r1, d + 1), dtype=torch.float32, device=DEV)
    L.l1s_status_reset(ws)
    L.fct_embed(A, b, prm, pix, ws)
    flags = L.l1s_status_read(ws)
    return pix.cpu().double().numpy(), flags


def check_pix(got: np.ndarray, X: np.ndarray, prm, rel: float = PIX_REL):
    ref, tsum = fct.fct1_embed(X, prm.s, prm.r1, prm.seed, prm.problem_id, prm.global_row_offset,
                               bool(prm.sign_flip))
    err = np.abs(got - ref)
    bound = rel * tsum
    bad = err > bound
    assert not bad.any(), (f"{int(bad.sum())} entries of Π1X outside {rel}·Σ|terms|; worst ratio "
                           f"{float((err / np.maximum(tsum, 1e-300)).max()):.3e}")
    return float((err / np.maximum(tsum, 1e-300)).max())


def lambda_tol(X: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Rounding bound of an FP32 Λ row: (q+2)·2^-24·max_j Σ_k |X_ik||M_kj| (FMA chain of q terms
    plus the rounding of M to FP32)."""
    from oracle import leverage

    q = X.shape[1]
    return (q + 2) * 2.0 ** -24 * leverage.lambda_term_scale(X, M)


def tensor_core_form(dtype: str, d: int, r2: int, lda) -> bool:
    """Shapes whose λ runs on the tensor cores: BF16 A with 16 < d ≤ 64, r2 ∈ {16, 32} and a
    row pitch that is a multiple of 16 bytes."""
    pitch = d if lda is None else lda
    return dtype == "bf16" and 16 < d <= 64 and r2 in (16, 32) and (pitch * 2) % 16 == 0


def lambda_tol_tc(X: np.ndarray, Mm: np.ndarray) -> np.ndarray:
    """Rounding bound of a tensor-core Λ row against the FP64 value with the same BF16 M_A:
    the BF16 products are exact in FP32; the K = d accumulation and the FP32 b term add at
    most (d + 2) roundings; a factor 2 covers an accumulator that truncates instead of
    rounding to nearest."""
    from oracle import leverage

    q = X.shape[1]
    return 2 * (q + 2) * 2.0 ** -24 * leverage.lambda_term_scale(X, Mm)


def ambiguous(u: np.ndarray, p: np.ndarray, rel: float) -> np.ndarray:
    return np.abs(u - p) <= rel * np.maximum(p, 1e-300)


def fsum(a) -> float:
    return math.fsum(np.asarray(a, dtype=np.float64).tolist())
