"""Conditioning quality on the GPU (§6.1): κ̄₁(U) of the ℓ1 basis U = A·R⁻¹.

The conditioning study of §6.1 computes, for a tall test matrix A (n × d), the basis
U = A·R⁻¹ with R from the QR of Π·A, and reports κ̄₁(U) = α·β with α = ‖U‖₁ and
β = 1 / min_{‖z‖_∞ = 1} ‖U·z‖₁.  The minimum is the smallest of d ℓ1 regressions
min_y ‖U_{:,j} + U_{:,−j}·y‖₁ (a minimiser on the box boundary has a unit coordinate).

Every numerical step runs in the library: Π·A by fct_embed (FCT1, or the slow Cauchy
transform), R by l1_condition, U and α by l1_basis, each regression by l1_solve (IRLS
finished by certified simplex pivots).  This module only arranges those calls: A's last
column is passed as the library's b, so X = [A_{:, <d}, −A_{:, d}] = A·diag(1, …, 1, −1);
the QR of Π·X is then R·D with D that sign diagonal, and U_X = U·D, whose κ̄₁ equals
U's (‖U·D‖₁ = ‖U‖₁ and D maps the unit box onto itself).  Identical rows of U are passed
to the regressions once, with their count as the weight (the ℓ1 objective is the same).
"""
from __future__ import annotations

import torch

from . import l1fct as L


def kappa_bar(A: torch.Tensor, r1: int, s: int, seed: int = 0, problem_id: int = 0, transform: int = 0,
              stream=None) -> dict:
    """κ̄₁ of the ℓ1 basis of A (device, n × d FP32, d ≥ 2) conditioned by Π (FCT1 with block
    size s, or the slow Cauchy transform when transform = 1) with r1 rows."""
    n, d = A.shape
    dev = A.device
    Ap = A[:, : d - 1]                                   # rows of A with lda = d
    bp = A[:, d - 1].contiguous()
    prm = L.make_params(s, r1, 1, n / 2.0, seed=seed, problem_id=problem_id, transform=transform)
    ws = L.workspace(prm, n, d - 1, device=dev)         # its leading regions also serve l1_solve
    pix = torch.empty((r1, d), dtype=torch.float32, device=dev)
    R = torch.empty((d, d), dtype=torch.float64, device=dev)
    L.l1s_status_reset(ws, stream=stream)
    L.fct_embed(Ap, bp, prm, pix, ws, stream=stream)
    L.l1_condition(pix, prm, R, None, ws, stream=stream)
    flags = L.l1s_status_read(ws, stream=stream)
    U = torch.empty((n, d), dtype=torch.float64, device=dev)
    alpha = torch.empty(1, dtype=torch.float64, device=dev)
    L.l1_basis(Ap, bp, R, U, None, alpha, stream=stream)
    uniq, counts = torch.unique(U, dim=0, return_counts=True)
    m_rows = uniq.shape[0]
    wts = counts.to(torch.float64).contiguous()
    cnt = torch.full((1,), m_rows, dtype=torch.int64, device=dev)
    x = torch.empty(d - 1, dtype=torch.float64, device=dev)
    obj = torch.empty(1, dtype=torch.float64, device=dev)
    values = []
    for j in range(d):
        order = [k for k in range(d) if k != j] + [j]    # rows [U_{:, −j}, U_{:, j}]: b = −U_{:, j}
        rows = uniq[:, order].contiguous()
        L.l1s_status_reset(ws, stream=stream)
        L.l1_solve(rows, wts, cnt, m_rows, d - 1, 100, x, obj, ws, stream=stream)
        flags |= L.l1s_status_read(ws, stream=stream)
        values.append(float(obj.item()))
    a = float(alpha.item())
    m = min(values)
    return {"kappa_bar": a / m, "alpha": a, "min_box": m, "status": flags, "R": R}
