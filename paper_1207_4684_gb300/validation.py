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
              fjlt_rows: int = 0, stream=None) -> dict:
    """κ̄₁ of the ℓ1 basis of A (device, n × d FP32, d ≥ 2) conditioned by Π (FCT1 with block
    size s, the slow Cauchy transform when transform = 1, FCT2 with blocks of t = s rows of
    which fjlt_rows are kept when transform = 2) with r1 rows."""
    n, d = A.shape
    dev = A.device
    Ap = A[:, : d - 1]                                   # rows of A with lda = d
    bp = A[:, d - 1].contiguous()
    prm = L.make_params(s, r1, 1, n / 2.0, seed=seed, problem_id=problem_id, transform=transform,
                        fjlt_rows=fjlt_rows)
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


# ----------------------------------------------------------------- §6.3: many coresets, one pass
def many_solutions(A: torch.Tensor, b: torch.Tensor, prm: L.Params, k: int, capacity: int | None = None,
                   max_iter: int = 100, stream=None) -> dict:
    """The k approximate solutions of one sampling pass (§6.3): Π1·X by fct_embed, R and M
    by l1_condition, λ and Σλ by l1_lambda (one read of A each), then k coresets from that
    λ (l1_sample_lambda, coreset j drawn with problem id prm.problem_id + j) and their k
    weighted ℓ1 solves side by side (l1_solve_many).  Returns the device results and the
    CUDA-event time of each phase."""
    n, d = A.shape
    dev = A.device
    q = d + 1
    dt = L.BF16 if A.dtype == torch.bfloat16 else L.F32
    cap = int(capacity if capacity is not None else 2 * prm.coreset_size + 64)
    ws = torch.empty(L.sample_lambda_workspace_size(prm, n, d, dt, k), dtype=torch.uint8, device=dev)
    pix = torch.empty((prm.r1, q), dtype=torch.float32, device=dev)
    M = torch.empty((q, prm.r2), dtype=torch.float64, device=dev)
    lam = torch.empty(n, dtype=torch.float32, device=dev)
    tot = torch.empty(1, dtype=torch.float64, device=dev)
    idx = torch.empty((k, cap), dtype=torch.int64, device=dev)
    w = torch.empty((k, cap), dtype=torch.float64, device=dev)
    core = torch.empty((k, cap, q), dtype=torch.float64, device=dev)
    cnt = torch.empty(k, dtype=torch.int64, device=dev)
    sws = torch.empty(L.solve_many_workspace_size(cap, d, k), dtype=torch.uint8, device=dev)
    x = torch.empty((k, d), dtype=torch.float64, device=dev)
    obj = torch.empty(k, dtype=torch.float64, device=dev)
    flags = torch.zeros(k, dtype=torch.int32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.stream(st):
        L.l1s_status_reset(ws, stream=st)
        ev[0].record(st)
        L.fct_embed(A, b, prm, pix, ws, stream=st)
        ev[1].record(st)
        L.l1_condition(pix, prm, None, M, ws, stream=st)
        ev[2].record(st)
        L.l1_lambda(A, b, M, prm, lam, tot, ws, stream=st)
        ev[3].record(st)
        L.l1_sample_lambda(A, b, lam, tot, prm, k, cap, idx, w, core, cnt, ws, stream=st)
        ev[4].record(st)
        L.l1_solve_many(core, w, cnt, cap, d, k, max_iter, x, obj, flags, sws, stream=st)
        ev[5].record(st)
    st.synchronize()
    names = ("embed", "condition", "lambda", "sample", "solve")
    return {"x": x, "objective": obj, "count": cnt, "solve_flags": flags, "status": L.l1s_status_read(ws, st),
            "lambda_total": tot, "idx": idx, "w": w, "coreset": core, "capacity": cap,
            "phase_ms": {nm: ev[i].elapsed_time(ev[i + 1]) for i, nm in enumerate(names)}}


def canonical_box(cols: torch.Tensor, b: torch.Tensor, d: int):
    """Lower and upper per-coordinate medians of b (FP64): the box of minimisers of ‖A·x − b‖₁
    when row i of A is e_{cols_i} (the separable design of §6.3)."""
    lo = torch.empty(d, dtype=torch.float64)
    hi = torch.empty(d, dtype=torch.float64)
    for j in range(d):
        v = torch.sort(b[cols == j].to(torch.float64)).values
        m = v.numel()
        lo[j] = v[(m + 1) // 2 - 1].item()
        hi[j] = v[m // 2].item()
    return lo, hi


def box_errors(x: torch.Tensor, lo: torch.Tensor, hi: torch.Tensor) -> dict:
    """Relative 1-, 2- and ∞-norm distance of each row of x (k × d) from the optimal box,
    relative to the same norm of lo (the columns of the §6.3 error table)."""
    x = x.detach().cpu().to(torch.float64)
    e = torch.clamp(torch.maximum(lo - x, x - hi), min=0.0)
    return {"l1": (e.sum(1) / lo.abs().sum()).tolist(),
            "l2": (e.norm(dim=1) / lo.norm()).tolist(),
            "linf": (e.abs().amax(1) / lo.abs().max()).tolist()}
