"""Parity at the full sizes of the measured workloads, in the launch configuration that
bench.py times (default schedules, inputs resident in device memory).

colscale_n4M_d16 (n = 2^22, d = 16, FP32): every entry of Π1X against the oracle over
all rows; R and M against the oracle's QR of the same Π1X; λ on 20000 sampled rows,
computed by the oracle one by one with the GPU's M; the keep decision of every row from
the GPU's λ; the one-call pass against those decisions; the solve against the LP on its
coreset and the objective over all rows in FP64.

t2rows_n16M_d32_bf16 (n = 2^24, d = 32, BF16 A, tensor-core λ): Π1X by a property that
holds at any size (the sum of the two halves' embeddings, drawn with their global row
ids, equals the embedding of all rows) and, entry by entry, against the oracle on the
first 2^20 rows in the same launch geometry; λ on sampled rows against the oracle with
the BF16-rounded M, the keep decision of every row, and the objective over all rows.

spiky_n64M_d64 (n = 2^26, d = 64, FP32, the headline workload): the same property checks
of Π1X (halves, and every entry on a 2^20-row prefix), R and M against the oracle's QR
of the GPU's Π1X, λ on sampled rows, the keep decision of every row, and the objective of
the one-call pass over all rows.
"""
import math

import numpy as np
import pytest
import torch

import paper_1207_4684_gb300 as L
from gpu_util import DEV, PIX_REL, ambiguous, check_pix, fsum, gpu_pix, host_x, lambda_tol, lambda_tol_tc, to_device
from oracle import condition, leverage, rng, sampling, solve
from synth import WORKLOADS, make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1207_4684_gb300 import build

    build.build()
    L.load()
    torch.cuda.set_device(0)


def _phases(A, b, prm, ws, q, r1, r2):
    pix = torch.empty((r1, q), dtype=torch.float32, device=DEV)
    R = torch.empty((q, q), dtype=torch.float64, device=DEV)
    M = torch.empty((q, r2), dtype=torch.float64, device=DEV)
    L.l1s_status_reset(ws)
    L.fct_embed(A, b, prm, pix, ws)
    L.l1_condition(pix, prm, R, M, ws)
    assert L.l1s_status_read(ws) == 0
    return pix, R, M


def _check_sampling(A, b, M, prm, x_rows, w, ws, n, sample_rows, tc=False):
    """λ on sampled rows against the oracle; the keep decision of every row from the GPU's λ.
    x_rows(rows) gives the FP64 rows [A_i, −b_i] of X for sorted row ids."""
    cap = int(2 * w.coreset) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=DEV)
    wts = torch.empty(cap, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    lam = torch.empty(n, dtype=torch.float32, device=DEV)
    L.l1s_status_reset(ws)
    L.l1_sample(A, b, M, prm, cap, idx, wts, None, cnt, lam, ws)
    assert L.l1s_status_read(ws) == 0
    lam_g = lam.cpu().double().numpy()
    Mh = M.cpu().numpy()
    Mm = leverage.mixed_precision_m(Mh) if tc else Mh
    rows = np.sort(np.random.default_rng(0).choice(n, sample_rows, replace=False))
    Xr = x_rows(rows)
    ref = leverage.lambda_estimates(Xr, Mm)
    tol = lambda_tol_tc(Xr, Mm) if tc else lambda_tol(Xr, Mm)
    assert np.all(np.abs(lam_g[rows] - ref) <= tol), float((np.abs(lam_g[rows] - ref) / tol).max())
    p, _, _ = sampling.probabilities(lam_g, w.coreset, fsum(lam_g))
    u = rng.sample_uniforms(w.seed, w.problem_id, np.arange(n))
    k = int(cnt.item())
    got = idx[:k].cpu().numpy()
    keep = np.zeros(n, bool)
    keep[got] = True
    # τ = m_s/Σλ: the GPU's Σλ is within 1e-12 of the correctly rounded sum used here
    amb = ambiguous(u, p, 1e-11)
    assert np.array_equal(keep[~amb], (u < p)[~amb]), int((keep != (u < p)).sum())
    assert np.allclose(wts[:k].cpu().numpy(), 1.0 / p[got], rtol=1e-11, atol=0)
    return p, u


def test_colscale_n4M_d16_full_size():
    w = WORKLOADS["colscale_n4M_d16"]
    pr = make_problem(w)
    A, b = to_device(pr)
    X = host_x(pr)
    n, d = pr["A"].shape
    q = d + 1
    prm = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id)
    ws = L.workspace(prm, n, d)
    pix, R, M = _phases(A, b, prm, ws, q, w.r1, w.r2)
    pix_h = pix.cpu().double().numpy()
    check_pix(pix_h, X, prm, PIX_REL)                               # all 355 × 17 entries, all rows
    _, r_ref = condition.qr_positive(pix_h)
    m_ref = condition.m_matrix(r_ref, rng.pi2_matrix(w.seed, w.problem_id, q, w.r2))
    assert np.allclose(R.cpu().numpy(), r_ref, rtol=0, atol=1e-11 * np.abs(r_ref).max())
    assert np.allclose(M.cpu().numpy(), m_ref, rtol=0, atol=1e-14 * np.linalg.cond(r_ref) * np.abs(m_ref).max())
    p, u = _check_sampling(A, b, M, prm, lambda r: X[r], w, ws, n, 20000)
    # the one-call pass (its own Π1X: FP32 sums in another order) against those decisions
    cap = int(2 * w.coreset) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=DEV)
    wts = torch.empty(cap, dtype=torch.float64, device=DEV)
    core = torch.empty((cap, q), dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    L.l1_coreset(A, b, prm, cap, idx, wts, core, cnt, ws)
    assert L.l1s_status_read(ws) == 0
    k = int(cnt.item())
    got = idx[:k].cpu().numpy()
    keep = np.zeros(n, bool)
    keep[got] = True
    amb = ambiguous(u, p, 1e-4)
    assert np.array_equal(keep[~amb], (u < p)[~amb])
    # step 8 on that coreset: the GPU solve against the oracle's LP, and the objective
    Xc = core[:k].cpu().numpy()
    wc = wts[:k].cpu().numpy()
    assert np.array_equal(Xc, X[got])
    x = torch.empty(d, dtype=torch.float64, device=DEV)
    obj = torch.empty(1, dtype=torch.float64, device=DEV)
    L.l1_solve(core, wts, cnt, cap, d, 100, x, obj, ws)
    _, f_lp = solve.lad_lp(Xc[:, :-1], -Xc[:, -1], wc)
    f_gpu = solve.weighted_objective(Xc[:, :-1], -Xc[:, -1], wc, x.cpu().numpy())
    assert abs(f_gpu - f_lp) <= 1e-6 * f_lp, (f_gpu, f_lp)
    full = torch.empty(1, dtype=torch.float64, device=DEV)
    L.l1_objective(A, b, x, full, ws)
    f_full = solve.objective(X[:, :-1], -X[:, -1], x.cpu().numpy())
    assert abs(full.item() - f_full) <= 1e-12 * f_full


def test_t2rows_n16M_d32_bf16_full_size():
    w = WORKLOADS["t2rows_n16M_d32_bf16"]
    pr = make_problem(w)
    A, b = to_device(pr)
    n, d = pr["A"].shape
    q = d + 1
    prm = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id)
    ws = L.workspace(prm, n, d, L.BF16)
    pix, R, M = _phases(A, b, prm, ws, q, w.r1, w.r2)
    # Π1 is linear and its draws follow global row ids: the two halves add up to the whole
    half = n // 2                                                   # a multiple of s
    parts = []
    for lo, hi in ((0, half), (half, n)):
        prm_h = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id,
                              global_row_offset=lo)
        ws_h = L.workspace(prm_h, hi - lo, d, L.BF16)
        pp, _, _ = _phases(A[lo:hi], b[lo:hi], prm_h, ws_h, q, w.r1, w.r2)
        parts.append(pp.double())
        del ws_h
    tot = (parts[0] + parts[1]).cpu().numpy()
    whole = pix.double().cpu().numpy()
    # FP32 sums in different orders: within 2e-5 of the column's largest entry (a proxy for
    # the sum of |terms|, which heavy-tailed Cauchy weights make comparable to it)
    col = np.abs(whole).max(axis=0, keepdims=True)
    err = np.abs(tot - whole) / col
    assert np.all(err <= 2e-5), float(err.max())
    X = host_x(pr)
    # Every entry of Π1X against the oracle on the first 2^20 rows: the same kernel and
    # grid as the full launch (the grid is capped by the SM count well below 2^20 rows),
    # each block walking its pipeline through many tiles.
    pre = 1 << 20
    got_pre, flags = gpu_pix(A[:pre], b[:pre], prm)
    assert flags == 0
    check_pix(got_pre, X[:pre], prm, PIX_REL)
    _check_sampling(A, b, M, prm, lambda r: X[r], w, ws, n, 20000, tc=True)
    x, f, rows, rc = L.l1_regress(A, b, prm, ws)
    assert rc == 0, rc
    f_ref = solve.objective(X[:, :-1], -X[:, -1], x.numpy())
    assert abs(f - f_ref) <= 1e-12 * f_ref
    assert math.isfinite(f) and 0 < rows < 2 * w.coreset + 64


def test_spiky_n64M_d64_full_size():
    """The measured headline workload: Π1X by halves additivity and, entry by entry, on a
    2^20-row prefix; R and M against the oracle's QR of the GPU's Π1X; λ on sampled rows;
    every keep decision; the one-call pass's objective over all rows.  X is never formed
    whole in FP64 (35 GB): rows are widened where they are needed."""
    w = WORKLOADS["spiky_n64M_d64"]
    pr = make_problem(w)
    A, b = to_device(pr)
    n, d = pr["A"].shape
    q = d + 1

    def x_rows(rows):
        return np.concatenate([pr["A"][rows].astype(np.float64), -pr["b"][rows].astype(np.float64)[:, None]],
                              axis=1)

    prm = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id)
    ws = L.workspace(prm, n, d)
    pix, R, M = _phases(A, b, prm, ws, q, w.r1, w.r2)
    half = n // 2                                                   # a multiple of s
    parts = []
    for lo, hi in ((0, half), (half, n)):
        prm_h = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id,
                              global_row_offset=lo)
        ws_h = L.workspace(prm_h, hi - lo, d)
        pp, _, _ = _phases(A[lo:hi], b[lo:hi], prm_h, ws_h, q, w.r1, w.r2)
        parts.append(pp.double())
        del ws_h
    tot = (parts[0] + parts[1]).cpu().numpy()
    whole = pix.double().cpu().numpy()
    col = np.abs(whole).max(axis=0, keepdims=True)
    err = np.abs(tot - whole) / col
    assert np.all(err <= 2e-5), float(err.max())
    pre = 1 << 20
    got_pre, flags = gpu_pix(A[:pre], b[:pre], prm)
    assert flags == 0
    check_pix(got_pre, x_rows(np.arange(pre)), prm, PIX_REL)
    _, r_ref = condition.qr_positive(whole)
    m_ref = condition.m_matrix(r_ref, rng.pi2_matrix(w.seed, w.problem_id, q, w.r2))
    assert np.allclose(R.cpu().numpy(), r_ref, rtol=0, atol=1e-11 * np.abs(r_ref).max())
    assert np.allclose(M.cpu().numpy(), m_ref, rtol=0, atol=1e-14 * np.linalg.cond(r_ref) * np.abs(m_ref).max())
    _check_sampling(A, b, M, prm, x_rows, w, ws, n, 20000)
    x, f, rows, rc = L.l1_regress(A, b, prm, ws)
    assert rc == 0, rc
    xh = x.numpy()
    step = 1 << 22
    f_ref = math.fsum(solve.objective(pr["A"][lo:lo + step].astype(np.float64),
                                      pr["b"][lo:lo + step].astype(np.float64), xh) for lo in range(0, n, step))
    assert abs(f - f_ref) <= 1e-12 * f_ref
    assert math.isfinite(f) and 0 < rows < 2 * w.coreset + 64
