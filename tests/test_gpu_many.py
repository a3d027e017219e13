"""k coresets from one λ (l1_sample_lambda), k solves side by side (l1_solve_many), and the
separable canonical-row design of the large-scale experiment (§6.3), on the GPU.

Bars: with Σλ from l1_lambda and k = 1 the coreset is l1_sample's, bit for bit; coreset j
of k is the oracle's Bernoulli sample with problem id problem_id + j given the same λ and
Σλ, bit for bit (indices, weights, rows), with even and odd global row offsets; the
OptimizedFastCauchyRegression form likewise with p̂ = min(1, s·λ̂); an overflowing capacity
keeps the ordered prefix and raises CAPACITY; Σλ = 0 raises ZERO_MASS and keeps nothing.
Each of k side-by-side solves has the objective of l1_solve on the same coreset (1e-9
relative) and of the oracle's LP (1e-6 relative, the coreset-objective tolerance).  On the
canonical design the library's k solutions are certified, and their distance from the
optimal box (per-coordinate medians, checked against the oracle) is small.
"""
import numpy as np
import pytest
import torch

import paper_1207_4684_gb300 as L
from gpu_util import DEV, host_x, problem, to_device
from oracle import rng, sampling, separable, solve
from synth import canonical_design, r1_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1207_4684_gb300 import build

    build.build()
    L.load()
    torch.cuda.set_device(0)


def _lambda(A, b, prm, ws):
    """M from this pass's own Π1X, then λ and Σλ by l1_lambda."""
    n, d = A.shape
    q = d + 1
    pix = torch.empty((prm.r1, q), dtype=torch.float32, device=DEV)
    M = torch.empty((q, prm.r2), dtype=torch.float64, device=DEV)
    lam = torch.empty(n, dtype=torch.float32, device=DEV)
    tot = torch.empty(1, dtype=torch.float64, device=DEV)
    L.l1s_status_reset(ws)
    L.fct_embed(A, b, prm, pix, ws)
    L.l1_condition(pix, prm, None, M, ws)
    L.l1_lambda(A, b, M, prm, lam, tot, ws)
    return M, lam, tot


def _sample_many(A, b, lam, tot, prm, k, cap):
    n, d = A.shape
    ws = torch.empty(L.sample_lambda_workspace_size(prm, n, d, L.BF16 if A.dtype == torch.bfloat16 else L.F32, k),
                     dtype=torch.uint8, device=DEV)
    idx = torch.full((k, cap), -1, dtype=torch.int64, device=DEV)
    w = torch.zeros((k, cap), dtype=torch.float64, device=DEV)
    core = torch.zeros((k, cap, d + 1), dtype=torch.float64, device=DEV)
    cnt = torch.zeros(k, dtype=torch.int64, device=DEV)
    L.l1s_status_reset(ws)
    L.l1_sample_lambda(A, b, lam, tot, prm, k, cap, idx, w, core, cnt, ws)
    flags = L.l1s_status_read(ws)
    return idx.cpu().numpy(), w.cpu().numpy(), core.cpu().numpy(), cnt.cpu().numpy(), flags


@pytest.mark.parametrize("n,d,dtype", [(70001, 8, "f32"), (40000, 24, "bf16")])
def test_k1_equals_l1_sample(n, d, dtype):
    pr = problem(n, d, seed=3, dtype=dtype)
    A, b = to_device(pr)
    prm = L.make_params(64, r1_for(d), 16, 900.0, seed=11)
    dt = L.BF16 if dtype == "bf16" else L.F32
    ws = L.workspace(prm, n, d, dt)
    M, lam, tot = _lambda(A, b, prm, ws)
    cap = 2000
    idx = torch.full((cap,), -1, dtype=torch.int64, device=DEV)
    w = torch.zeros(cap, dtype=torch.float64, device=DEV)
    core = torch.zeros((cap, d + 1), dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    lam_s = torch.empty(n, dtype=torch.float32, device=DEV)
    L.l1s_status_reset(ws)
    L.l1_sample(A, b, M, prm, cap, idx, w, core, cnt, lam_s, ws)
    assert L.l1s_status_read(ws) == 0
    assert torch.equal(lam_s, lam)
    i1, w1, c1, n1, flags = _sample_many(A, b, lam, tot, prm, 1, cap)
    assert flags == 0
    c = int(cnt.item())
    assert n1[0] == c and 0 < c <= cap
    assert np.array_equal(i1[0, :c], idx[:c].cpu().numpy())
    assert np.array_equal(w1[0, :c], w[:c].cpu().numpy())
    assert np.array_equal(c1[0, :c], core[:c].cpu().numpy())


@pytest.mark.parametrize("s,offset", [(64, 0), (64, 64 * 1001), (1, 12345)])
def test_k_coresets_match_oracle(s, offset):
    n, d, k, m = 50003, 8, 5, 700.0
    pr = problem(n, d, seed=5)
    A, b = to_device(pr)
    prm = L.make_params(s, r1_for(d), 16, m, seed=4, problem_id=7, global_row_offset=offset)
    ws = L.workspace(prm, n, d)
    _, lam, tot = _lambda(A, b, prm, ws)
    cap = 1500
    idx, w, core, cnt, flags = _sample_many(A, b, lam, tot, prm, k, cap)
    assert flags == 0
    X = host_x(pr)
    p, _, _ = sampling.probabilities(lam.cpu().numpy().astype(np.float64), m, total=float(tot.item()))
    for j in range(k):
        u = rng.sample_uniforms(4, 7 + j, offset + np.arange(n))
        ri, rw = sampling.bernoulli_sample(p, u)
        c = int(cnt[j])
        assert c == len(ri) and c <= cap, (j, c, len(ri))
        assert np.array_equal(idx[j, :c], ri), j
        assert np.array_equal(w[j, :c], rw), j
        assert np.array_equal(core[j, :c], X[ri]), j
    # independent coresets: the overlap of two is about Σ p̂², far below either size
    both = np.intersect1d(idx[0, :cnt[0]], idx[1, :cnt[1]]).size
    assert both < 5 * (float(np.sum(p * p)) + 10)


def test_optimized_form_many():
    n, d, k, scale = 30000, 8, 3, 0.4
    pr = problem(n, d, seed=6)
    A, b = to_device(pr)
    prm = L.make_params(64, r1_for(d), 8, 4000.0, seed=9, variant=1, sample_scale=scale)
    lam = torch.from_numpy(np.abs(np.random.default_rng(2).standard_cauchy(n)).astype(np.float32) * 0.05).to(DEV)
    idx, w, core, cnt, flags = _sample_many(A, b, lam, None, prm, k, 8000)
    assert flags == 0
    p = sampling.probabilities_scaled(lam.cpu().numpy().astype(np.float64), scale)
    for j in range(k):
        ri, rw = sampling.bernoulli_sample(p, rng.sample_uniforms(9, j, np.arange(n)))
        c = int(cnt[j])
        assert c == len(ri)
        assert np.array_equal(idx[j, :c], ri) and np.array_equal(w[j, :c], rw)


def test_capacity_and_zero_mass():
    n, d = 20000, 4
    pr = problem(n, d, seed=8)
    A, b = to_device(pr)
    prm = L.make_params(64, r1_for(d), 16, 500.0, seed=1)
    ws = L.workspace(prm, n, d)
    _, lam, tot = _lambda(A, b, prm, ws)
    full_i, _, _, full_c, f0 = _sample_many(A, b, lam, tot, prm, 2, 2000)
    assert f0 == 0
    small_i, _, _, small_c, f1 = _sample_many(A, b, lam, tot, prm, 2, 10)
    assert f1 == L.flag(7)                        # CAPACITY
    assert np.array_equal(small_c, full_c)
    assert np.array_equal(small_i[:, :10], full_i[:, :10])
    zero = torch.zeros(1, dtype=torch.float64, device=DEV)
    _, _, _, zc, fz = _sample_many(A, b, lam, zero, prm, 3, 100)
    assert fz == L.flag(6) and np.all(zc == 0)    # ZERO_MASS


def _solve_one(core, w, cnt, cap, d):
    x = torch.empty(d, dtype=torch.float64, device=DEV)
    obj = torch.empty(1, dtype=torch.float64, device=DEV)
    ws = torch.empty(1 << 26, dtype=torch.uint8, device=DEV)
    L.l1_solve(core, w, cnt, cap, d, 100, x, obj, ws)
    return x.cpu().numpy(), float(obj.item())


@pytest.mark.parametrize("d,k", [(4, 3), (12, 6)])
def test_solve_many_matches_single_and_lp(d, k):
    n, m = 60000, 600.0
    pr = problem(n, d, seed=10)
    A, b = to_device(pr)
    prm = L.make_params(64, r1_for(d), 16, m, seed=2)
    ws = L.workspace(prm, n, d)
    _, lam, tot = _lambda(A, b, prm, ws)
    cap = 1400
    dw = torch.empty(L.sample_lambda_workspace_size(prm, n, d, L.F32, k), dtype=torch.uint8, device=DEV)
    idx = torch.empty((k, cap), dtype=torch.int64, device=DEV)
    w = torch.empty((k, cap), dtype=torch.float64, device=DEV)
    core = torch.empty((k, cap, d + 1), dtype=torch.float64, device=DEV)
    cnt = torch.empty(k, dtype=torch.int64, device=DEV)
    L.l1_sample_lambda(A, b, lam, tot, prm, k, cap, idx, w, core, cnt, dw)
    sws = torch.empty(L.solve_many_workspace_size(cap, d, k), dtype=torch.uint8, device=DEV)
    x = torch.empty((k, d), dtype=torch.float64, device=DEV)
    obj = torch.empty(k, dtype=torch.float64, device=DEV)
    fl = torch.full((k,), -1, dtype=torch.int32, device=DEV)
    L.l1_solve_many(core, w, cnt, cap, d, k, 100, x, obj, fl, sws)
    torch.cuda.synchronize()
    assert torch.all(fl == 0), fl
    for j in range(k):
        c = int(cnt[j].item())
        assert 0 < c <= cap
        x1, f1 = _solve_one(core[j].contiguous(), w[j].contiguous(), cnt[j:j + 1].clone(), cap, d)
        fj = float(obj[j].item())
        assert abs(fj - f1) <= 1e-9 * f1, (j, fj, f1)
        rows = core[j, :c].cpu().numpy()
        _, f_lp = solve.lad_lp(rows[:, :d], -rows[:, d], w[j, :c].cpu().numpy())
        assert abs(fj - f_lp) <= 1e-6 * f_lp, (j, fj, f_lp)
        f_x = solve.weighted_objective(rows[:, :d], -rows[:, d], w[j, :c].cpu().numpy(), x[j].cpu().numpy())
        assert abs(f_x - fj) <= 1e-9 * fj


def test_canonical_design_many_solutions():
    """§6.3 at n = 2^18: the slow Cauchy transform conditions, 16 coresets of about 10^4 rows
    come from one λ, and 16 solves run side by side."""
    from paper_1207_4684_gb300 import validation

    n, d, k, m = 1 << 18, 15, 16, 1e4
    cd = canonical_design(n, d, seed=4)
    cols = torch.from_numpy(cd["cols"].astype(np.int64)).to(DEV)
    A = torch.zeros((n, d), dtype=torch.float32, device=DEV)
    A.scatter_(1, cols[:, None], 1.0)
    b = torch.from_numpy(cd["b"]).to(DEV)
    prm = L.make_params(128, r1_for(d), 16, m, seed=5, transform=1)
    out = validation.many_solutions(A, b, prm, k)
    assert out["status"] == 0
    assert torch.all(out["solve_flags"] == 0)
    cnt = out["count"].cpu().numpy()
    # E[count] = Σ min(1, τ·λ_i) ≤ m_s: the rarest entries (8 rows at n = 2^18) are all kept
    assert np.all((cnt > 0.5 * m) & (cnt < m + 6 * np.sqrt(m))), cnt
    lo, hi = validation.canonical_box(cols, b, d)
    olo, ohi = separable.canonical_optimum(cd["cols"], cd["b"], d)
    assert np.array_equal(lo.numpy(), olo) and np.array_equal(hi.numpy(), ohi)
    err = validation.box_errors(out["x"], lo, hi)
    ref = [separable.relative_errors(xj, olo, ohi, olo) for xj in out["x"].cpu().numpy()]
    for key in ("l1", "l2", "linf"):
        assert np.allclose(err[key], [r[key] for r in ref], rtol=1e-12, atol=0)
    assert max(err["l1"]) < 0.2 and np.median(err["l1"]) < 0.08, err["l1"]
    # every coordinate is sampled: ℓ1 conditioning spreads the coreset across the 15 entries
    idx = out["idx"].cpu().numpy()
    for j in range(k):
        got = np.bincount(cd["cols"][idx[j, : cnt[j]]].astype(np.int64), minlength=d)
        assert got.min() > 0, got


def test_canonical_coresets_solved_to_their_weighted_medians():
    """At n = 2^22 and 10^5-row coresets, the solves' vertex start passes over hundreds of rows
    of the large groups (their A parts repeat) before every coordinate has a row; each solve
    must still end certified, at the coreset's own optimum: per coordinate a weighted median
    of the group's responses (oracle weighted_median), objective within 1e-12."""
    from paper_1207_4684_gb300 import validation

    n, d, k, m = 1 << 22, 15, 4, 1e5
    cd = canonical_design(n, d, seed=9)
    cols = torch.from_numpy(cd["cols"].astype(np.int64)).to(DEV)
    A = torch.zeros((n, d), dtype=torch.float32, device=DEV)
    A.scatter_(1, cols[:, None], 1.0)
    b = torch.from_numpy(cd["b"]).to(DEV)
    prm = L.make_params(1, r1_for(d), 16, m, seed=3, transform=1)
    out = validation.many_solutions(A, b, prm, k)
    assert out["status"] == 0
    assert torch.all(out["solve_flags"] == 0), out["solve_flags"]
    for j in range(k):
        c = int(out["count"][j].item())
        X = out["coreset"][j, :c].cpu().numpy()
        w = out["w"][j, :c].cpu().numpy()
        Aj, bj = X[:, :d], -X[:, d]
        g = Aj.argmax(1)
        xm = np.array([solve.weighted_median(bj[g == t], w[g == t]) for t in range(d)])
        f_opt = solve.weighted_objective(Aj, bj, w, xm)
        f = float(out["objective"][j].item())
        assert abs(f - f_opt) <= 1e-12 * f_opt, (j, f, f_opt)
