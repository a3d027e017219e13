"""OptimizedFastCauchyRegression (Figure "mainOpt") on the GPU against the FP64 oracle.

Differences from FastCauchyRegression: Π2 is Gaussian (Box–Muller on Philox stream
1) and p̂_i = min{1, s·λ̂_i} with the sampling size s given, without Σλ.  Bars: Π2
entries within FP64 rounding of the oracle's (two libm implementations), λ̂ within
the FP32 bound of its dot products, the kept set equal to the oracle's decisions
wherever u_i is not within rounding of p̂_i, the weights 1/p̂_i.
"""
import math

import numpy as np
import pytest
import torch

import paper_1207_4684_gb300 as L
from gpu_util import DEV, host_x, lambda_tol, problem, to_device
from oracle import condition, fct, leverage, rng, sampling
from synth import r1_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1207_4684_gb300 import build

    build.build()
    L.load()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("seed,pid,q,r2", [(0, 0, 9, 8), (77, 3, 17, 8), (5, 1, 33, 32), (2**40 + 1, 9, 65, 7)])
def test_gaussian_pi2_parity(seed, pid, q, r2):
    prm = L.make_params(s=64, r1=max(q, 2), r2=r2, coreset=100.0, seed=seed, problem_id=pid, variant=1,
                        sample_scale=1.0)
    got = L.l1s_debug_pi2(prm, q).cpu().numpy()
    ref = rng.pi2_gaussian_matrix(seed, pid, q, r2)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12), float(np.abs(got - ref).max())


@pytest.mark.parametrize("n,d,r2", [(70001, 8, 8), (100000, 16, 8), (30000, 32, 8), (20000, 4, 8)])
def test_lambda_r2_8_parity(n, d, r2):
    pr = problem(n, d, seed=d + 1)
    A, b = to_device(pr)
    X = host_x(pr)
    _, rm = condition.qr_positive(np.random.default_rng(3).standard_normal((4 * (d + 1), d + 1)))
    M = condition.m_matrix(rm, rng.pi2_gaussian_matrix(1, 0, d + 1, r2))
    prm = L.make_params(64, d + 1, r2, 100.0, variant=1, sample_scale=1.0)
    ws = L.workspace(prm, n, d)
    lam = torch.empty(n, dtype=torch.float32, device=DEV)
    tot = torch.zeros(1, dtype=torch.float64, device=DEV)
    L.l1_lambda(A, b, torch.from_numpy(np.ascontiguousarray(M)).to(DEV), prm, lam, tot, ws)
    got = lam.cpu().double().numpy()
    ref = leverage.lambda_estimates(X, M)
    assert np.all(np.abs(got - ref) <= lambda_tol(X, M) + 1e-300)


@pytest.mark.parametrize("n,d,s,m", [(65536, 8, 64, 2000.0), (50000, 16, 256, 1500.0), (3001, 4, 16, 400.0)])
def test_optimized_coreset_matches_oracle(n, d, s, m):
    pr = problem(n, d, seed=40 + d)
    A, b = to_device(pr)
    X = host_x(pr)
    r1, r2, seed, pid = r1_for(d), 8, 12, 2
    pix, _ = fct.fct1_embed(X, s, r1, seed, pid, 0, True)
    _, rm = condition.qr_positive(pix)
    M = condition.m_matrix(rm, rng.pi2_gaussian_matrix(seed, pid, d + 1, r2))
    lam = leverage.lambda_estimates(X, M)
    scale = m / math.fsum(lam.tolist())          # expected coreset size ≈ m
    p = sampling.probabilities_scaled(lam, scale)
    u = rng.sample_uniforms(seed, pid, np.arange(n))
    prm = L.make_params(s, r1, r2, m, seed=seed, problem_id=pid, variant=1, sample_scale=scale)
    ws = L.workspace(prm, n, d)
    cap = int(2 * m) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=DEV)
    w = torch.empty(cap, dtype=torch.float64, device=DEV)
    core = torch.empty((cap, d + 1), dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    L.l1_coreset(A, b, prm, cap, idx, w, core, cnt, ws)
    assert L.l1s_status_read(ws) == 0
    k = int(cnt.item())
    got = idx[:k].cpu().numpy()
    keep_g = np.zeros(n, bool)
    keep_g[got] = True
    amb = np.abs(u - p) <= 1e-3 * np.maximum(p, 1e-300)
    assert np.array_equal(keep_g[~amb], (u < p)[~amb]), int((keep_g != (u < p)).sum())
    assert np.allclose(w[:k].cpu().numpy(), 1.0 / p[got], rtol=1e-2, atol=0)
    assert np.array_equal(core[:k].cpu().numpy(), X[got])
    assert abs(k - p.sum()) < 6 * math.sqrt(p.sum()) + 2


def test_variant_argument_checks():
    with pytest.raises(L.L1SError) as e:
        L.l1s_workspace_size(L.make_params(64, 20, 8, 100.0, variant=1, sample_scale=0.0), 1000, 4)
    assert e.value.code == 1 and "sample_scale" in str(e.value)
    with pytest.raises(L.L1SError) as e:
        L.l1s_workspace_size(L.make_params(64, 20, 8, 100.0, variant=2, sample_scale=1.0), 1000, 4)
    assert e.value.code == 1 and "variant" in str(e.value)


@pytest.mark.parametrize("n,d,r2,offset,with_lam", [(70001, 16, 8, 0, True), (50001, 8, 16, 12345, False),
                                                     (40000, 32, 16, 7, True), (30000, 4, 8, 1, False),
                                                     (65, 16, 8, 3, False)])
def test_fused_lambda_mark(n, d, r2, offset, with_lam):
    """λ̂ and the keep decision in one pass (no Σλ): given the same M, the kept set equals
    the decisions u_i < min(1, s·λ̂_i) from the GPU's own λ̂ (FP32, compared with the oracle
    within its rounding bound), and the weights 1/p̂ of the kept rows come from a λ̂ that
    is bit-identical to the one the decision used (recomputed by the compaction when λ̂
    is not returned).  Odd row offsets exercise the uniform pairs that straddle rows."""
    pr = problem(n, d, seed=60 + d)
    A, b = to_device(pr)
    X = host_x(pr)
    _, rm = condition.qr_positive(np.random.default_rng(4).standard_normal((4 * (d + 1), d + 1)))
    M = condition.m_matrix(rm, rng.pi2_gaussian_matrix(9, 1, d + 1, r2))
    Md = torch.from_numpy(np.ascontiguousarray(M)).to(DEV)
    lam_ref = leverage.lambda_estimates(X, M)
    m = min(1500.0, n / 4)
    scale = m / math.fsum(lam_ref.tolist())
    s = 64 if offset % 64 == 0 else 1            # row offsets are multiples of s
    prm = L.make_params(s, r1_for(d), r2, m, seed=9, problem_id=1, global_row_offset=offset, variant=1,
                        sample_scale=scale)
    ws = L.workspace(prm, n, d)
    # λ̂ from the λ kernel (same operation order) for the decisions and weights
    lam_k = torch.empty(n, dtype=torch.float32, device=DEV)
    L.l1_lambda(A, b, Md, prm, lam_k, torch.zeros(1, dtype=torch.float64, device=DEV), ws)
    lam_g = lam_k.cpu().double().numpy()
    assert np.all(np.abs(lam_g - lam_ref) <= lambda_tol(X, M) + 1e-300)
    cap = int(2 * m) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=DEV)
    w = torch.empty(cap, dtype=torch.float64, device=DEV)
    core = torch.empty((cap, d + 1), dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    lam_out = torch.full((n,), -1.0, dtype=torch.float32, device=DEV) if with_lam else None
    L.l1s_status_reset(ws)
    L.l1_sample(A, b, Md, prm, cap, idx, w, core, cnt, lam_out, ws)
    assert L.l1s_status_read(ws) == 0
    if with_lam:
        assert torch.equal(lam_out, lam_k)
    k = int(cnt.item())
    got = idx[:k].cpu().numpy()
    p = np.minimum(1.0, scale * lam_g)
    u = rng.sample_uniforms(9, 1, offset + np.arange(n))
    keep_g = np.zeros(n, bool)
    keep_g[got] = True
    amb = np.abs(u - p) <= 1e-12 * p
    assert np.array_equal(keep_g[~amb], (u < p)[~amb]), int((keep_g != (u < p)).sum())
    assert np.all(np.diff(got) > 0)
    assert np.array_equal(w[:k].cpu().numpy(), 1.0 / p[got])
    assert np.array_equal(core[:k].cpu().numpy(), X[got])


def test_optimized_batch_members():
    """OptimizedFastCauchyRegression members of a batch (M in shared memory): each member's
    kept set against the oracle's decisions from its own FP64 pass."""
    members = [(40000, 16, 256, 8, 900.0), (20001, 8, 64, 16, 600.0), (7000, 4, 16, 8, 300.0),
               (30000, 32, 256, 8, 800.0)]
    data, probs = [], []
    for pid, (n, d, s, r2, m) in enumerate(members):
        pr = problem(n, d, seed=200 + pid)
        X = host_x(pr)
        pix, _ = fct.fct1_embed(X, s, r1_for(d), 3, pid, 0, True)
        _, rm = condition.qr_positive(pix)
        M = condition.m_matrix(rm, rng.pi2_gaussian_matrix(3, pid, d + 1, r2))
        lam = leverage.lambda_estimates(X, M)
        scale = m / math.fsum(lam.tolist())
        A, b = to_device(pr)
        prm = L.make_params(s, r1_for(d), r2, m, seed=3, problem_id=pid, variant=1, sample_scale=scale)
        cap = int(2 * m) + 64
        out = dict(idx=torch.full((cap,), -1, dtype=torch.int64, device=DEV),
                   w=torch.zeros(cap, dtype=torch.float64, device=DEV),
                   cnt=torch.zeros(1, dtype=torch.int64, device=DEV))
        data.append(dict(X=X, A=A, b=b, p=sampling.probabilities_scaled(lam, scale),
                         u=rng.sample_uniforms(3, pid, np.arange(n)), out=out))
        probs.append(L.make_problem(A, b, prm, cap, out["idx"], out["w"], None, out["cnt"]))
    ws = L.batched_workspace(probs)
    flags = torch.zeros(len(probs), dtype=torch.int32, device=DEV)
    L.l1_regress_batched(probs, ws, flags)
    torch.cuda.synchronize()
    assert int(flags.abs().sum().item()) == 0
    for e in data:
        k = int(e["out"]["cnt"].item())
        got = e["out"]["idx"][:k].cpu().numpy()
        p, u = e["p"], e["u"]
        keep_g = np.zeros(len(p), bool)
        keep_g[got] = True
        amb = np.abs(u - p) <= 1e-3 * np.maximum(p, 1e-300)
        assert np.array_equal(keep_g[~amb], (u < p)[~amb])
        assert np.allclose(e["out"]["w"][:k].cpu().numpy(), 1.0 / p[got], rtol=1e-2, atol=0)
