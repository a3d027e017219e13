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
