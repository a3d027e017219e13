"""Multiple ℓ1 regression (§4.2.1, FastCauchyRegression(A, B)) on the GPU against the FP64 oracle.

X = [A, −B] has q = d + k columns and one coreset serves all k right-hand sides.
Bars: the kept set equals the oracle's Bernoulli decisions (its own FP64 Π1X, QR, M, λ)
wherever u_i is not within 1e-4·p̂_i of p̂_i; weights 1/p̂ within 1e-2; coreset rows
are exactly the rows [A_i, −B_i] of X; each column of W reaches the LP optimum of its
coreset problem within 1e-6 and its objective equals ‖A·W_j − B_j‖₁ in FP64.
"""
import numpy as np
import pytest
import torch

import paper_1207_4684_gb300 as L
from gpu_util import DEV, ambiguous
from oracle import pipeline, solve
from synth import r1_for
from synth.inputs import bf16_bits_to_f32, f32_to_bf16_bits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1207_4684_gb300 import build

    build.build()
    L.load()
    torch.cuda.set_device(0)


def make_xb(n, d, k, seed, sparse=False):
    """[A | B] in FP32: A Gaussian, B = A·W* + noise (Laplace with 5% 100·Cauchy outliers,
    or, with sparse=True, 1% gross errors and exact elsewhere)."""
    g = np.random.default_rng(seed)
    A = g.standard_normal((n, d)).astype(np.float32)
    W = g.standard_normal((d, k))
    if sparse:
        E = np.where(g.random((n, k)) < 0.01, 50.0 * g.standard_normal((n, k)), 0.0)
    else:
        E = g.laplace(size=(n, k))
        out = g.random((n, k)) < 0.05
        E[out] = 100.0 * g.standard_cauchy(int(out.sum()))
    B = (A.astype(np.float64) @ W + E).astype(np.float32)
    return np.ascontiguousarray(np.concatenate([A, B], axis=1)), W


def x_device(XB, dtype):
    if dtype == "bf16":
        bits = f32_to_bf16_bits(XB)
        return torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).to(DEV), bf16_bits_to_f32(bits)
    return torch.from_numpy(XB).to(DEV), XB


@pytest.mark.parametrize("n,d,k,s,r2,m,dtype", [(65536, 8, 3, 64, 16, 2000.0, "f32"),
                                                 (40001, 16, 4, 256, 16, 1500.0, "f32"),
                                                 (20000, 8, 2, 64, 16, 800.0, "bf16"),
                                                 (3000, 3, 1, 16, 16, 300.0, "f32")])
def test_multi_coreset_matches_oracle(n, d, k, s, r2, m, dtype):
    XB, _ = make_xb(n, d, k, seed=n + d + k)
    Xd, XB_vals = x_device(XB, dtype)
    r1 = r1_for(d + k)
    ref = pipeline.fast_cauchy_multiple_regression(XB_vals[:, :d], XB_vals[:, d:], s, r1, r2, m, seed=6,
                                                   problem_id=2, solve_lp=False)
    prm = L.make_params(s, r1, r2, m, seed=6, problem_id=2)
    ws = L.multi_workspace(prm, n, d, k, L.BF16 if dtype == "bf16" else L.F32)
    cap = int(2 * m) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=DEV)
    w = torch.empty(cap, dtype=torch.float64, device=DEV)
    core = torch.empty((cap, d + k), dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    L.l1_coreset_multi(Xd, k, prm, cap, idx, w, core, cnt, ws)
    assert L.l1s_status_read(ws) == 0
    kk = int(cnt.item())
    got = idx[:kk].cpu().numpy()
    p, u = ref["p"], ref["u"]
    amb = ambiguous(u, p, 1e-4)
    kg = np.zeros(n, bool)
    kg[got] = True
    assert np.array_equal(kg[~amb], (u < p)[~amb]), int((kg != (u < p)).sum())
    assert np.allclose(w[:kk].cpu().numpy(), 1.0 / p[got], rtol=1e-2, atol=0)
    assert np.array_equal(core[:kk].cpu().numpy(), ref["X"][got])


@pytest.mark.parametrize("n,d,k,sparse", [(30000, 4, 3, False), (50000, 8, 2, True)])
def test_multi_regress(n, d, k, sparse):
    XB, Wstar = make_xb(n, d, k, seed=7 * n + k, sparse=sparse)
    Xd = torch.from_numpy(XB).to(DEV)
    r1, m = r1_for(d + k), 1500.0
    prm = L.make_params(64, r1, 16, m, seed=11)
    ws = L.multi_workspace(prm, n, d, k)
    W, f, rows, rc = L.l1_regress_multi(Xd, k, prm, ws)
    assert rc == 0, rc
    A = XB[:, :d].astype(np.float64)
    Bm = XB[:, d:].astype(np.float64)
    W = W.numpy()
    for j in range(k):
        fj = solve.objective(A, Bm[:, j], W[:, j])
        assert abs(f[j].item() - fj) <= 1e-12 * fj, j
        f_star = solve.objective(A, Bm[:, j], Wstar[:, j])
        assert f[j].item() <= 1.01 * f_star, j
    if sparse:
        # ℓ1 regression recovers W* exactly under sparse gross errors (within FP32 storage of B)
        assert np.allclose(W, Wstar, rtol=0, atol=1e-5), np.abs(W - Wstar).max()
    # the same coreset, solved column by column by the oracle's LP
    cap = int(2 * m) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=DEV)
    w = torch.empty(cap, dtype=torch.float64, device=DEV)
    core = torch.empty((cap, d + k), dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    L.l1_coreset_multi(Xd, k, prm, cap, idx, w, core, cnt, ws)
    kk = int(cnt.item())
    C = core[:kk].cpu().numpy()
    wc = w[:kk].cpu().numpy()
    x = torch.empty(d, dtype=torch.float64, device=DEV)
    obj = torch.empty(1, dtype=torch.float64, device=DEV)
    sws = L.workspace(L.make_params(64, r1, 16, m), 1 << 10, d)
    for j in range(k):
        Cj = torch.from_numpy(np.ascontiguousarray(np.concatenate([C[:, :d], C[:, d + j:d + j + 1]], axis=1)))
        L.l1_solve(Cj.to(DEV), w[:kk].contiguous(), cnt, kk, d, 100, x, obj, sws)
        _, f_lp = solve.lad_lp(C[:, :d], -C[:, d + j], wc)
        f_gpu = solve.weighted_objective(C[:, :d], -C[:, d + j], wc, x.cpu().numpy())
        assert abs(f_gpu - f_lp) <= 1e-6 * f_lp, (j, f_gpu, f_lp)


def test_multi_argument_checks():
    prm = L.make_params(64, 40, 16, 100.0)
    with pytest.raises(L.L1SError):
        L.l1s_multi_workspace_size(prm, 1000, 4, 0)
    with pytest.raises(L.L1SError):
        L.l1s_multi_workspace_size(prm, 1000, 100, 40)
    X = torch.zeros((1000, 6), dtype=torch.float32, device=DEV)
    ws = L.multi_workspace(prm, 1000, 4, 2)
    cap = 300
    idx = torch.empty(cap, dtype=torch.int64, device=DEV)
    w = torch.empty(cap, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    with pytest.raises(L.L1SError):       # workspace sized for k = 2, call with k = 1 and a wider "A"
        L.l1_coreset_multi(X[:, :5], 3, prm, cap, idx, w, None, cnt, ws[:1024])
