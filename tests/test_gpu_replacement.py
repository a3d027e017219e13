"""Sampling exactly m rows with replacement (params.variant = 2; the alternative that the
caption of Figure 2 allows) on the GPU against the FP64 oracle.

Draw t takes the row i with C_{i−1} ≤ u_t·Σλ < C_i (C the running FP64 sum of λ) and the
weight Σλ/(m·λ_i).  Bars: given the same λ, every draw equals the oracle's except where
u_t·Σλ lies within 1e-12·Σλ of a boundary C_i (the two running sums add in different
orders); weights within 1e-12; rows of zero λ are never drawn; coreset rows are the rows
of X.  For a whole pass (own Π1X, M, λ) a draw must fall in the oracle's interval of its
row widened by 1e-5·Σλ (the FP32 rounding of λ), and at least 95% of draws must agree.
"""
import numpy as np
import pytest
import torch

import paper_1207_4684_gb300 as L
from gpu_util import DEV, host_x, problem, to_device
from oracle import condition, pipeline, rng, sampling
from synth import r1_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1207_4684_gb300 import build

    build.build()
    L.load()
    torch.cuda.set_device(0)


def buffers(cap, q):
    return (torch.full((cap,), -1, dtype=torch.int64, device=DEV), torch.zeros(cap, dtype=torch.float64, device=DEV),
            torch.zeros((cap, q), dtype=torch.float64, device=DEV), torch.zeros(1, dtype=torch.int64, device=DEV))


@pytest.mark.parametrize("n,d,r2,m,zero_rows", [(100000, 8, 16, 3000, 1000), (70001, 16, 16, 20000, 0),
                                                (5000, 4, 16, 700, 37), (3, 2, 16, 10, 1)])
def test_replacement_draws_given_lambda(n, d, r2, m, zero_rows):
    pr = problem(n, d, seed=70 + d)
    if zero_rows:
        pr["A"][:zero_rows] = 0.0
        pr["b"][:zero_rows] = 0.0
    A, b = to_device(pr)
    X = host_x(pr)
    _, rm = condition.qr_positive(np.random.default_rng(5).standard_normal((4 * (d + 1), d + 1)))
    M = condition.m_matrix(rm, rng.pi2_matrix(3, 1, d + 1, r2))
    Md = torch.from_numpy(np.ascontiguousarray(M)).to(DEV)
    prm = L.make_params(64, r1_for(max(d, 2)), r2, float(m), seed=3, problem_id=1, variant=2)
    ws = L.workspace(prm, n, d)
    cap = 2 * m + 64
    idx, w, core, cnt = buffers(cap, d + 1)
    lam = torch.empty(n, dtype=torch.float32, device=DEV)
    L.l1s_status_reset(ws)
    L.l1_sample(A, b, Md, prm, cap, idx, w, core, cnt, lam, ws)
    assert L.l1s_status_read(ws) == 0
    assert int(cnt.item()) == m
    lam_g = lam.cpu().double().numpy()
    u = rng.replacement_uniforms(3, 1, np.arange(m))
    ref_idx, ref_w, cdf = sampling.sample_with_replacement(lam_g, m, u)
    got = idx[:m].cpu().numpy()
    total = cdf[-1]
    tgt = u * total
    lo = np.where(ref_idx > 0, cdf[np.maximum(ref_idx - 1, 0)], 0.0)
    amb = (np.abs(tgt - lo) <= 1e-12 * total) | (np.abs(cdf[ref_idx] - tgt) <= 1e-12 * total)
    assert np.array_equal(got[~amb], ref_idx[~amb]), int((got != ref_idx).sum())
    assert np.all(lam_g[got] > 0)
    assert np.allclose(w[:m].cpu().numpy()[~amb], ref_w[~amb], rtol=1e-12, atol=0)
    assert np.array_equal(core[:m].cpu().numpy(), X[got])


@pytest.mark.parametrize("n,d,s,m,seed,data_seed", [(65536, 8, 64, 2000, 0, None), (30000, 8, 64, 800, 6, 300),
                                                    (12345, 16, 256, 500, 6, 301)])
def test_replacement_whole_pass(n, d, s, m, seed, data_seed):
    from synth import WORKLOADS, make_problem

    if data_seed is None:
        pr = make_problem(WORKLOADS["gauss_n65536_d8"])
    else:
        pr = problem(n, d, seed=data_seed)
    A, b = to_device(pr)
    X = host_x(pr)
    r1, r2 = r1_for(d), 16
    ref = pipeline.fast_cauchy_regression(pr["A"], pr["b"], s, r1, r2, float(m), seed=seed,
                                          solve_lp=False, variant=2)
    prm = L.make_params(s, r1, r2, float(m), seed=seed, variant=2)
    ws = L.workspace(prm, n, d)
    cap = 2 * m + 64
    idx, w, core, cnt = buffers(cap, d + 1)
    L.l1_coreset(A, b, prm, cap, idx, w, core, cnt, ws)
    assert L.l1s_status_read(ws) == 0
    got = idx[:m].cpu().numpy()
    cdf = np.cumsum(ref["lam"])
    total = cdf[-1]
    tgt = rng.replacement_uniforms(seed, 0, np.arange(m)) * total
    lo = np.where(got > 0, cdf[np.maximum(got - 1, 0)], 0.0)
    delta = 1e-5 * total
    assert np.all((lo - delta <= tgt) & (tgt < cdf[got] + delta))
    assert (got == ref["idx"]).mean() >= 0.95
    assert np.allclose(w[:m].cpu().numpy(), total / (m * ref["lam"][got]), rtol=1e-4)
    assert np.array_equal(core[:m].cpu().numpy(), X[got])


def test_replacement_argument_checks():
    with pytest.raises(L.L1SError) as e:
        L.l1s_workspace_size(L.make_params(64, 20, 16, 100.5, variant=2), 1000, 4)
    assert e.value.code == 1 and "integer" in str(e.value)
    with pytest.raises(L.L1SError):
        L.l1s_workspace_size(L.make_params(64, 20, 16, 100.0, variant=2, sample_scale=1.0), 1000, 4)


def test_replacement_batch_members():
    """Members of a batch drawing with replacement (M in shared memory, workspace slices):
    each member's draws fall in the oracle's intervals of its own whole pass, and equal the
    draws of the same problem run alone (l1_coreset) except where the target lies within
    1e-5·Σλ of a boundary of the running sum (the two Π1X may differ in their last bits), so a
    member that read another member's slice of the workspace would fail.  The members'
    device inputs stay alive (in `data`) until the batch has run."""
    members = [(30000, 8, 64, 16, 800), (12345, 16, 256, 16, 500), (5000, 4, 16, 16, 300)]
    data, probs = [], []
    for pid, (n, d, s, r2, m) in enumerate(members):
        pr = problem(n, d, seed=300 + pid)
        ref = pipeline.fast_cauchy_regression(pr["A"], pr["b"], s, r1_for(d), r2, float(m), seed=6,
                                              problem_id=pid, solve_lp=False, variant=2)
        A, b = to_device(pr)
        prm = L.make_params(s, r1_for(d), r2, float(m), seed=6, problem_id=pid, variant=2)
        cap = 2 * m + 64
        idx, w, _, cnt = buffers(cap, d + 1)
        alone_ws = L.workspace(prm, n, d)
        aidx, aw, _, acnt = buffers(cap, d + 1)
        L.l1_coreset(A, b, prm, cap, aidx, aw, None, acnt, alone_ws)
        assert L.l1s_status_read(alone_ws) == 0
        data.append(dict(ref=ref, m=m, idx=idx, w=w, cnt=cnt, A=A, b=b, alone=aidx[:m].cpu().numpy()))
        probs.append(L.make_problem(A, b, prm, cap, idx, w, None, cnt))
    ws = L.batched_workspace(probs)
    flags = torch.zeros(len(probs), dtype=torch.int32, device=DEV)
    L.l1_regress_batched(probs, ws, flags)
    torch.cuda.synchronize()
    assert int(flags.abs().sum().item()) == 0
    for pid, e in enumerate(data):
        m = e["m"]
        assert int(e["cnt"].item()) == m
        got = e["idx"][:m].cpu().numpy()
        cdf = np.cumsum(e["ref"]["lam"])
        total = cdf[-1]
        tgt = rng.replacement_uniforms(6, pid, np.arange(m)) * total
        lo = np.where(got > 0, cdf[np.maximum(got - 1, 0)], 0.0)
        delta = 1e-5 * total
        assert np.all((lo - delta <= tgt) & (tgt < cdf[got] + delta)), pid
        assert (got == e["ref"]["idx"]).mean() >= 0.95, pid
        k = np.clip(np.searchsorted(cdf, tgt), 1, cdf.size - 1)
        near = np.minimum(np.abs(tgt - cdf[k - 1]), np.abs(tgt - cdf[k])) <= delta
        assert np.array_equal(got[~near], e["alone"][~near]), (pid, int((got != e["alone"]).sum()))
        assert np.allclose(e["w"][:m].cpu().numpy(), total / (m * e["ref"]["lam"][got]), rtol=1e-4), pid
