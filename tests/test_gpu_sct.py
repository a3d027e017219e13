"""The slow Cauchy transform Π1·X = (4/r1)·C·X (§3; the conditioning of §6.3) on the GPU
against the FP64 oracle, through the C ABI.

Π1X element by element within 1e-5 of the sum of |contributing terms| (the FP32 bar of the
FCT1 path), at widths of X that take one, two and three column slices, with BF16 storage,
global row offsets and ragged row counts; the one-call pass (steps 1-7 with the slow
transform as Π1) against the oracle's keep decisions; the same from host memory, where the
rows arrive in chunks whose partials add up.
"""
import numpy as np
import pytest
import torch

import paper_1207_4684_gb300 as L
from gpu_util import DEV, PIX_REL, ambiguous, host_x, problem, to_device
from oracle import condition, leverage, rng, sampling, sct
from synth import r1_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1207_4684_gb300 import build

    build.build()
    L.load()
    torch.cuda.set_device(0)


def gpu_sct(A, b, prm):
    n, d = A.shape
    ws = L.workspace(prm, n, d, L.BF16 if A.dtype == torch.bfloat16 else L.F32)
    pix = torch.empty((prm.r1, d + 1), dtype=torch.float32, device=DEV)
    L.l1s_status_reset(ws)
    L.fct_embed(A, b, prm, pix, ws)
    return pix.cpu().double().numpy(), L.l1s_status_read(ws)


@pytest.mark.parametrize("n,d,r1,dtype,offset", [(5000, 4, 45, "f32", 0), (70001, 16, 355, "f32", 0),
                                                  (20000, 8, 134, "bf16", 12345), (3001, 40, 1181, "f32", 0),
                                                  (1, 3, 7, "f32", 0), (100000, 32, 888, "bf16", 0)])
def test_sct_embed_parity(n, d, r1, dtype, offset):
    pr = problem(n, d, seed=n % 97 + d, dtype=dtype)
    A, b = to_device(pr)
    prm = L.make_params(1, r1, 16, 100.0, seed=3, problem_id=4, global_row_offset=offset, transform=1)
    got, flags = gpu_sct(A, b, prm)
    assert flags == 0
    ref, tsum = sct.sct_embed(host_x(pr), r1, seed=3, problem_id=4, row_offset=offset)
    err = np.abs(got - ref)
    ratio = float((err / np.maximum(tsum, 1e-300)).max())
    assert np.all(err <= PIX_REL * tsum), f"worst |GPU − oracle| / Σ|terms| = {ratio:.3e}"


def _oracle_decisions(X, r1, r2, m, seed):
    n, q = X.shape
    pix, _ = sct.sct_embed(X, r1, seed=seed)
    _, rm = condition.qr_positive(pix)
    M = condition.m_matrix(rm, rng.pi2_matrix(seed, 0, q, r2))
    lam = leverage.lambda_estimates(X, M)
    p, _, _ = sampling.probabilities(lam, m)
    u = rng.sample_uniforms(seed, 0, np.arange(n))
    return p, u


@pytest.mark.parametrize("host", [False, True])
def test_sct_coreset_matches_the_oracle(host):
    """Steps 1-7 with the slow transform as Π1 (the conditioning the paper runs at scale)."""
    n, d, r2, m, seed = (1 << 20) + 77 if host else 200003, 16, 16, 3000.0, 8
    pr = problem(n, d, seed=21)
    X = host_x(pr)
    r1 = r1_for(d)
    prm = L.make_params(1, r1, r2, m, seed=seed, transform=1)
    cap = int(2 * m) + 64
    if host:
        ws = L.workspace(prm, n, d, host_staging=True)
        A = torch.from_numpy(pr["A"]).pin_memory()
        b = torch.from_numpy(pr["b"]).pin_memory()
        idx = torch.empty(cap, dtype=torch.int64).pin_memory()
        w = torch.empty(cap, dtype=torch.float64).pin_memory()
        cnt = torch.zeros(1, dtype=torch.int64)
        assert L.l1_coreset_host(A, b, prm, cap, idx, w, cnt, ws) == 0
        got = idx[:int(cnt.item())].numpy()
    else:
        A, b = to_device(pr)
        ws = L.workspace(prm, n, d)
        idx = torch.empty(cap, dtype=torch.int64, device=DEV)
        w = torch.empty(cap, dtype=torch.float64, device=DEV)
        cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
        L.l1_coreset(A, b, prm, cap, idx, w, None, cnt, ws)
        assert L.l1s_status_read(ws) == 0
        got = idx[:int(cnt.item())].cpu().numpy()
    p, u = _oracle_decisions(X, r1, r2, m, seed)
    keep = np.zeros(n, bool)
    keep[got] = True
    amb = ambiguous(u, p, 1e-4)
    assert np.array_equal(keep[~amb], (u < p)[~amb]), int((keep != (u < p)).sum())
