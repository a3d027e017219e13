"""FCT2 (§3.2): Π1·X = (8/r1)·√(πt/(2s))·C·H̃·X with one SRHT block G per t rows, on the GPU
against the FP64 oracle through the C ABI.

Π1X element by element within 1e-5 of the sum of |contributing terms| (the FP32 bar of the
other transforms), for FP32 and BF16 storage, ragged row counts, block offsets, the default
and explicit numbers of kept rows, and widths of X that take one to three column slices of
the slow transform; the one-call pass with FCT2 as Π1 against the oracle's keep decisions.
"""
import math

import numpy as np
import pytest
import torch

import paper_1207_4684_gb300 as L
from gpu_util import DEV, PIX_REL, ambiguous, host_x, problem, to_device
from oracle import condition, fct2, leverage, rng, sampling
from synth import r1_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1207_4684_gb300 import build

    build.build()
    L.load()
    torch.cuda.set_device(0)


def default_rows(d, t):
    return int(min(t, max(1, math.ceil(2 * d * math.log(d))))) if d > 1 else 1


@pytest.mark.parametrize("n,d,t,sf,r1,dtype,offset", [
    (5000, 4, 32, 12, 45, "f32", 0),
    (70001, 16, 512, 0, 355, "f32", 0),            # default rows: ⌈2·16·ln 16⌉ = 89
    (20000, 8, 128, 34, 134, "bf16", 128 * 7),
    (3001, 40, 1024, 17, 1181, "f32", 0),          # three slices of the slow transform
    (1, 3, 16, 5, 7, "f32", 0),
    (9000, 16, 4096, 200, 355, "f32", 4096),       # one partial block, two passes of outputs
])
def test_fct2_embed_parity(n, d, t, sf, r1, dtype, offset):
    pr = problem(n, d, seed=n % 89 + d, dtype=dtype)
    A, b = to_device(pr)
    prm = L.make_params(t, r1, 16, 100.0, seed=6, problem_id=3, global_row_offset=offset, transform=2,
                        fjlt_rows=sf)
    ws = L.workspace(prm, n, d, L.BF16 if dtype == "bf16" else L.F32)
    pix = torch.empty((r1, d + 1), dtype=torch.float32, device=DEV)
    L.l1s_status_reset(ws)
    L.fct_embed(A, b, prm, pix, ws)
    assert L.l1s_status_read(ws) == 0
    got = pix.cpu().double().numpy()
    ref, tsum = fct2.fct2_embed(host_x(pr), t, sf or default_rows(d, t), r1, seed=6, problem_id=3, row_offset=offset)
    err = np.abs(got - ref)
    ratio = float((err / np.maximum(tsum, 1e-300)).max())
    assert np.all(err <= PIX_REL * tsum), f"worst |GPU − oracle| / Σ|terms| = {ratio:.3e}"


def test_fct2_rejects_bad_rows():
    prm = L.make_params(64, 45, 16, 100.0, transform=2, fjlt_rows=65)
    with pytest.raises(L.L1SError):
        L.l1s_workspace_size(prm, 1000, 4)


def test_fct2_coreset_matches_the_oracle():
    """Steps 1-7 with FCT2 as Π1."""
    n, d, r2, m, seed, t, sf = 200003, 16, 16, 3000.0, 8, 512, 89
    pr = problem(n, d, seed=23)
    X = host_x(pr)
    r1 = r1_for(d)
    prm = L.make_params(t, r1, r2, m, seed=seed, transform=2, fjlt_rows=sf)
    cap = int(2 * m) + 64
    A, b = to_device(pr)
    ws = L.workspace(prm, n, d)
    idx = torch.empty(cap, dtype=torch.int64, device=DEV)
    w = torch.empty(cap, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    L.l1_coreset(A, b, prm, cap, idx, w, None, cnt, ws)
    assert L.l1s_status_read(ws) == 0
    got = idx[:int(cnt.item())].cpu().numpy()
    pix, _ = fct2.fct2_embed(X, t, sf, r1, seed=seed)
    _, rm = condition.qr_positive(pix)
    M = condition.m_matrix(rm, rng.pi2_matrix(seed, 0, d + 1, r2))
    lam = leverage.lambda_estimates(X, M)
    p, _, _ = sampling.probabilities(lam, m)
    u = rng.sample_uniforms(seed, 0, np.arange(n))
    keep = np.zeros(n, bool)
    keep[got] = True
    amb = ambiguous(u, p, 1e-4)
    assert np.array_equal(keep[~amb], (u < p)[~amb]), int((keep != (u < p)).sum())
