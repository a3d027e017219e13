"""Row shards of one problem on one GPU through the library (shard.ShardPass).

Two shards (rows cut at a multiple of s, the second with a ragged tail) each embed their
rows with their global row offset; their Π1X are summed, both condition the sum, each
computes λ on its rows, their Σλ are summed, and each samples with the summed Σλ
(l1_sample_lambda).  Bars: the summed Π1X matches the unsharded l1 pass's within the FP32
tolerance of Π1X; the union of the shards' kept rows equals the unsharded coreset
(l1_coreset) except for rows whose uniform lies within 1e-4 relative of p̂ (where FP32
rounding of the summed Π1X may decide); weights of common rows agree within 1e-4
relative; coreset rows are the rows of X.  The shards run one after the other on the
device, with the sums formed between their phases.
"""
import numpy as np
import pytest
import torch

import paper_1207_4684_gb300 as L
from gpu_util import DEV, check_pix, host_x, problem, to_device
from oracle import rng
from paper_1207_4684_gb300.shard import ShardPass, shard_rows
from synth import r1_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1207_4684_gb300 import build

    build.build()
    L.load()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("n,d,dtype,s", [(90037, 8, "f32", 64), (70001, 24, "bf16", 256)])
def test_two_shards_equal_unsharded(n, d, dtype, s):
    pr = problem(n, d, seed=12, dtype=dtype)
    A, b = to_device(pr)
    m, cap = 1500.0, 4000
    prm = L.make_params(s, r1_for(d), 16, m, seed=6)
    dt = L.BF16 if dtype == "bf16" else L.F32
    # unsharded pass
    ws = L.workspace(prm, n, d, dt)
    idx = torch.empty(cap, dtype=torch.int64, device=DEV)
    w = torch.empty(cap, dtype=torch.float64, device=DEV)
    core = torch.empty((cap, d + 1), dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    L.l1_coreset(A, b, prm, cap, idx, w, core, cnt, ws)
    assert L.l1s_status_read(ws) == 0
    c_ref = int(cnt.item())
    ref_idx = idx[:c_ref].cpu().numpy()
    ref_w = w[:c_ref].cpu().numpy()
    # two shards
    passes = []
    for r in range(2):
        lo, hi = shard_rows(n, s, 2, r)
        wsr = L.workspace(prm, hi - lo, d, dt)
        L.l1s_status_reset(wsr)
        passes.append(ShardPass(A[lo:hi], b[lo:hi].contiguous(), lo, prm, cap, wsr))
    pix = sum(sp.embed() for sp in passes)
    X = host_x(pr)
    check_pix(pix.cpu().double().numpy(), X, prm)
    tot = sum(sp.condition_and_lambda(pix) for sp in passes)
    outs = [sp.sample(tot) for sp in passes]
    for sp in passes:
        assert L.l1s_status_read(sp.ws) == 0
    got_idx = np.concatenate([o[0][: int(o[3].item())].cpu().numpy() for o in outs])
    got_w = np.concatenate([o[1][: int(o[3].item())].cpu().numpy() for o in outs])
    got_core = np.concatenate([o[2][: int(o[3].item())].cpu().numpy() for o in outs])
    assert np.all(np.diff(got_idx) > 0)
    assert np.array_equal(got_core, X[got_idx])
    # λ of the unsharded pass for the ambiguity band (an independent l1_lambda call)
    lam = torch.cat([sp.lam for sp in passes]).cpu().numpy().astype(np.float64)
    p = np.minimum(1.0, m / float(tot.item()) * lam)
    u = rng.sample_uniforms(6, 0, np.arange(n))
    diff = np.setxor1d(got_idx, ref_idx)
    assert np.all(np.abs(u[diff] - p[diff]) <= 1e-4 * p[diff]), diff
    assert diff.size <= 3
    common, ia, ib = np.intersect1d(got_idx, ref_idx, return_indices=True)
    assert np.allclose(got_w[ia], ref_w[ib], rtol=1e-4, atol=0)
    assert common.size >= c_ref - 3


@pytest.mark.parametrize("transform,t,sf", [(1, 1, 0), (2, 512, 89)])
def test_two_shards_other_transforms(transform, t, sf):
    """The slow transform (draws keyed by global row ids) and FCT2 (blocks of t rows cut at
    shard boundaries, H̃X rows keyed by global block): the shards' summed Π1X matches the
    unsharded pass's within the FP32 rounding of its terms, and their kept rows are the
    unsharded coreset's outside the 1e-4 band."""
    n, d, m, cap = 60011, 16, 1200.0, 3000
    pr = problem(n, d, seed=31)
    A, b = to_device(pr)
    prm = L.make_params(t, r1_for(d), 16, m, seed=9, transform=transform, fjlt_rows=sf)
    ws = L.workspace(prm, n, d)
    pix_full = torch.empty((prm.r1, d + 1), dtype=torch.float32, device=DEV)
    L.l1s_status_reset(ws)
    L.fct_embed(A, b, prm, pix_full, ws)
    idx = torch.empty(cap, dtype=torch.int64, device=DEV)
    w = torch.empty(cap, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    L.l1_coreset(A, b, prm, cap, idx, w, None, cnt, ws)
    assert L.l1s_status_read(ws) == 0
    ref_idx = idx[: int(cnt.item())].cpu().numpy()
    passes = []
    for r in range(2):
        lo, hi = shard_rows(n, t if transform == 2 else 64, 2, r)
        wsr = L.workspace(prm, hi - lo, d)
        L.l1s_status_reset(wsr)
        passes.append(ShardPass(A[lo:hi], b[lo:hi].contiguous(), lo, prm, cap, wsr))
    pix = sum(sp.embed() for sp in passes)
    scale = pix_full.abs().max().item()
    assert torch.allclose(pix, pix_full, rtol=1e-4, atol=1e-5 * scale), float((pix - pix_full).abs().max())
    tot = sum(sp.condition_and_lambda(pix) for sp in passes)
    outs = [sp.sample(tot) for sp in passes]
    for sp in passes:
        assert L.l1s_status_read(sp.ws) == 0
    got = np.concatenate([o[0][: int(o[3].item())].cpu().numpy() for o in outs])
    lam = torch.cat([sp.lam for sp in passes]).cpu().numpy().astype(np.float64)
    p = np.minimum(1.0, m / float(tot.item()) * lam)
    u = rng.sample_uniforms(9, 0, np.arange(n))
    diff = np.setxor1d(got, ref_idx)
    assert np.all(np.abs(u[diff] - p[diff]) <= 1e-4 * p[diff]), diff
    assert diff.size <= 3
