"""l1_lambda_noalloc: the λ pass for callers that cannot allocate device memory.

Such callers cannot hand the library a workspace (their host program owns all
device memory, or a running loop must not pay cudaMalloc's device-wide
synchronisation), so this entry point keeps its scratch in a library-owned
device array.  Its results must equal those of l1_lambda, which takes a
workspace, on two calls in a row with different shapes (the shared array keeps
the previous call's contents).  Collected last so that a stop-at-first-failure
run has already run every other test.
"""
import math

import numpy as np
import pytest
import torch

import paper_1207_4684_gb300 as L
from gpu_util import DEV, fsum, host_x, lambda_tol, lambda_tol_tc, problem, tensor_core_form, to_device
from oracle import condition, leverage, rng

pytestmark = pytest.mark.gpu


def _case(n, d, r2, dtype, seed):
    pr = problem(n, d, seed=seed, dtype=dtype)
    A, b = to_device(pr)
    g = np.random.default_rng(seed)
    _, rm = condition.qr_positive(g.standard_normal((4 * (d + 1), d + 1)))
    M = np.ascontiguousarray(condition.m_matrix(rm, rng.pi2_matrix(seed, 0, d + 1, r2)))
    return pr, A, b, M


def test_lambda_noalloc_matches_workspace_entry_point():
    from paper_1207_4684_gb300 import build

    build.build()
    L.load()
    torch.cuda.set_device(0)
    for n, d, r2, dtype, seed in ((100003, 16, 16, "f32", 1), (50000, 32, 32, "bf16", 2)):
        pr, A, b, M = _case(n, d, r2, dtype, seed)
        Md = torch.from_numpy(M).to(DEV)
        prm = L.make_params(64, max(d + 1, 10), r2, 100.0)
        ws = L.workspace(prm, n, d, L.BF16 if dtype == "bf16" else L.F32)
        lam_ws = torch.empty(n, dtype=torch.float32, device=DEV)
        tot_ws = torch.zeros(1, dtype=torch.float64, device=DEV)
        L.l1_lambda(A, b, Md, prm, lam_ws, tot_ws, ws)
        lam = torch.full((n,), float("nan"), dtype=torch.float32, device=DEV)
        tot = torch.zeros(1, dtype=torch.float64, device=DEV)
        L.l1_lambda_noalloc(A, b, Md, prm, lam, tot)
        torch.cuda.synchronize()
        got = lam.cpu().double().numpy()
        want = lam_ws.cpu().double().numpy()
        X = host_x(pr)
        if tensor_core_form(dtype, d, r2, None):
            Mref = leverage.mixed_precision_m(M)
            tol = lambda_tol_tc(X, Mref)
        else:
            Mref, tol = M, lambda_tol(X, M)
        assert np.all(np.abs(got - want) <= tol), "λ differs from l1_lambda"
        assert math.isclose(tot.item(), tot_ws.item(), rel_tol=1e-12)
        assert math.isclose(tot.item(), fsum(got), rel_tol=1e-12)
        ref = leverage.lambda_estimates(X, Mref)
        assert np.all(np.abs(got - ref) <= tol)


def test_lambda_noalloc_rejects_sizes_beyond_its_scratch():
    L.load()
    n, r2 = 400000, 64                  # enough rows for the full count of Σλ partial sums (8 per SM)
    lam = torch.empty(n, dtype=torch.float32, device=DEV)
    tot = torch.zeros(1, dtype=torch.float64, device=DEV)
    b = torch.zeros(n, dtype=torch.float32, device=DEV)
    for d, fits in ((64, True), (128, False)):     # q·r2 = 4160 fits the 40 KiB scratch, 8256 does not
        prm = L.make_params(64, 200, r2, 100.0)
        A = torch.ones((n, d), dtype=torch.float32, device=DEV)
        M = torch.ones((d + 1, r2), dtype=torch.float64, device=DEV)
        if fits:
            L.l1_lambda_noalloc(A, b, M, prm, lam, tot)
            torch.cuda.synchronize()
            assert torch.all(lam == float(d)).item()
        else:
            with pytest.raises(L.L1SError) as e:
                L.l1_lambda_noalloc(A, b, M, prm, lam, tot)
            assert e.value.code == 1 and "scratch" in str(e.value)
