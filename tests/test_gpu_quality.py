"""The ℓ1 basis U = X·R⁻¹ (§4.1) and the conditioning metric κ̄₁ of §6.1 on the GPU.

l1_basis against the FP64 oracle's U = X·R⁻¹ (same R) element by element; κ̄₁ of a GPU
basis against the oracle's κ̄₁ of the same U (exact LPs); and, as a statistical check
rather than parity, the quartiles of κ̄₁ for FCT1 and the slow Cauchy transform on the test
matrices A1 and A2 of §6.1 against the published quartiles (Tables 2 and 3).
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import paper_1207_4684_gb300 as L
from gpu_util import DEV, fsum, host_x, problem, to_device
from oracle import quality
from synth import kappa_test_matrix

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "kappa_bar_quartiles.json")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1207_4684_gb300 import build

    build.build()
    L.load()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("n,d,dtype", [(50001, 4, "f32"), (20000, 16, "f32"), (9000, 33, "bf16")])
def test_l1_basis_matches_the_oracle(n, d, dtype):
    pr = problem(n, d, seed=d, dtype=dtype)
    A, b = to_device(pr)
    X = host_x(pr)
    g = np.random.default_rng(d)
    R = np.triu(g.standard_normal((d + 1, d + 1)), 1) / np.sqrt(d + 1) + np.diag(g.uniform(1.0, 3.0, d + 1))
    U = torch.empty((n, d + 1), dtype=torch.float64, device=DEV)
    rn = torch.empty(n, dtype=torch.float64, device=DEV)
    tot = torch.empty(1, dtype=torch.float64, device=DEV)
    L.l1_basis(A, b, torch.from_numpy(R).to(DEV), U, rn, tot)
    ref = np.linalg.solve(R.T, X.T).T                  # U·R = X
    got = U.cpu().numpy()
    # forward substitution: each computed row solves a perturbed system U_i·(R + δR) = X_i with
    # |δR| ≤ q·u·|R|, so |δU_i| ≤ q·u·|U_i|·|R|·|R⁻¹| to first order (the same bound for the reference)
    rinv = np.abs(np.linalg.inv(R))
    tol = 4 * (d + 1) * 2.0 ** -53 * (np.abs(ref) @ np.abs(R) @ rinv)
    assert np.all(np.abs(got - ref) <= np.maximum(tol, 1e-300)), float((np.abs(got - ref) / tol).max())
    assert np.allclose(rn.cpu().numpy(), np.abs(got).sum(axis=1), rtol=1e-14, atol=0)
    assert math.isclose(tot.item(), fsum(rn.cpu().numpy()), rel_tol=1e-12)


@pytest.mark.parametrize("kind,transform", [("A1", 0), ("A2", 0), ("A1", 1)])
def test_kappa_bar_matches_the_oracle_on_the_same_basis(kind, transform):
    from paper_1207_4684_gb300 import validation

    n, d = 1 << 12, 4
    A = torch.from_numpy(kappa_test_matrix(kind, n, d, seed=3)).to(DEV)
    r1 = math.ceil(2 * d * math.log(d))
    out = validation.kappa_bar(A, r1, 16, seed=7, transform=transform)
    # A1 is ill-conditioned enough (κ₂ ~ 1e5) for the FP32-resolution rank test to flag it; R is still formed
    assert (out["status"] & ~L.flag(4)) == 0, out["status"]
    Rh = out["R"].cpu().numpy()
    Ah = A.cpu().double().numpy()
    Ah[:, -1] = -Ah[:, -1]                             # X = A·diag(1, …, 1, −1), as the library sees it
    U = np.linalg.solve(Rh.T, Ah.T).T
    ref = quality.kappa_bar_1(U)
    assert abs(out["kappa_bar"] - ref) <= 1e-6 * ref, (out["kappa_bar"], ref)


@pytest.mark.parametrize("kind", ["A1", "A2"])
def test_fct2_kappa_bar_matches_the_oracle_on_the_same_basis(kind):
    from paper_1207_4684_gb300 import validation

    n, d = 1 << 12, 4
    A = torch.from_numpy(kappa_test_matrix(kind, n, d, seed=5)).to(DEV)
    r1 = math.ceil(2 * d * math.log(d))
    out = validation.kappa_bar(A, r1, 32, seed=9, transform=2, fjlt_rows=math.ceil(2 * d * math.log(d)))
    assert (out["status"] & ~L.flag(4)) == 0, out["status"]
    Rh = out["R"].cpu().numpy()
    Ah = A.cpu().double().numpy()
    Ah[:, -1] = -Ah[:, -1]
    U = np.linalg.solve(Rh.T, Ah.T).T
    ref = quality.kappa_bar_1(U)
    assert abs(out["kappa_bar"] - ref) <= 1e-6 * ref, (out["kappa_bar"], ref)


@pytest.mark.parametrize("size,n,d", [("2^18x4", 1 << 18, 4)])
def test_fct2_kappa_bar_quartiles_against_the_paper(size, n, d):
    """FCT2 with the experiments' settings read with FCT1's and FCT2's labels swapped (§6.1):
    r1 = ⌈2d ln d⌉, s = ⌈2d ln d⌉ rows of G kept per block of t = 2^⌈log₂ 2d²⌉ rows: the median
    of κ̄₁ over 9 runs within a factor 3 of the published interquartile range, far below κ̄₁(A)."""
    from paper_1207_4684_gb300 import validation

    ref = json.load(open(GOLDEN))[size]
    r1 = math.ceil(2 * d * math.log(d))
    sf = math.ceil(2 * d * math.log(d))
    t = 1 << math.ceil(math.log2(2 * d * d))
    for kind in ("A1", "A2"):
        A = torch.from_numpy(kappa_test_matrix(kind, n, d, seed=11)).to(DEV)
        vals = [validation.kappa_bar(A, r1, t, seed=200 + k, transform=2, fjlt_rows=sf)["kappa_bar"]
                for k in range(9)]
        med = float(np.median(vals))
        q1, q3 = ref["FCT2"][kind]
        assert q1 / 3 <= med <= 3 * q3, (kind, med, q1, q3)
        assert med < ref["kappa_bar_A"][kind] / 100, (kind, med)


@pytest.mark.parametrize("size,n,d", [("2^18x4", 1 << 18, 4)])
def test_kappa_bar_quartiles_against_the_paper(size, n, d):
    """FCT1 (r1 = ⌈2d ln d⌉, s = 2^⌈log₂(2d ln d)⌉) and the slow transform on A1 and A2: the
    median of κ̄₁ over 9 runs lies within a factor 3 of the published interquartile range, and
    conditioning lowers κ̄₁ far below κ̄₁(A)."""
    from paper_1207_4684_gb300 import validation

    ref = json.load(open(GOLDEN))[size]
    r1 = math.ceil(2 * d * math.log(d))
    s = 1 << math.ceil(math.log2(2 * d * math.log(d)))
    for kind in ("A1", "A2"):
        A = torch.from_numpy(kappa_test_matrix(kind, n, d, seed=11)).to(DEV)
        for name, transform in (("FCT1", 0), ("CT", 1)):
            vals = [validation.kappa_bar(A, r1, s, seed=100 + k, transform=transform)["kappa_bar"] for k in range(9)]
            med = float(np.median(vals))
            q1, q3 = ref[name][kind]
            assert q1 / 3 <= med <= 3 * q3, (kind, name, med, q1, q3)
            assert med < ref["kappa_bar_A"][kind] / 100, (kind, name, med)
