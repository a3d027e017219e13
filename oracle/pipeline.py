"""FastCauchyRegression end to end, FP64 oracle side (Figure 2, steps 1-8).

Test infrastructure: only the tests, the smoke check and the bench's CPU
baseline use this module; the CUDA path shares no code with it.

Each step is one call into the modules of this package, in the figure's
order, and every intermediate is returned so that tests can compare the CUDA
path with it step by step.
"""
from __future__ import annotations

import time

import numpy as np

from . import condition, fct, leverage, rng, sampling, solve


def form_x(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """X = [A, −b] ∈ R^{n×(d+1)} in FP64 (Figure 2, step 1, k = 1)."""
    A = np.asarray(A, dtype=np.float64)
    return np.concatenate([A, -np.asarray(b, dtype=np.float64)[:, None]], axis=1)


def form_x_multi(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = [A, −B] ∈ R^{n×(d+k)} in FP64 (§4.2.1, multiple ℓ1 regression: Z = [W; I_k])."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    return np.concatenate([A, -B], axis=1)


def coreset_of_x(X: np.ndarray, s: int, r1: int, r2: int, coreset: float, seed: int = 0,
                 problem_id: int = 0, sign_flip: bool = True, variant: int = 0,
                 sample_scale: float = 0.0, timings: dict | None = None) -> dict:
    """Figure 2 steps 2-7 on a given X (any number of columns q): Π1X, its QR, M = R⁻¹Π2,
    λ, p̂ and the Bernoulli coreset, with every intermediate."""
    t = {} if timings is None else timings
    t0 = time.perf_counter()
    n, q = X.shape
    pix, tsum = fct.fct1_embed(X, s, r1, seed, problem_id, 0, sign_flip)     # step 2, Π1X
    t1 = time.perf_counter()
    _, r_mat = condition.qr_positive(pix)                                     # step 2, QR
    condition.check_rank(r_mat)
    pi2 = (rng.pi2_gaussian_matrix(seed, problem_id, q, r2) if variant == 1
           else rng.pi2_matrix(seed, problem_id, q, r2))                      # step 3
    m_mat = condition.m_matrix(r_mat, pi2)                                    # R⁻¹Π2
    t2 = time.perf_counter()
    lam = leverage.lambda_estimates(X, m_mat)                                 # steps 4-5
    t3 = time.perf_counter()
    if variant == 2:                                      # exactly m_s draws with replacement
        m = int(coreset)
        u = rng.replacement_uniforms(seed, problem_id, np.arange(m))
        idx, wts, cdf = sampling.sample_with_replacement(lam, m, u)
        total = float(cdf[-1])
        p_hat, tau = lam / total, 1.0 / total
    else:
        if variant == 1:
            p_hat, tau, total = sampling.probabilities_scaled(lam, sample_scale), sample_scale, None
        else:
            p_hat, tau, total = sampling.probabilities(lam, coreset)          # step 6
        u = rng.sample_uniforms(seed, problem_id, np.arange(n))
        idx, wts = sampling.bernoulli_sample(p_hat, u)                        # step 7
    t4 = time.perf_counter()
    t.update({"fct": t1 - t0, "condition": t2 - t1, "lambda": t3 - t2, "sample": t4 - t3})
    return {"X": X, "PiX": pix, "T": tsum, "R": r_mat, "Pi2": pi2, "M": m_mat,
            "lam": lam, "lam_total": total, "tau": tau, "p": p_hat, "u": u,
            "idx": idx, "w": wts}


def fast_cauchy_regression(A, b, s: int, r1: int, r2: int, coreset: float,
                           seed: int = 0, problem_id: int = 0, sign_flip: bool = True,
                           solve_lp: bool = True, timings: dict | None = None,
                           variant: int = 0, sample_scale: float = 0.0) -> dict:
    """All intermediates of Figure 2 for one problem (rows are numbered from 0).

    variant 1 is OptimizedFastCauchyRegression (Figure "mainOpt"): Π2 Gaussian and
    p̂ = min{1, sample_scale·λ̂} without the Σλ normalisation; variant 2 draws exactly
    m_s rows with replacement with p̂_i = λ_i/Σλ (the caption of Figure 2)."""
    t = {} if timings is None else timings
    X = form_x(A, b)                                                          # step 1
    out = coreset_of_x(X, s, r1, r2, coreset, seed, problem_id, sign_flip, variant, sample_scale, t)
    t4 = time.perf_counter()
    if solve_lp:                                                              # step 8
        idx, wts = out["idx"], out["w"]
        xs, fs = solve.lad_lp(X[idx, :-1], -X[idx, -1], wts)
        out["x_hat"] = xs
        out["coreset_objective"] = fs
        out["objective"] = solve.objective(X[:, :-1], -X[:, -1], xs)
    t["solve"] = time.perf_counter() - t4
    return out


def fast_cauchy_multiple_regression(A, B, s: int, r1: int, r2: int, coreset: float,
                                    seed: int = 0, problem_id: int = 0, sign_flip: bool = True,
                                    solve_lp: bool = True, variant: int = 0,
                                    sample_scale: float = 0.0) -> dict:
    """FastCauchyRegression(A, B) of §4.2.1: the same steps on X = [A, −B] (q = d + k
    columns), one coreset for all k right-hand sides, then k weighted ℓ1 problems
    min_w Σ_i w_i |A_i·w − B_ij| on it.  W is d × k (column j solves right-hand side j)."""
    A = np.asarray(A, dtype=np.float64)
    d = A.shape[1]
    X = form_x_multi(A, B)
    k = X.shape[1] - d
    out = coreset_of_x(X, s, r1, r2, coreset, seed, problem_id, sign_flip, variant, sample_scale)
    if solve_lp:
        idx, wts = out["idx"], out["w"]
        W = np.zeros((d, k))
        fc = np.zeros(k)
        f = np.zeros(k)
        for j in range(k):
            bj = -X[:, d + j]
            W[:, j], fc[j] = solve.lad_lp(X[idx, :d], bj[idx], wts)
            f[j] = solve.objective(X[:, :d], bj, W[:, j])
        out["W"] = W
        out["coreset_objectives"] = fc
        out["objectives"] = f
    return out
