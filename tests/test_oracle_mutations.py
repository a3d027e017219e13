"""Plant plausible mistakes in the FP64 oracle and check that a pin catches each.

Every mutation is applied to the oracle on the CPU with monkeypatch; the test
passes only if the named pin check raises AssertionError on the mutated
oracle.  This shows the pins in pins.py are not vacuous.
"""
import numpy as np
import pytest

import pins
from oracle import condition, fct, fct2, leverage, pipeline, quality, rng, sampling, sct, separable, solve

ORIG_EMBED = fct.fct1_embed
ORIG_HAD = fct.sylvester_hadamard
ORIG_CAUCHY = rng.cauchy_from_k
ORIG_QR = condition.qr_positive
ORIG_M = condition.m_matrix
ORIG_LAMBDA = leverage.lambda_estimates
ORIG_PROB = sampling.probabilities
ORIG_BERN = sampling.bernoulli_sample
ORIG_LP = solve.lad_lp
ORIG_FORMX = pipeline.form_x
ORIG_FORM_X_MULTI = pipeline.form_x_multi
ORIG_REPLACE = sampling.sample_with_replacement
ORIG_GAUSS = rng.pi2_gaussian_matrix
ORIG_SCALED = sampling.probabilities_scaled
ORIG_SCT = sct.sct_embed
ORIG_SCT_MATRIX = rng.sct_matrix
ORIG_FJLT_DRAWS = rng.fjlt_draws
ORIG_FCT2_SCALE = fct2.fct2_scale
ORIG_FCT2 = fct2.fct2_embed
ORIG_MINBOX = quality.min_l1_on_unit_box
ORIG_WOBJ = solve.weighted_objective


def embed_offset_ignored(X, s, r1, seed=0, problem_id=0, row_offset=0, sign_flip=True, draws=None):
    """FCT1 with the rows' variates drawn from local row ids (the global offset dropped)."""
    return ORIG_EMBED(X, s, r1, seed, problem_id, 0, sign_flip, draws)


def embed_ragged_tail_dropped(X, s, r1, seed=0, problem_id=0, row_offset=0, sign_flip=True, draws=None):
    """FCT1 that drops the last, partial block of s rows instead of padding it with zeros."""
    X = np.asarray(X)
    m = X.shape[0] - X.shape[0] % s
    return ORIG_EMBED(X[:m] if m else X, s, r1, seed, problem_id, row_offset, sign_flip, draws)


def replace_next_row(lam, m, u):
    """Each draw takes the row after the one whose interval of the running sum holds it."""
    idx, _, cdf = ORIG_REPLACE(lam, m, u)
    lam = np.asarray(lam, dtype=np.float64)
    idx = np.minimum(idx + 1, lam.size - 1)
    with np.errstate(divide="ignore"):
        return idx, cdf[-1] / (m * lam[idx]), cdf


def lambda_mean(X, M, chunk=1 << 20):
    """The mean of |X·M| over the r2 columns instead of their median."""
    return np.abs(np.asarray(X, dtype=np.float64) @ np.asarray(M, dtype=np.float64)).mean(axis=1)


def pi2_gaussian_entries(seed, problem_id, q, r2):
    """Π2 with standard Gaussian entries where FastCauchyRegression draws Cauchys."""
    return np.random.default_rng(seed + 7 * problem_id).standard_normal((q, r2))


def minbox_last_coordinate_only(U):
    """Only the faces z_{d−1} = ±1 of the unit box searched (the other d − 1 regressions skipped)."""
    U = np.asarray(U, dtype=np.float64)
    if U.shape[1] == 1:
        return ORIG_MINBOX(U)
    _, v = solve.lad_lp(U[:, :-1], -U[:, -1])
    return v


def kappa_alpha_row_max(U):
    """α as the largest row ℓ1 norm instead of the entrywise ℓ1 norm of U."""
    U = np.asarray(U, dtype=np.float64)
    return float(np.abs(U).sum(axis=1).max()) / quality.min_l1_on_unit_box(U)


def fjlt_no_signs(seed, problem_id, t, s):
    D, sel = ORIG_FJLT_DRAWS(seed, problem_id, t, s)
    return np.ones_like(D), sel


def fjlt_one_row(seed, problem_id, t, s):
    D, sel = ORIG_FJLT_DRAWS(seed, problem_id, t, s)
    return D, np.full_like(sel, sel[0])


def fct2_scale_no_sqrt(t, s, r1):
    return 8.0 / r1


def fct2_same_columns(X, t, s, r1, seed=0, problem_id=0, row_offset=0):
    import math
    X = np.asarray(X, dtype=np.float64)
    n, q = X.shape
    nb = -(-n // t)
    Xp = np.zeros((nb * t, q))
    Xp[:n] = X
    G = fct2.fjlt_matrix(seed, problem_id, t, s)
    Y = np.einsum("rt,btq->brq", G, Xp.reshape(nb, t, q)).reshape(nb * s, q)
    C = rng.sct_matrix(seed, problem_id, np.arange(nb * s) % s, r1)
    sc = fct2.fct2_scale(t, s, r1)
    return sc * (C @ Y), sc * (np.abs(C) @ np.abs(Y))


def canonical_mean(cols, b, d):
    cols = np.asarray(cols)
    m = np.array([np.mean(b[cols == j]) for j in range(d)])
    return m, m


def canonical_hi_low(cols, b, d):
    cols = np.asarray(cols)
    lo = np.empty(d)
    for j in range(d):
        v = np.sort(b[cols == j])
        lo[j] = v[(v.size + 1) // 2 - 1]
    return lo, lo


def _draws_of(X, s, r1, seed, problem_id, row_offset, draws):
    if draws is not None:
        return dict(draws)
    n_pad = fct.padded_rows(X.shape[0], s)
    return rng.fct_draws(seed, problem_id, row_offset + np.arange(n_pad), r1)


def embed_no_identity(X, s, r1, seed=0, problem_id=0, row_offset=0, sign_flip=True, draws=None):
    dr = _draws_of(X, s, r1, seed, problem_id, row_offset, draws)
    dr["cauchy_i"] = np.zeros_like(dr["cauchy_i"])
    return ORIG_EMBED(X, s, r1, seed, problem_id, row_offset, sign_flip, dr)


def embed_no_hadamard(X, s, r1, seed=0, problem_id=0, row_offset=0, sign_flip=True, draws=None):
    dr = _draws_of(X, s, r1, seed, problem_id, row_offset, draws)
    dr["cauchy_h"] = np.zeros_like(dr["cauchy_h"])
    return ORIG_EMBED(X, s, r1, seed, problem_id, row_offset, sign_flip, dr)


def embed_factor2(*a, **k):
    p, t = ORIG_EMBED(*a, **k)
    return p / 2, t / 2


def embed_swapped_halves(X, s, r1, seed=0, problem_id=0, row_offset=0, sign_flip=True, draws=None):
    dr = _draws_of(X, s, r1, seed, problem_id, row_offset, draws)
    dr["hash_h"], dr["hash_i"] = dr["hash_i"], dr["hash_h"]
    return ORIG_EMBED(X, s, r1, seed, problem_id, row_offset, sign_flip, dr)


def embed_sign_ignored(X, s, r1, seed=0, problem_id=0, row_offset=0, sign_flip=True, draws=None):
    return ORIG_EMBED(X, s, r1, seed, problem_id, row_offset, False, draws)


def embed_abs_terms_wrong(*a, **k):
    p, t = ORIG_EMBED(*a, **k)
    return p, np.abs(p)


def had_unnormalized_sign(s):
    h = np.ones((1, 1))
    while h.shape[0] < s:
        h = np.block([[h, h], [-h, h]])
    return h


def had_scaled(s):
    return ORIG_HAD(s) * np.sqrt(s)


def cauchy_neg(k):
    return -ORIG_CAUCHY(k)


def cauchy_offset(k):
    k = np.asarray(k, dtype=np.int64)
    u = k.astype(np.float64) * 2.0 ** -24
    return np.tan(np.pi * (u - 0.5))


def qr_no_signfix(pix):
    return np.linalg.qr(np.asarray(pix, dtype=np.float64), mode="reduced")


def qr_transposed(pix):
    q, r = ORIG_QR(pix)
    return q, r.T


def m_times_r(r_mat, pi2):
    return r_mat @ pi2


def lambda_upper_median(X, M, chunk=1 << 20):
    lam = np.abs(np.asarray(X, dtype=np.float64) @ M)
    return np.sort(lam, axis=1)[:, M.shape[1] // 2]


def lambda_no_rinv(X, M, chunk=1 << 20):
    return ORIG_LAMBDA(X, M * np.linspace(0.2, 5.0, M.shape[0])[:, None])


def prob_no_cap(lam, coreset, total=None):
    p, tau, tot = ORIG_PROB(lam, coreset, total)
    lam = np.asarray(lam, dtype=np.float64)
    return tau * lam, tau, tot


def bern_weights_p(p, u):
    idx, w = ORIG_BERN(p, u)
    return idx, 1.0 / w


def lp_unweighted(A, b, w=None):
    return ORIG_LP(A, b, None)


def formx_multi_plus_b(A, B):
    return ORIG_FORM_X_MULTI(A, -np.asarray(B, dtype=np.float64))


def replace_weight_mp(lam, m, u):
    idx, w, cdf = ORIG_REPLACE(lam, m, u)
    return idx, 1.0 / w, cdf


def replace_unscaled_target(lam, m, u):
    lam = np.asarray(lam, dtype=np.float64)
    cdf = np.cumsum(lam)
    idx = np.minimum(np.searchsorted(cdf, np.asarray(u)[:m], side="right"), lam.size - 1)
    return idx, cdf[-1] / (m * np.maximum(lam[idx], 1e-300)), cdf


def formx_plus_b(A, b):
    return np.concatenate([np.asarray(A, float), np.asarray(b, float)[:, None]], axis=1)


def gauss_var2(seed, problem_id, q, r2):
    return ORIG_GAUSS(seed, problem_id, q, r2) * np.sqrt(2.0)


def gauss_pair_copy(seed, problem_id, q, r2):
    z = ORIG_GAUSS(seed, problem_id, q, r2).ravel().copy()
    z[1::2] = z[0::2][: z[1::2].size]
    return z.reshape(q, r2)


def scaled_no_cap(lam, scale):
    return float(scale) * np.asarray(lam, dtype=np.float64)


def sct_scale_one_over_r1(*a, **k):
    p, t = ORIG_SCT(*a, **k)
    return p / 4, t / 4


def sct_group_ignored(seed, problem_id, rows, r1):
    c = ORIG_SCT_MATRIX(seed, problem_id, rows, 4)
    return np.tile(c, ((r1 + 3) // 4, 1))[:r1]


def sct_last_block_dropped(X, r1, seed=0, problem_id=0, row_offset=0, block=1 << 14):
    n = X.shape[0]
    keep = max(1, n - n // 3)
    return ORIG_SCT(X[:keep], r1, seed, problem_id, row_offset, block)


MUTATIONS = [
    ("identity half dropped", fct, "fct1_embed", embed_no_identity, pins.check_fct_dense),
    ("row offset ignored", fct, "fct1_embed", embed_offset_ignored, pins.check_fct_row_offset),
    ("ragged tail dropped", fct, "fct1_embed", embed_ragged_tail_dropped, pins.check_fct_dense),
    ("slow transform scaled by 1/r1", sct, "sct_embed", sct_scale_one_over_r1, pins.check_sct_stability),
    ("slow transform: one call for all groups", rng, "sct_matrix", sct_group_ignored, pins.check_sct_draws),
    ("slow transform: last rows dropped", sct, "sct_embed", sct_last_block_dropped, pins.check_sct_stability),
    ("Hadamard half dropped", fct, "fct1_embed", embed_no_hadamard, pins.check_fct_dense),
    ("factor 4 → 2", fct, "fct1_embed", embed_factor2, pins.check_fct_blocks),
    ("halves swapped", fct, "fct1_embed", embed_swapped_halves, pins.check_fct_dense),
    ("sign flip ignored", fct, "fct1_embed", embed_sign_ignored, pins.check_fct_dense),
    ("Σ|terms| wrong", fct, "fct1_embed", embed_abs_terms_wrong, pins.check_fct_mass),
    ("Hadamard recursion sign", fct, "sylvester_hadamard", had_unnormalized_sign, pins.check_hadamard_closed_form),
    ("Hadamard not normalized", fct, "sylvester_hadamard", had_scaled, pins.check_fct_blocks),
    ("Cauchy sign", rng, "cauchy_from_k", cauchy_neg, pins.check_cauchy_quantiles),
    ("Cauchy cell edge", rng, "cauchy_from_k", cauchy_offset, pins.check_cauchy_quantiles),
    ("R sign not fixed", condition, "qr_positive", qr_no_signfix, pins.check_qr),
    ("R transposed", condition, "qr_positive", qr_transposed, pins.check_qr),
    ("R·Π2 for R⁻¹·Π2", condition, "m_matrix", m_times_r, pins.check_qr),
    ("upper median", leverage, "lambda_estimates", lambda_upper_median, pins.check_lambda_distribution),
    ("mean for median", leverage, "lambda_estimates", lambda_mean, pins.check_lambda_distribution),
    ("Gaussian Π2 in FastCauchyRegression", rng, "pi2_matrix", pi2_gaussian_entries, pins.check_lambda_distribution),
    ("R⁻¹ distorted", condition, "m_matrix", lambda r, p: ORIG_M(r, p) * np.linspace(0.2, 5, r.shape[0])[:, None],
     pins.check_lambda_distribution),
    ("p̂ not capped at 1", sampling, "probabilities", prob_no_cap, pins.check_sampling),
    ("weight p̂ for 1/p̂", sampling, "bernoulli_sample", bern_weights_p, pins.check_sampling),
    ("LP ignores weights", solve, "lad_lp", lp_unweighted, pins.check_solver),
    ("objective ignores weights", solve, "weighted_objective", lambda A, b, w, x: ORIG_WOBJ(A, b, None, x),
     pins.check_solver),
    ("X = [A, +b]", pipeline, "form_x", formx_plus_b, pins.check_solver),
    ("Gaussian Π2 variance 2", rng, "pi2_gaussian_matrix", gauss_var2, pins.check_gaussian_pi2),
    ("Box–Muller pair copied", rng, "pi2_gaussian_matrix", gauss_pair_copy, pins.check_gaussian_pi2),
    ("upper median (Gaussian)", leverage, "lambda_estimates", lambda_upper_median,
     pins.check_gaussian_lambda_distribution),
    ("Gaussian Π2 variance 2 in λ̂", rng, "pi2_gaussian_matrix", gauss_var2, pins.check_gaussian_lambda_distribution),
    ("scaled p̂ not capped", sampling, "probabilities_scaled", scaled_no_cap, pins.check_scaled_probabilities),
    ("X = [A, +B] (multiple)", pipeline, "form_x_multi", formx_multi_plus_b, pins.check_multiple_regression),
    ("with-replacement draw one row late", sampling, "sample_with_replacement", replace_next_row,
     pins.check_with_replacement),
    ("with-replacement weight m·p̂", sampling, "sample_with_replacement", replace_weight_mp,
     pins.check_with_replacement),
    ("with-replacement target u, not u·Σλ", sampling, "sample_with_replacement", replace_unscaled_target,
     pins.check_with_replacement),
    ("Philox Weyl constant off by one", rng, "PHILOX_W0", np.uint64(0x9E3779B8), pins.check_philox_key_schedule),
    ("FJLT signs dropped", rng, "fjlt_draws", fjlt_no_signs, pins.check_fjlt_spread),
    ("FJLT one sampled row repeated", rng, "fjlt_draws", fjlt_one_row, pins.check_fjlt_isometry),
    ("FCT2 scale without √(πt/2s)", fct2, "fct2_scale", fct2_scale_no_sqrt, pins.check_fct2_stability),
    ("FCT2 blocks share C's columns", fct2, "fct2_embed", fct2_same_columns, pins.check_fct2_dense),
    ("κ̄₁: one face of the unit box searched", quality, "min_l1_on_unit_box", minbox_last_coordinate_only,
     pins.check_kappa_bar),
    ("κ̄₁: α as the largest row norm", quality, "kappa_bar_1", kappa_alpha_row_max, pins.check_kappa_bar),
    ("separable optimum: mean for median", separable, "canonical_optimum", canonical_mean,
     pins.check_canonical_optimum),
    ("separable optimum: upper median = lower", separable, "canonical_optimum", canonical_hi_low,
     pins.check_canonical_optimum),
]


@pytest.mark.parametrize("name,mod,attr,bad,check", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_mutation(monkeypatch, name, mod, attr, bad, check):
    monkeypatch.setattr(mod, attr, bad)
    with pytest.raises(AssertionError):
        check()
