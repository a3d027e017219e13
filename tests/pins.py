"""Checks that pin the FP64 oracle to facts outside itself.

Each check raises AssertionError when the oracle disagrees with what the
paper or the mathematics fixes: closed forms, invariants stated in the
paper's proofs, brute force on tiny inputs, and exact distributional
consequences of Cauchy 1-stability.  test_oracle_pins.py runs every check on
the oracle as written; test_oracle_mutations.py plants plausible mistakes in
the oracle and asserts that some check here catches each of them.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import stats

from oracle import condition, fct, fct2, leverage, pipeline, quality, rng, sampling, sct, separable, solve


# ----------------------------------------------------------------- Hadamard
def check_hadamard_closed_form(max_log2: int = 10) -> None:
    """Sylvester H_s has entries (−1)^{popcount(i AND j)} and H_s·H_s = s·I (§3.1)."""
    for lg in range(0, max_log2 + 1):
        s = 1 << lg
        h = fct.sylvester_hadamard(s)
        i = np.arange(s)
        par = np.vectorize(lambda v: bin(v).count("1") & 1)(i[:, None] & i[None, :])
        assert np.array_equal(h, np.where(par == 1, -1.0, 1.0)), f"H_{s} entries"
        assert np.array_equal(h @ h, s * np.eye(s)), f"H_{s}^2 != s I"


# ----------------------------------------------------------------- Cauchy
def check_cauchy_quantiles(step: int = 1) -> None:
    """c(k) is the standard Cauchy quantile at (k+½)·2^-24.

    Tail form: P(C > |c|) = atan(1/|c|)/π must equal min(u, 1−u), and the
    sign of c must be the sign of u − ½.  Also compared with tan(π(u−½)) away
    from the poles (a different formula).
    """
    k = np.arange(0, 1 << 24, step, dtype=np.int64)
    c = rng.cauchy_from_k(k)
    u = (k.astype(np.float64) + 0.5) * 2.0 ** -24
    tail = np.arctan2(1.0, np.abs(c)) / np.pi
    assert np.allclose(tail, np.minimum(u, 1.0 - u), rtol=1e-13, atol=0), "Cauchy tail"
    assert np.array_equal(np.sign(c), np.sign(u - 0.5)), "Cauchy sign"
    mid = np.abs(u - 0.5) < 0.4
    assert np.allclose(c[mid], np.tan(np.pi * (u[mid] - 0.5)), rtol=1e-12, atol=1e-15), "tan form"
    try:
        import mpmath
    except ImportError:
        return
    mpmath.mp.prec = 120
    for kk in (0, 1, 2, 1000, (1 << 23) - 2, (1 << 23) - 1, 1 << 23, (1 << 23) + 1, (1 << 24) - 2, (1 << 24) - 1,
               5_000_000, 12_345_678):
        exact = mpmath.tan(mpmath.pi * (mpmath.mpf(kk) + mpmath.mpf(0.5) - mpmath.mpf(2) ** 23) / mpmath.mpf(2) ** 24)
        got = float(rng.cauchy_from_k(np.array([kk]))[0])
        assert abs(got - float(exact)) <= 4e-16 * abs(float(exact)), f"relative accuracy at k={kk}"


def check_draw_statistics(n: int = 1 << 18, r1: int = 97, seed: int = 12345) -> None:
    """Uniform buckets, balanced signs, Cauchy scales and uniforms with the right laws."""
    d = rng.fct_draws(seed, 3, np.arange(n), r1)
    for key in ("hash_h", "hash_i"):
        cnt = np.bincount(d[key], minlength=r1)
        assert cnt.size == r1
        p = stats.chisquare(cnt).pvalue
        assert p > 1e-5, f"{key} not uniform (p={p})"
    joint = np.bincount(d["hash_h"] % 8 * 8 + d["hash_i"] % 8, minlength=64).reshape(8, 8)
    assert stats.chi2_contingency(joint).pvalue > 1e-5, "hash_h, hash_i dependent"
    plus = int((d["sigma"] > 0).sum())
    assert abs(plus - n / 2) < 5 * math.sqrt(n) / 2, "sign imbalance"
    for key in ("cauchy_h", "cauchy_i"):
        ks = stats.kstest(d[key], "cauchy")
        assert ks.pvalue > 1e-5, f"{key} not Cauchy (p={ks.pvalue})"
    sg = d["sigma"]
    assert abs(np.mean(sg * np.sign(d["cauchy_i"]))) < 5 / math.sqrt(n), "σ tied to C_I sign"
    u = rng.sample_uniforms(seed, 3, np.arange(n))
    assert np.all((u >= 0) & (u < 1))
    assert stats.kstest(u, "uniform").pvalue > 1e-5, "sampling uniforms"
    assert abs(np.corrcoef(u[0::2], u[1::2])[0, 1]) < 5 / math.sqrt(n / 2), "even/odd rows correlated"
    pi2 = rng.pi2_matrix(seed, 3, 257, 64)
    assert stats.kstest(pi2.ravel(), "cauchy").pvalue > 1e-5, "Π2 entries"
    a = rng.fct_draws(seed, 4, np.arange(n), r1)["cauchy_h"]
    assert stats.kstest(a - 0.0, "cauchy").pvalue > 1e-5
    assert not np.array_equal(a, d["cauchy_h"]), "problem id ignored"


# ----------------------------------------------------------------- FCT1
def check_fct_dense(cases=((1000, 64, 37), (2048, 256, 23), (4096, 64, 53), (300, 128, 11)),
                    seed: int = 7) -> None:
    """Block-wise Π1·X equals the explicit product 4·B·C·H̃·D of the four factors."""
    g = np.random.default_rng(seed)
    for n, s, r1 in cases:
        for sign_flip in (True, False):
            X = g.standard_normal((n, 5))
            pix, tsum = fct.fct1_embed(X, s, r1, seed, 1, 0, sign_flip)
            n_pad = fct.padded_rows(n, s)
            xp = np.zeros((n_pad, 5))
            xp[:n] = X
            dense = fct.dense_pi1(n, s, r1, seed, 1, 0, sign_flip) @ xp
            scale = np.abs(dense).max()
            assert np.allclose(pix, dense, rtol=1e-12, atol=1e-12 * scale), f"Π1X n={n} s={s}"
            assert np.all(tsum >= np.abs(pix) * (1 - 1e-12)), "T < |Π1X|"


def _identity_draws(n_pad: int):
    """C ≡ 1 and every virtual row in its own bucket: Hadamard row ι → 2ι, identity row ι → 2ι+1."""
    rows = np.arange(n_pad)
    return {"hash_h": 2 * rows, "hash_i": 2 * rows + 1,
            "cauchy_h": np.ones(n_pad), "cauchy_i": np.ones(n_pad),
            "sigma": np.where(rows % 3 == 0, -1.0, 1.0)}


def check_fct_blocks(seed: int = 11) -> None:
    """With C ≡ 1 and injective buckets Π1X exposes g = H̃·D·x, which must satisfy
    ‖G_s z‖₂² = 2‖z‖₂² (proof of FCT1), the uncertainty lemma ‖G_s z‖₁ ≥ ½ s^{1/4}‖z‖₂,
    and H_s z = the closed-form Walsh sum Σ_j (−1)^{popcount(i∧j)} z_j / √s."""
    g = np.random.default_rng(seed)
    for s in (1, 2, 16, 64, 256):
        n = 3 * s + (s // 2 if s > 1 else 0)
        n_pad = fct.padded_rows(n, s)
        X = g.standard_normal((n, 3))
        X[: s // 2 + 1, 1] = 0.0
        X[0, 1] = 5.0                     # a spiky column: the adversarial case of the lemma
        dr = _identity_draws(n_pad)
        pix, tsum = fct.fct1_embed(X, s, 2 * n_pad, draws=dr)
        gh = pix[0::2] / 4.0
        gi = pix[1::2] / 4.0
        xp = np.zeros((n_pad, 3))
        xp[:n] = X
        z = dr["sigma"][:, None] * xp
        assert np.allclose(gi, z, rtol=0, atol=1e-13), "identity half"
        idx = np.arange(s)
        walsh = np.where(np.vectorize(lambda v: bin(v).count("1") & 1)(idx[:, None] & idx[None, :]) == 1, -1.0, 1.0)
        for beta in range(n_pad // s):
            zb = z[beta * s:(beta + 1) * s]
            hb = gh[beta * s:(beta + 1) * s]
            assert np.allclose(hb, walsh @ zb / math.sqrt(s), atol=1e-12), "H_s z"
            for c in range(3):
                gz = np.concatenate([hb[:, c], zb[:, c]])
                n2 = np.sum(zb[:, c] ** 2)
                assert math.isclose(np.sum(gz ** 2), 2 * n2, rel_tol=1e-12, abs_tol=1e-12), "energy"
                assert np.sum(np.abs(gz)) >= 0.5 * s ** 0.25 * math.sqrt(n2) - 1e-12, "uncertainty"
        assert np.allclose(tsum[1::2], np.abs(pix[1::2]), atol=1e-13), "T of an identity row"
        blocksum = np.repeat(np.abs(z).reshape(-1, s, 3).sum(axis=1), s, axis=0)
        assert np.allclose(tsum[0::2], 4.0 * blocksum / math.sqrt(s), rtol=1e-13), "T of a Hadamard row"


def check_fct_row_offset(seed: int = 29) -> None:
    """Π1 is one linear map of all n rows whose variates (D, C, B) belong to global row ids,
    so cutting X at a multiple of s and embedding the two parts with their row offsets gives
    two matrices that add up to the embedding of the whole, and so do their Σ|terms|; the
    ragged tail pads with zero rows either way (§3.1; row ids as the shards' reading)."""
    g = np.random.default_rng(seed)
    for s in (1, 4, 64):
        n = 7 * s + s // 2 + 1
        cut = 3 * s
        X = g.standard_normal((n, 4))
        r1 = 37
        whole, tw = fct.fct1_embed(X, s, r1, seed=5, problem_id=1)
        top, tt = fct.fct1_embed(X[:cut], s, r1, seed=5, problem_id=1, row_offset=0)
        bot, tb = fct.fct1_embed(X[cut:], s, r1, seed=5, problem_id=1, row_offset=cut)
        assert np.all(np.abs(top + bot - whole) <= 1e-12 * tw + 1e-300), f"additivity at s = {s}"
        assert np.allclose(tt + tb, tw, rtol=1e-12, atol=0), f"Σ|terms| additivity at s = {s}"
        # the offset matters: the bottom part embedded as if its rows came first differs
        wrong, _ = fct.fct1_embed(X[cut:], s, r1, seed=5, problem_id=1, row_offset=0)
        assert np.abs(top + wrong - whole).max() > 1e-6 * np.abs(whole).max(), "row ids ignored"


def check_fct_mass(seed: int = 5) -> None:
    """With C ≡ 1 and random buckets, Σ_rows Π1X = 4·Σ g per column (the hashed sums add
    up, proof of FCT1), and Σ_rows T = 4·(1 + √s)·‖z‖₁: every input entry enters one identity
    row and the s Hadamard rows of its block with |H_s entry| = 1/√s."""
    g = np.random.default_rng(seed)
    n, s, r1 = 700, 64, 19
    X = g.standard_normal((n, 4))
    n_pad = fct.padded_rows(n, s)
    dr = rng.fct_draws(seed, 0, np.arange(n_pad), r1)
    dr = dict(dr, cauchy_h=np.ones(n_pad), cauchy_i=np.ones(n_pad))
    pix, tsum = fct.fct1_embed(X, s, r1, draws=dr)
    dense_g = _explicit_g(X, s, dr["sigma"])
    assert np.allclose(pix.sum(0), 4 * dense_g.sum(0), rtol=1e-12), "mass"
    z1 = np.abs(dense_g[fct.padded_rows(n, s):]).sum(0)          # identity half = z
    assert np.allclose(tsum.sum(0), 4 * (1 + math.sqrt(s)) * z1, rtol=1e-12), "ℓ1 mass"


def _explicit_g(X, s, sigma):
    n = X.shape[0]
    n_pad = fct.padded_rows(n, s)
    xp = np.zeros((n_pad, X.shape[1]))
    xp[:n] = X
    z = sigma[:n_pad, None] * xp
    idx = np.arange(s)
    walsh = np.where(np.vectorize(lambda v: bin(v).count("1") & 1)(idx[:, None] & idx[None, :]) == 1, -1.0, 1.0)
    gh = np.concatenate([walsh @ z[b * s:(b + 1) * s] / math.sqrt(s) for b in range(n_pad // s)])
    return np.concatenate([gh, z])


def check_fct_stability(seeds: int = 40) -> None:
    """Conditional on B, (Π1X)_jc is a Cauchy scaled by γ_jc = 4·Σ_{v→j}|g_vc| with g = H̃·D·x
    (1-stability, §2; proof of FCT1): the standardized entries pooled over seeds pass a KS test
    against Cauchy(0,1).  g comes from the closed-form Walsh matrix, not from the oracle."""
    g = np.random.default_rng(99)
    n, s, r1 = 512, 64, 13
    X = g.standard_normal((n, 3))
    vals = []
    for sd in range(seeds):
        dr = rng.fct_draws(1000 + sd, 0, np.arange(n), r1)
        pix, _ = fct.fct1_embed(X, s, r1, draws=dr)
        gfull = np.abs(_explicit_g(X, s, dr["sigma"]))          # [Hadamard half; identity half]
        buckets = np.concatenate([dr["hash_h"], dr["hash_i"]])
        gam = np.stack([4.0 * np.bincount(buckets, weights=gfull[:, c], minlength=r1) for c in range(3)], axis=1)
        vals.append((pix / gam).ravel())
    v = np.concatenate(vals)
    assert stats.kstest(v, "cauchy").pvalue > 1e-4, "Π1X entries not Cauchy-scaled"


# ----------------------------------------------------------------- conditioning
def check_qr(seed: int = 3) -> None:
    """Q·R = Π1X, QᵀQ = I, R upper with positive diagonal, RᵀR = Gram (Cholesky route),
    R·M = Π2, and Π1X·R⁻¹ has orthonormal columns (Figure 2, step 2)."""
    g = np.random.default_rng(seed)
    A = g.standard_normal((355, 17)) * (10.0 ** g.uniform(-2, 2, 17))[None, :]
    qm, rm = condition.qr_positive(A)
    assert np.allclose(qm @ rm, A, rtol=0, atol=1e-12 * np.abs(A).max()), "QR product"
    assert np.allclose(qm.T @ qm, np.eye(17), atol=1e-13), "Q orthonormal"
    assert np.allclose(rm, np.triu(rm)), "R upper"
    assert np.all(np.diag(rm) > 0), "diag R > 0"
    chol = np.linalg.cholesky(A.T @ A).T
    assert np.allclose(rm, chol, rtol=1e-8, atol=1e-8 * np.abs(rm).max()), "R vs Cholesky"
    pi2 = rng.pi2_matrix(1, 0, 17, 16)
    mm = condition.m_matrix(rm, pi2)
    assert np.allclose(rm @ mm, pi2, rtol=1e-11, atol=1e-11 * np.abs(pi2).max()), "R·M = Π2"
    ri = condition.r_inverse(rm)
    assert np.allclose((A @ ri).T @ (A @ ri), np.eye(17), atol=1e-10), "Π1X R⁻¹ orthonormal"
    bad = A.copy()
    bad[:, 3] = bad[:, 2]
    try:
        condition.check_rank(condition.qr_positive(bad)[1])
    except condition.RankDeficient:
        pass
    else:
        raise AssertionError("rank deficiency not detected")


# ----------------------------------------------------------------- leverage
def _half_cauchy_median_fraction(r2: int, k: int) -> float:
    f = lambda x: 2.0 / math.pi * math.atan(x)   # noqa: E731  CDF of |Cauchy|
    return float(stats.binom.sf(k - 1, r2, f(1.5)) - stats.binom.sf(k - 1, r2, f(0.5)))


def check_lambda_distribution(r2: int = 16, seeds: int = 300, rows: int = 128) -> None:
    """Λ_ij / ‖U_(i)‖₁ is standard Cauchy (proof of the fast ℓ1 regression theorem), and
    the share of rows with ½‖U_(i)‖₁ ≤ λ_i ≤ 3/2‖U_(i)‖₁ matches the exact order-statistic
    value for the lower median of r2 half-Cauchys (0.8328 for r2 = 16)."""
    g = np.random.default_rng(17)
    X = g.standard_normal((rows, 6)) * np.array([1, 10, 0.1, 3, 1, 1.0])[None, :]
    _, rm = condition.qr_positive(g.standard_normal((40, 6)))
    ri = condition.r_inverse(rm)
    norms = leverage.exact_row_l1(X, ri)
    assert np.allclose(norms, np.abs(X @ np.linalg.inv(rm)).sum(1), rtol=1e-12)
    fr, std = [], []
    for sd in range(seeds):
        pi2 = rng.pi2_matrix(500 + sd, 0, 6, r2)
        mm = condition.m_matrix(rm, pi2)
        lam = leverage.lambda_estimates(X, mm)
        i = sd % rows                      # one row per seed: its r2 entries are independent
        std.append((X[i] @ mm) / norms[i])
        ratio = lam / norms
        fr.append(np.mean((ratio >= 0.5) & (ratio <= 1.5)))
    fr = np.array(fr)
    assert stats.kstest(np.concatenate(std), "cauchy").pvalue > 1e-4, "Λ/‖U‖₁ not Cauchy"
    want = _half_cauchy_median_fraction(r2, (r2 - 1) // 2 + 1)
    se = fr.std(ddof=1) / math.sqrt(seeds)
    assert abs(fr.mean() - want) < 4 * se + 1e-3, f"median fraction {fr.mean()} vs {want}"


# ----------------------------------------------------------------- sampling
def check_sampling(seed: int = 21) -> None:
    """p̂ = min(1, m_s λ/Σλ) sums to m_s when no row saturates; kept rows satisfy u < p̂ in
    ascending order; S concentrates at Σp̂; the Horvitz–Thompson sum Σ_kept |r_i|/p̂_i is
    unbiased for ‖r‖₁ (ℓ1 sampling lemma, E[D_ii] = 1)."""
    g = np.random.default_rng(seed)
    n = 50000
    flat = g.uniform(1.0, 2.0, 4000)
    pf, tf, _ = sampling.probabilities(flat, 500.0)
    assert pf.max() < 1.0 and math.isclose(pf.sum(), 500.0, rel_tol=1e-12), "Σp̂ = m_s"
    lam = np.abs(g.standard_cauchy(n)) + 0.01
    lam[:3] = 1e6                                           # saturating rows
    p, tau, total = sampling.probabilities(lam, 1000.0)
    assert math.isclose(total, math.fsum(lam.tolist()), rel_tol=0)
    assert np.all(p[:3] == 1.0) and p.max() <= 1.0 and p.sum() <= 1000.0 * (1 + 1e-12)
    free = p < 1.0
    assert np.allclose(p[free] / lam[free], tau, rtol=1e-15)
    assert math.isclose(tau, 1000.0 / total, rel_tol=1e-15)
    u = rng.sample_uniforms(seed, 0, np.arange(n))
    idx, w = sampling.bernoulli_sample(p, u)
    mask = np.zeros(n, bool)
    mask[idx] = True
    assert np.array_equal(mask, u < p) and np.all(np.diff(idx) > 0)
    assert np.allclose(w, 1.0 / p[idx], rtol=0)
    es, var = p.sum(), (p * (1 - p)).sum()
    assert abs(idx.size - es) < 5 * math.sqrt(var) + 1
    r = np.abs(g.standard_normal(n)) * lam
    est = []
    for sd in range(200):
        u = rng.sample_uniforms(seed + 1 + sd, 0, np.arange(n))
        k, ww = sampling.bernoulli_sample(p, u)
        est.append(np.sum(ww * r[k]))
    est = np.array(est)
    assert abs(est.mean() - r.sum()) < 5 * est.std(ddof=1) / math.sqrt(est.size), "HT biased"


# ----------------------------------------------------------------- solve
def check_solver(seed: int = 8) -> None:
    """LP optimum = brute-force vertex optimum on tiny instances; = weighted median for a
    single all-ones column; = per-coordinate weighted median for canonical-vector rows
    (the separable design of the large-scale experiment, §6.3)."""
    g = np.random.default_rng(seed)
    for m, d in ((7, 1), (9, 2), (12, 3), (11, 2)):
        A = g.standard_normal((m, d))
        b = g.standard_normal(m) * 3
        w = g.uniform(0.2, 3.0, m)
        _, f_lp = solve.lad_lp(A, b, w)
        _, f_bf = solve.lad_bruteforce(A, b, w)
        assert math.isclose(f_lp, f_bf, rel_tol=1e-12, abs_tol=1e-12), f"LP vs brute force {m}x{d}"
    b = g.standard_cauchy(301)
    w = g.uniform(0.5, 2.0, 301)
    x, f = solve.lad_lp(np.ones((301, 1)), b, w)
    med = solve.weighted_median(b, w)
    assert math.isclose(f, solve.weighted_objective(np.ones((301, 1)), b, w, [med]), rel_tol=1e-12)
    d = 5
    rows = g.integers(0, d, 400)
    A = np.eye(d)[rows]
    b = g.standard_normal(400) + rows
    w = g.uniform(0.5, 2.0, 400)
    x, f = solve.lad_lp(A, b, w)
    xm = np.array([solve.weighted_median(b[rows == j], w[rows == j]) for j in range(d)])
    assert math.isclose(f, solve.weighted_objective(A, b, w, xm), rel_tol=1e-12), "canonical rows"
    Xr = np.array([[1.0, 2.0], [3.0, -1.0]])
    assert np.allclose(pipeline.form_x(Xr, np.array([5.0, 7.0])) @ np.array([0.5, -1.0, 1.0]),
                       Xr @ np.array([0.5, -1.0]) - np.array([5.0, 7.0])), "X·[x;1] = Ax − b"


ALL_CHECKS = [check_hadamard_closed_form, check_cauchy_quantiles, check_draw_statistics,
              check_fct_dense, check_fct_blocks, check_fct_mass, check_fct_stability,
              check_qr, check_lambda_distribution, check_sampling, check_solver]


# ----------------------------------------------------------------- BF16 rounding of M
def check_bf16_round() -> None:
    """Values with at most 8 significant bits are unchanged; midpoints go to the even
    neighbour; the relative error is at most 2^-8 (half an ulp of an 8-bit significand at the
    bottom of a binade) plus the FP32 step."""
    from oracle import leverage

    exact = np.array([1.0, -3.5, 0.0078125, 2.0 ** -30 * 255 / 128, 1.9921875, -100.0])
    assert np.array_equal(leverage.bf16_round(exact), exact)
    ulp = 2.0 ** -7
    assert leverage.bf16_round(np.array([1.0 + ulp / 2]))[0] == 1.0            # tie → even (1.0)
    assert leverage.bf16_round(np.array([1.0 + 3 * ulp / 2]))[0] == 1.0 + 2 * ulp  # tie → even
    assert leverage.bf16_round(np.array([1.0 + ulp / 2 + 1e-6]))[0] == 1.0 + ulp   # past the midpoint
    # the FP32 step comes first: a nudge below FP32 resolution is lost and the tie goes to even
    assert leverage.bf16_round(np.array([1.0 + ulp / 2 + 1e-9]))[0] == 1.0
    g = np.random.default_rng(3)
    x = g.standard_normal(100000) * 10.0 ** g.uniform(-5, 5, 100000)
    r = leverage.bf16_round(x)
    assert np.all(np.abs(r - x) <= (2.0 ** -8 + 2.0 ** -23) * np.abs(x))   # BF16 half-ulp + the FP32 step
    assert np.quantile(np.abs(r - x) / np.abs(x), 0.99) > 2.0 ** -9      # and it is attained
    M = g.standard_normal((5, 3))
    mm = leverage.mixed_precision_m(M)
    assert np.array_equal(mm[-1], M[-1].astype(np.float32)) and np.array_equal(mm[:-1], leverage.bf16_round(M[:-1]))


# ----------------------------------------------------------------- OptimizedFastCauchyRegression
def check_gaussian_pi2(q: int = 64, r2: int = 800) -> None:
    """The Gaussian Π2 (Figure "mainOpt", step 4) is standard normal (KS), the two entries of
    each Box–Muller pair are uncorrelated and their squared sum is χ²₂ (exponential, mean 2) —
    which a pair built from one uniform twice, or a wrong ρ, fails — and different problems
    draw independent matrices."""
    z = rng.pi2_gaussian_matrix(99, 3, q, r2).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-4, "Π2 entries not N(0,1)"
    a, b = z[0::2], z[1::2]
    assert abs(np.corrcoef(a, b)[0, 1]) < 4 / math.sqrt(a.size), "pair correlated"
    assert stats.kstest(a * a + b * b, "expon", args=(0, 2)).pvalue > 1e-4, "pair radius not χ²₂"
    other = rng.pi2_gaussian_matrix(99, 4, q, r2).ravel()
    assert abs(np.corrcoef(z, other)[0, 1]) < 4 / math.sqrt(z.size), "problems not independent"


def _half_normal_median_cdf(x: float, r2: int) -> float:
    """P(lower median of r2 independent |N(0,1)| ≤ x): at least (r2−1)//2 + 1 of them ≤ x."""
    p = math.erf(x / math.sqrt(2.0))
    return float(stats.binom.sf((r2 - 1) // 2, r2, p))


def check_gaussian_lambda_distribution(r2: int = 8, seeds: int = 400, rows: int = 64) -> None:
    """With a Gaussian Π2, Λ_ij = (X·R⁻¹·Π2)_ij is N(0, ‖U_(i)‖₂²) (the intuition given for
    OptimizedFastCauchyRegression), so λ̂_i/‖U_(i)‖₂ follows the lower-median order statistic of
    r2 half-normals: KS against its exact CDF."""
    g = np.random.default_rng(23)
    X = g.standard_normal((rows, 5)) * np.array([1, 7, 0.2, 2, 1.0])[None, :]
    _, rm = condition.qr_positive(g.standard_normal((30, 5)))
    l2 = np.linalg.norm(X @ np.linalg.inv(rm), axis=1)
    ratios = []
    for sd in range(seeds):
        mm = condition.m_matrix(rm, rng.pi2_gaussian_matrix(700 + sd, 0, 5, r2))
        lam = leverage.lambda_estimates(X, mm)
        ratios.append(lam[sd % rows] / l2[sd % rows])
    cdf = np.vectorize(lambda x: _half_normal_median_cdf(x, r2))
    assert stats.kstest(np.array(ratios), cdf).pvalue > 1e-4, "λ̂/‖U‖₂ not the half-normal median"


def check_scaled_probabilities(seed: int = 31) -> None:
    """p̂ = min{1, s·λ̂} without normalisation: linear below saturation, 1 above, and the
    Horvitz–Thompson sum over the Bernoulli sample is unbiased for Σ|r_i|."""
    g = np.random.default_rng(seed)
    lam = np.abs(g.standard_normal(20000)) + 1e-3
    p = sampling.probabilities_scaled(lam, 0.4)
    below = 0.4 * lam < 1.0
    assert np.array_equal(p[below], 0.4 * lam[below]) and np.all(p[~below] == 1.0)
    r = np.abs(g.standard_normal(20000))
    est = []
    for t in range(200):
        u = g.uniform(size=lam.size)
        idx, w = sampling.bernoulli_sample(p, u)
        est.append(math.fsum((r[idx] * w).tolist()))
    est = np.array(est)
    assert abs(est.mean() - r.sum()) < 4 * est.std(ddof=1) / math.sqrt(len(est)), "HT biased"


def _all_checks():
    return ALL_CHECKS + [check_bf16_round, check_gaussian_pi2, check_gaussian_lambda_distribution,
                         check_scaled_probabilities, check_multiple_regression, check_with_replacement,
                         check_sct_draws, check_sct_stability, check_sct_embedding_bound, check_kappa_bar,
                         check_canonical_optimum, check_fjlt_isometry, check_fjlt_spread, check_fct2_dense,
                         check_fct2_stability, check_fct2_embedding_bound, check_philox_key_schedule,
                         check_fct_row_offset]


# ----------------------------------------------------------------- slow Cauchy transform
def check_sct_draws(rows: int = 20000, r1: int = 13, seed: int = 77) -> None:
    """Entries of the slow transform's C (stream 4) are standard Cauchy (KS), and entries drawn
    from different words and from different calls of a row are independent (rank correlation
    near zero, as it is for independent draws)."""
    C = rng.sct_matrix(seed, 3, np.arange(rows) + 1000, r1)
    assert C.shape == (r1, rows)
    for r in range(r1):
        assert stats.kstest(C[r], "cauchy").pvalue > 1e-4, f"row {r} of C not Cauchy"
    for a, b in ((0, 1), (0, 4), (3, 7), (5, 12)):
        rho = stats.spearmanr(C[a], C[b]).statistic
        assert abs(rho) < 5.0 / math.sqrt(rows), f"rows {a} and {b} of C are dependent (rho {rho:.3f})"


def check_sct_stability(seeds: int = 30) -> None:
    """1-stability (§2): column c of C·X is a vector of independent Cauchys scaled by ‖X_{:,c}‖₁,
    so (r1/4)·(Π1X)_{rc}/‖X_{:,c}‖₁ pooled over entries and seeds passes a KS test against
    Cauchy(0,1); the norms come from X directly, not from the oracle."""
    g = np.random.default_rng(5)
    n, r1 = 1500, 37
    X = g.standard_normal((n, 3)) * np.array([1.0, 10.0, 0.01])
    vals = []
    for sd in range(seeds):
        pix, _ = sct.sct_embed(X, r1, seed=500 + sd, problem_id=1, block=512)
        vals.append(((r1 / 4.0) * pix / np.abs(X).sum(axis=0)).ravel())
    assert stats.kstest(np.concatenate(vals), "cauchy").pvalue > 1e-4, "slow transform not Cauchy-scaled"


def check_sct_embedding_bound(seed: int = 9) -> None:
    """The lower bound of the theorem of §3 on the slow transform: ‖y‖₁ ≤ (4/r1)‖C·y‖₁ for y in
    the column space of X (r1 = ⌈8·d·ln d⌉ here), for every one of 50 random y.  The sum of r1
    half-Cauchys exceeds r1/4 by a wide margin, so a missing factor or dropped rows fail it."""
    g = np.random.default_rng(seed)
    n, d = 3000, 6
    X = g.standard_normal((n, d))
    r1 = int(math.ceil(8 * d * math.log(d)))
    pix, tsum = sct.sct_embed(X, r1, seed=seed, block=1024)
    assert np.all(tsum >= np.abs(pix) * (1 - 1e-12)), "sum of |terms| below |entry|"
    for _ in range(50):
        x = g.standard_normal(d)
        ratio = np.abs(pix @ x).sum() / np.abs(X @ x).sum()
        assert ratio >= 1.0, f"(4/r1)·‖C·y‖₁ / ‖y‖₁ = {ratio:.3f} < 1"


# ----------------------------------------------------------------- multiple regression
def check_multiple_regression(seed: int = 17) -> None:
    """FastCauchyRegression(A, B) of §4.2.1.  (1) k = 1 reduces to the single right-hand
    side pipeline (same draws, same coreset, same solution).  (2) B = A·W* + E with sparse gross
    errors E is fitted exactly (ℓ1 regression's exact recovery): W = W* column by column
    and objective j is ‖E_j‖₁.  (3) The objectives
    add up to the entrywise ℓ1 norm of X·Z with X = [A, −B] and Z = [W; I_k]."""
    g = np.random.default_rng(seed)
    n, d, k = 3000, 4, 3
    A = g.standard_normal((n, d))
    Wstar = g.standard_normal((d, k))
    B = A @ Wstar + g.laplace(size=(n, k))
    one = pipeline.fast_cauchy_multiple_regression(A, B[:, :1], 64, 40, 16, 300.0, seed=2)
    ref = pipeline.fast_cauchy_regression(A, B[:, 0], 64, 40, 16, 300.0, seed=2)
    assert np.array_equal(one["idx"], ref["idx"]) and np.array_equal(one["w"], ref["w"])
    assert np.allclose(one["W"][:, 0], ref["x_hat"], rtol=0, atol=1e-9)
    assert abs(one["objectives"][0] - ref["objective"]) <= 1e-12 * ref["objective"]
    # sparse gross errors (1% of rows) keep X full rank, and ℓ1 regression recovers W* exactly
    E = np.where(g.random((n, k)) < 0.01, 50.0 * g.standard_normal((n, k)), 0.0)
    exact = pipeline.fast_cauchy_multiple_regression(A, A @ Wstar + E, 64, 40, 16, 600.0, seed=3)
    assert np.allclose(exact["W"], Wstar, rtol=0, atol=1e-8), np.abs(exact["W"] - Wstar).max()
    assert np.allclose(exact["objectives"], np.abs(E).sum(axis=0), rtol=1e-10, atol=0)
    res = pipeline.fast_cauchy_multiple_regression(A, B, 64, 40, 16, 300.0, seed=4)
    Z = np.vstack([res["W"], np.eye(k)])
    X = pipeline.form_x_multi(A, B)
    assert abs(np.abs(X @ Z).sum() - res["objectives"].sum()) <= 1e-12 * res["objectives"].sum()


# ----------------------------------------------------------------- sampling with replacement
def check_with_replacement(seed: int = 23) -> None:
    """Exactly m draws with p̂_i = λ_i/Σλ (caption of Figure 2).  (1) Each draw inverts the
    running sum: brute force over rows on a small case, zero-λ rows never drawn.  (2) Every
    weighted draw carries w_t·λ_{i_t} = Σλ/m, so the weights·λ add up to Σλ.  (3) Row
    frequencies follow p̂ (χ²).  (4) Σ_t w_t·r_{i_t} is unbiased for Σ_i r_i."""
    g = np.random.default_rng(seed)
    lam = np.abs(g.standard_cauchy(40))
    lam[[3, 17, 18]] = 0.0
    u = rng.replacement_uniforms(5, 1, np.arange(500))
    idx, w, cdf = sampling.sample_with_replacement(lam, 500, u)
    total = math.fsum(lam.tolist())
    for t in range(500):
        acc, want = 0.0, None
        for i in range(lam.size):
            acc += lam[i]
            if u[t] * cdf[-1] < acc:
                want = i
                break
        assert idx[t] == want, (t, idx[t], want)
    assert not np.isin(idx, [3, 17, 18]).any()
    assert np.allclose(w * lam[idx], total / 500, rtol=1e-12)
    lam2 = g.uniform(0.1, 1.0, 16)
    m = 200000
    u2 = rng.replacement_uniforms(9, 0, np.arange(m))
    idx2, w2, _ = sampling.sample_with_replacement(lam2, m, u2)
    f_obs = np.bincount(idx2, minlength=16)
    f_exp = m * lam2 / lam2.sum()
    chi2 = float(((f_obs - f_exp) ** 2 / f_exp).sum())
    assert stats.chi2.sf(chi2, 15) > 1e-4, chi2
    r = np.abs(g.standard_normal(16))
    est = []
    for rep in range(100):
        uu = rng.replacement_uniforms(100 + rep, 0, np.arange(50))
        ii, ww, _ = sampling.sample_with_replacement(lam2, 50, uu)
        est.append(float((ww * r[ii]).sum()))
    est = np.array(est)
    assert abs(est.mean() - r.sum()) < 4 * est.std(ddof=1) / math.sqrt(len(est)), "estimator biased"


# ----------------------------------------------------------------- conditioning quality (§6.1)
def check_kappa_bar(seed: int = 13) -> None:
    """κ̄₁: the identity basis I_d has α = d and min_{‖z‖∞=1} ‖z‖₁ = 1, so κ̄₁ = d (closed form);
    κ̄₁ is scale invariant (§6.1); and for a small U with d = 2 the minimum over the boundary of
    the unit box, found by brute force over every breakpoint of the piecewise-linear ‖U·z‖₁ on
    each face (z = (±1, t) or (t, ±1), t at a zero of some U_i·z, or t = ±1), matches the d
    regressions."""
    for d in (1, 2, 5):
        assert abs(quality.kappa_bar_1(np.eye(d)) - d) < 1e-9, f"κ̄₁(I_{d}) != {d}"
    g = np.random.default_rng(seed)
    U = g.standard_normal((7, 2)) * np.array([1.0, 30.0])
    k = quality.kappa_bar_1(U)
    assert abs(quality.kappa_bar_1(123.0 * U) - k) < 1e-9 * k, "κ̄₁ not scale invariant"
    cands = []
    for fixed in (0, 1):
        free = 1 - fixed
        ts = np.concatenate([[-1.0, 1.0], -U[:, fixed] / U[:, free]])
        for t in ts[np.abs(ts) <= 1.0]:
            z = np.empty(2)
            z[fixed], z[free] = 1.0, t
            cands.append(np.abs(U @ z).sum())
    brute = min(cands)
    got = quality.min_l1_on_unit_box(U)
    assert abs(got - brute) <= 1e-9 * brute, (got, brute)

# ----------------------------------------------------------------- separable design (§6.3)
def check_canonical_optimum(seed: int = 21) -> None:
    """For canonical-vector rows the LP optimum of ‖A·x − b‖₁ (HiGHS) has the objective of
    both corners of the oracle's box [lo, hi] and of a point inside it; moving one coordinate
    just outside the box raises the objective; groups of odd size give lo = hi; the distance
    to the box vanishes inside it and the relative errors follow their definitions."""
    g = np.random.default_rng(seed)
    d = 5
    sizes = [7, 10, 3, 8, 1]                  # odd and even groups, one singleton
    cols = g.permutation(np.repeat(np.arange(d), sizes))
    b = g.laplace(size=cols.size) + cols.astype(np.float64)
    A = np.eye(d)[cols]
    _, f_lp = solve.lad_lp(A, b)
    lo, hi = separable.canonical_optimum(cols, b, d)
    for j, m in enumerate(sizes):
        assert (lo[j] == hi[j]) == (m % 2 == 1), f"group {j} of size {m}"
        assert lo[j] <= hi[j]
    mid = 0.5 * (lo + hi)
    for x in (lo, hi, mid):
        assert math.isclose(solve.objective(A, b, x), f_lp, rel_tol=1e-12), "box point not optimal"
    for j in range(d):
        for x0, step in ((lo, -1e-3), (hi, 1e-3)):
            x = x0.copy()
            x[j] += step
            assert solve.objective(A, b, x) > f_lp * (1 + 1e-9), f"coordinate {j} leaves the box"
    assert np.all(separable.box_distance(mid, lo, hi) == 0.0)
    x = hi.copy()
    x[2] += 0.5
    x[0] = lo[0] - 0.25
    e = separable.relative_errors(x, lo, hi, lo)
    assert math.isclose(e["l1"], 0.75 / np.abs(lo).sum(), rel_tol=1e-12)
    assert math.isclose(e["l2"], math.sqrt(0.5 ** 2 + 0.25 ** 2) / np.linalg.norm(lo), rel_tol=1e-12)
    assert math.isclose(e["linf"], 0.5 / np.abs(lo).max(), rel_tol=1e-12)


# ----------------------------------------------------------------- FCT2 (§3.2)
def check_fjlt_isometry(t: int = 16, s: int = 4, seeds: int = 600) -> None:
    """The SRHT block G = √(t/s)·S·H_t·D has entries ±1/√s, so diag(GᵀG) = 1 exactly; over
    seeds E[GᵀG] = D·H_tᵀ·H_t·D = I (off-diagonal means near 0) and, rows being sampled
    independently, each off-diagonal entry has mean square 1/s (not 1, as for repeated rows)."""
    acc = np.zeros((t, t))
    acc2 = np.zeros((t, t))
    for sd in range(seeds):
        G = fct2.fjlt_matrix(sd, 0, t, s)
        assert np.allclose(np.abs(G), 1.0 / math.sqrt(s)), "entries of G are not ±1/√s"
        M = G.T @ G
        assert np.allclose(np.diag(M), 1.0), "diag(GᵀG) != 1"
        acc += M
        acc2 += M * M
    off = ~np.eye(t, dtype=bool)
    mean = acc / seeds
    assert np.abs(mean[off]).max() < 5.0 / math.sqrt(s * seeds), "E[GᵀG] is not I"
    ms = (acc2 / seeds)[off]
    assert abs(ms.mean() - 1.0 / s) < 0.1 / s, ("off-diagonal mean square", ms.mean(), 1.0 / s)


def check_fjlt_spread(t: int = 64, s: int = 16, seeds: int = 200) -> None:
    """The random signs spread a structured vector: for x = (1, …, 1), H_t·x = √t·e_0 alone,
    but H_t·D·x is a ±1-sum in every row, so ‖G·x‖₂² ≈ ‖x‖₂² = t (median over seeds within a
    factor 2)."""
    x = np.ones(t)
    r = [float(np.sum((fct2.fjlt_matrix(sd, 1, t, s) @ x) ** 2)) / t for sd in range(seeds)]
    med = float(np.median(r))
    assert 0.5 < med < 2.0, ("‖Gx‖² / ‖x‖² median", med)


def check_fct2_dense(seed: int = 5) -> None:
    """Π1·X from the blocks equals the explicit product of the factors,
    (8/r1)·√(πt/(2s))·C·H̃ with H̃ = diag(G, …, G) over the zero-padded rows, C's column k
    the Cauchys of row id (offset/t)·s + k, for a ragged n and a nonzero block offset."""
    g = np.random.default_rng(seed)
    t, s, r1 = 16, 6, 11
    n, q = 3 * t + 5, 3
    X = g.standard_normal((n, q))
    off = 7 * t
    got, _ = fct2.fct2_embed(X, t, s, r1, seed=seed, problem_id=2, row_offset=off)
    nb = -(-n // t)
    G = fct2.fjlt_matrix(seed, 2, t, s)
    Ht = np.zeros((nb * s, nb * t))
    for b in range(nb):
        Ht[b * s:(b + 1) * s, b * t:(b + 1) * t] = G
    C = rng.sct_matrix(seed, 2, (off // t) * s + np.arange(nb * s), r1)
    Xp = np.zeros((nb * t, q))
    Xp[:n] = X
    want = 8.0 / r1 * math.sqrt(math.pi * t / (2 * s)) * (C @ (Ht @ Xp))
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max()), "FCT2 blocks != dense product"


def check_fct2_stability(seeds: int = 400) -> None:
    """1-stability: for a fixed y, entry r of Π1·y is (8/r1)·√(πt/(2s)) times a standard Cauchy
    times ‖H̃y‖₁, so its ratio to scale·‖H̃y‖₁ is standard Cauchy over seeds (KS)."""
    t, s, r1, n = 32, 8, 10, 96
    y = np.random.default_rng(3).standard_normal((n, 1))
    ratios = []
    for sd in range(seeds):
        pix, _ = fct2.fct2_embed(y, t, s, r1, seed=sd)
        G = fct2.fjlt_matrix(sd, 0, t, s)
        hy = np.abs(np.einsum("rt,bt->br", G, y[:, 0].reshape(-1, t))).sum()
        ratios.append(pix[0, 0] / (8.0 / r1 * math.sqrt(math.pi * t / (2 * s)) * hy))   # §3.2's scale
    p = stats.kstest(ratios, "cauchy").pvalue
    assert p > 1e-3, ("Π1y is not scale·Cauchy·‖H̃y‖₁", p)


def check_fct2_embedding_bound(seed: int = 9) -> None:
    """The lower bound of Theorem FCT2, ‖y‖₁ ≤ ‖Π1·y‖₁ for y in the column space of X
    (d = 4, r1 = ⌈8 d ln d⌉, s = ⌈2 d ln d⌉, t = 2^⌈log₂ 2d²⌉), for every one of 50 random y."""
    g = np.random.default_rng(seed)
    d, n = 4, 2048
    r1, s, t = math.ceil(8 * d * math.log(d)), math.ceil(2 * d * math.log(d)), 32
    X = g.standard_normal((n, d)) * np.array([1.0, 10.0, 0.1, 3.0])
    for k in range(50):
        z = g.standard_normal(d)
        y = X @ z
        pix, _ = fct2.fct2_embed(y[:, None], t, s, r1, seed=100 + k)
        assert np.abs(pix).sum() >= np.abs(y).sum(), f"‖Π1y‖₁ < ‖y‖₁ for y {k}"


# ----------------------------------------------------------------- Philox4x32-10 key schedule
def check_philox_key_schedule() -> None:
    """Philox4x32-10 bumps its two key words by Weyl constants defined in closed form (Salmon et
    al., SC'11): ⌊2^32/φ⌋ (φ the golden ratio) and ⌊2^32·(√3 − 1)⌋, computed here with exact
    integer square roots; and the generator uses them: advancing the key of a call by one
    schedule step moves every one of its later round keys, so the outputs of the same counter
    under keys (k0, k1) and (k0 + W0, k1 + W1) differ.  (The multipliers have no closed form;
    they stay pinned by the output laws of check_draw_statistics.)"""
    from math import isqrt

    w0 = isqrt(5 << 62) - (1 << 31)        # 2^32/φ = 2^31·(√5 − 1)
    w1 = isqrt(3 << 64) - (1 << 32)        # 2^32·(√3 − 1)
    assert int(rng.PHILOX_W0) == w0, ("Weyl constant 0", hex(int(rng.PHILOX_W0)), hex(w0))
    assert int(rng.PHILOX_W1) == w1, ("Weyl constant 1", hex(int(rng.PHILOX_W1)), hex(w1))
    c = np.arange(64, dtype=np.uint64)
    a = np.stack(rng.philox4x32_10(c, 7, 9, 11, 12345, 678))
    b = np.stack(rng.philox4x32_10(c, 7, 9, 11, (12345 + w0) & 0xFFFFFFFF, (678 + w1) & 0xFFFFFFFF))
    assert (a != b).any(axis=0).all()
