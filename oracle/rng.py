"""Counter-based random draws of the method, FP64 oracle side.

Test infrastructure: only the tests, the smoke check and the bench's CPU
baseline use this module.  The CUDA library carries its own, separately
written implementation of the same generator; the two share no code.

The generator is Philox4x32 with 10 rounds, as published by Salmon, Moraes,
Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC'11): a
128-bit counter and a 64-bit key; each round multiplies counter words 0 and 2
by two fixed 32-bit constants, mixes the high halves with the other two words
and the key, and the key advances by two Weyl constants between rounds.

How the method's random objects are drawn from it (these are this library's
conventions; the paper only fixes the distributions):

* stream 0, one call per global input row i, counter (i_lo, i_hi, problem, 0):
  words (o0, o1, o2, o3) give the hash bucket of the Hadamard virtual row
  h_H = ⌊o0·r1 / 2^32⌋, its Cauchy scale from k = o1 >> 8, the hash bucket of
  the identity virtual row h_I = ⌊o2·r1 / 2^32⌋, its Cauchy scale from
  k = o3 >> 8, and the row sign σ = −1 if (o3 & 1) else +1.  These are the
  columns of B, the diagonal of C (§3.1, FCT1 construction) and the ±1
  diagonal D applied before H̃.
* stream 1, call t with counter (t, 0, problem, 1): the entries 4t … 4t+3 of
  Π2 (row-major, q × r2) from the four words, each through k = word >> 8
  (Figure 2, step 3).
* stream 1 for the Gaussian Π2 of OptimizedFastCauchyRegression (Figure
  "mainOpt", step 4): call t gives the entries 2t and 2t+1 by the Box–Muller
  transform (Box and Muller, 1958) of two 53-bit uniforms in (0, 1),
  u1 from (o0, o1) and u2 from (o2, o3), each ((o_a >> 5)·2^26 + (o_b >> 6) + ½)·2^-53:
  ρ = √(−2 ln u1), entry 2t = ρ·cos(2π u2), entry 2t+1 = ρ·sin(2π u2).
* stream 4 for the slow Cauchy transform (the dense r1 × n Cauchy matrix of the
  theorem of Sohler and Woodruff quoted in §3, which §6.3 uses to condition):
  entry (r, i) of C, for global row i and r = 4g + w, is word w of the call with
  counter (i_lo, (i_hi mod 2^16) + g·2^16, problem, 4), through k = word >> 8.
* stream 2, call t with counter (t_lo, t_hi, problem, 2) for t = ⌊i/2⌋: the
  sampling uniform of row i is u = ((o_a >> 5)·2^26 + (o_b >> 6))·2^-53 with
  (a, b) = (0, 1) for even i and (2, 3) for odd i (Figure 2, step 7).

A standard Cauchy variate from a 24-bit integer k is the inverse CDF at the
cell midpoint u = (k + ½)·2^-24, written with the reflected argument so that it
is accurate near the poles: with m = 2k + 1 − 2^24 (odd) and
w = (2^24 − |m|)·2^-25 ∈ (0, ½], c = sign(m)·cos(πw)/sin(πw) = tan(π(u − ½)),
evaluated as sign(m)·sin(π|m|·2^-25)/sin(πw) (cos(πw) = sin(π(½ − w))).
"""
from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)

STREAM_FCT = 0
STREAM_PI2 = 1
STREAM_SAMPLE = 2
STREAM_REPLACE = 3
STREAM_SCT = 4
STREAM_FJLT = 5


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on arrays of 32-bit counter words (held in uint64).

    Returns the four output words as uint64 arrays holding 32-bit values.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def _row_counter(rows):
    rows = np.asarray(rows, dtype=np.int64).astype(np.uint64)
    return rows & MASK32, rows >> np.uint64(32)


def bucket(word, r1: int):
    """Uniform bucket in [0, r1) from a 32-bit word: ⌊word·r1 / 2^32⌋."""
    return ((np.asarray(word, dtype=np.uint64) * np.uint64(r1)) >> np.uint64(32)).astype(np.int64)


def cauchy_from_k(k):
    """Standard Cauchy from a 24-bit integer k (inverse CDF at (k+½)/2^24), FP64.

    With v = u − ½ and w = ½ − |v| (both exact), tan(πv) = sign(v)·cos(πw)/sin(πw)
    and cos(πw) = sin(π|v|), so c = sign(v)·sin(π|v|)/sin(πw): both sines take
    arguments in (0, π/2] and keep full relative accuracy at both ends.
    """
    k = np.asarray(k, dtype=np.int64)
    m = 2 * k + 1 - (1 << 24)
    w = ((1 << 24) - np.abs(m)).astype(np.float64) * 2.0 ** -25
    v = np.abs(m).astype(np.float64) * 2.0 ** -25
    sign = np.where(m > 0, 1.0, -1.0)
    return sign * np.sin(np.pi * v) / np.sin(np.pi * w)


def fct_draws(seed: int, problem_id: int, rows, r1: int) -> dict:
    """Draws of FCT1 for global input rows `rows` (stream 0).

    Returns hash_h, hash_i (int64 buckets), k_h, k_i (24-bit integers),
    cauchy_h, cauchy_i (FP64 variates) and sigma (±1.0).
    """
    k0, k1 = _key(seed)
    lo, hi = _row_counter(rows)
    o0, o1, o2, o3 = philox4x32_10(lo, hi, np.uint64(problem_id), np.uint64(STREAM_FCT), k0, k1)
    k_h = (o1 >> np.uint64(8)).astype(np.int64)
    k_i = (o3 >> np.uint64(8)).astype(np.int64)
    return {
        "hash_h": bucket(o0, r1),
        "hash_i": bucket(o2, r1),
        "k_h": k_h,
        "k_i": k_i,
        "cauchy_h": cauchy_from_k(k_h),
        "cauchy_i": cauchy_from_k(k_i),
        "sigma": np.where((o3 & np.uint64(1)) != 0, -1.0, 1.0),
    }


def pi2_matrix(seed: int, problem_id: int, q: int, r2: int) -> np.ndarray:
    """Π2 ∈ R^{q×r2} of independent standard Cauchys (Figure 2, step 3), stream 1."""
    k0, k1 = _key(seed)
    n_entries = q * r2
    calls = (n_entries + 3) // 4
    t = np.arange(calls, dtype=np.uint64)
    words = philox4x32_10(t, np.uint64(0), np.uint64(problem_id), np.uint64(STREAM_PI2), k0, k1)
    w = np.stack(words, axis=1).reshape(-1)[:n_entries]
    return cauchy_from_k((w >> np.uint64(8)).astype(np.int64)).reshape(q, r2)


def pi2_gaussian_matrix(seed: int, problem_id: int, q: int, r2: int) -> np.ndarray:
    """Π2 ∈ R^{q×r2} of independent standard Gaussians (Figure "mainOpt", step 4), stream 1."""
    k0, k1 = _key(seed)
    n_entries = q * r2
    calls = (n_entries + 1) // 2
    t = np.arange(calls, dtype=np.uint64)
    o0, o1, o2, o3 = philox4x32_10(t, np.uint64(0), np.uint64(problem_id), np.uint64(STREAM_PI2), k0, k1)

    def open_uniform(wa, wb):
        bits = ((wa >> np.uint64(5)) << np.uint64(26)) | (wb >> np.uint64(6))
        return (bits.astype(np.float64) + 0.5) * 2.0 ** -53

    u1 = open_uniform(o0, o1)
    u2 = open_uniform(o2, o3)
    rho = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * calls)
    z[0::2] = rho * np.cos(2.0 * np.pi * u2)
    z[1::2] = rho * np.sin(2.0 * np.pi * u2)
    return z[:n_entries].reshape(q, r2)


def sample_uniform_bits(seed: int, problem_id: int, rows) -> np.ndarray:
    """53-bit integers U_i with u_i = U_i·2^-53 for global rows `rows` (stream 2)."""
    k0, k1 = _key(seed)
    rows = np.asarray(rows, dtype=np.int64)
    t = rows >> 1
    lo, hi = _row_counter(t)
    o0, o1, o2, o3 = philox4x32_10(lo, hi, np.uint64(problem_id), np.uint64(STREAM_SAMPLE), k0, k1)
    odd = (rows & 1) == 1
    wa = np.where(odd, o2, o0)
    wb = np.where(odd, o3, o1)
    return ((wa >> np.uint64(5)) << np.uint64(26)) | (wb >> np.uint64(6))


def sample_uniforms(seed: int, problem_id: int, rows) -> np.ndarray:
    """Sampling uniforms u_i ∈ [0, 1) in FP64 (exact: 53-bit integers × 2^-53)."""
    return sample_uniform_bits(seed, problem_id, rows).astype(np.float64) * 2.0 ** -53


def replacement_uniforms(seed: int, problem_id: int, draws) -> np.ndarray:
    """Uniforms u_t ∈ [0, 1) of the with-replacement draws t (stream 3, one Philox call per
    pair of draws (2k, 2k+1): words (0, 1) for the even draw, (2, 3) for the odd one)."""
    k0, k1 = _key(seed)
    draws = np.asarray(draws, dtype=np.int64)
    lo, hi = _row_counter(draws >> 1)
    o0, o1, o2, o3 = philox4x32_10(lo, hi, np.uint64(problem_id), np.uint64(STREAM_REPLACE), k0, k1)
    odd = (draws & 1) == 1
    wa = np.where(odd, o2, o0)
    wb = np.where(odd, o3, o1)
    bits = ((wa >> np.uint64(5)) << np.uint64(26)) | (wb >> np.uint64(6))
    return bits.astype(np.float64) * 2.0 ** -53


def sct_matrix(seed: int, problem_id: int, rows, r1: int) -> np.ndarray:
    """The r1 × len(rows) block of the slow Cauchy transform's matrix C for global rows
    `rows` (stream 4): column i holds C[:, i], entry r = 4g + w from word w of call g."""
    k0, k1 = _key(seed)
    rows = np.asarray(rows, dtype=np.int64)
    lo, hi = _row_counter(rows)
    groups = (r1 + 3) // 4
    out = np.empty((4 * groups, rows.size))
    for g in range(groups):
        c1 = (hi & np.uint64(0xFFFF)) | (np.uint64(g) << np.uint64(16))
        words = philox4x32_10(lo, c1, np.uint64(problem_id), np.uint64(STREAM_SCT), k0, k1)
        for w in range(4):
            out[4 * g + w] = cauchy_from_k((words[w] >> np.uint64(8)).astype(np.int64))
    return out[:r1]


def fjlt_draws(seed: int, problem_id: int, t: int, s: int):
    """The draws of FCT2's s × t FJLT block G (stream 5, one G for every block): call i
    (counter (i, 0, problem_id, 5)) gives D_i = −1 when bit 0 of its word 0 is set (i < t)
    and the Hadamard row of G's row i, ⌊word1·t / 2^32⌋ (i < s).  Returns (D as ±1
    floats of length t, the s selected rows)."""
    k0, k1 = _key(seed)
    calls = np.arange(max(t, s), dtype=np.uint64)
    o0, o1, _, _ = philox4x32_10(calls, np.uint64(0), np.uint64(problem_id), np.uint64(STREAM_FJLT), k0, k1)
    D = np.where((o0[:t] & np.uint64(1)) == 1, -1.0, 1.0)
    sel = ((o1[:s] * np.uint64(t)) >> np.uint64(32)).astype(np.int64)
    return D, sel
