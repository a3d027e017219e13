"""Seeded synthetic ℓ1-regression inputs.

The paper's own regression experiments (§6.2, §6.3) use synthetic data: a
Gaussian design, a planted solution x*, heavy-tailed noise and a small fraction
of gross outliers.  The workloads below follow that recipe at the sizes the
GB300 build is measured on.  Every array is produced by numpy's PCG64 from an
explicit seed, so the CUDA side and the FP64 oracle read the same bytes.

BF16 matrices are returned as uint16 bit patterns (round-to-nearest-even from
float32), because numpy has no bfloat16 type; both sides widen the same bits.

Nothing here draws the method's own random variables (signs, hashes, Cauchy
scalings, the second projection, sampling uniforms): those come from the
counter-based generator that each side implements separately.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np


def r1_for(d: int) -> int:
    """Rows of Π1·X used by every workload: ⌈8·d·ln d⌉ with d = columns of A.

    The paper's theory sets r1 = α·d·log(d/δ) (§3.1) and its experiments use
    ⌈2 d log d⌉ (§6.1); the workloads fix the constant at 8 with a natural log.
    """
    return int(math.ceil(8.0 * d * math.log(d)))


def block_size_for(d: int) -> int:
    """FCT1 block size where a workload does not fix it: ⌈2·d·ln d⌉ (the experiments'
    choice, §6.1) rounded up to a power of two, as FCT1 needs.  The same rule gives the
    fixed values s = 64 at d = 8 and s = 1024 at d = 64."""
    return 1 << int(math.ceil(math.log2(2.0 * d * math.log(d))))


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    d: int
    s: int            # Hadamard block size of FCT1
    r2: int           # columns of the second Cauchy projection Π2
    coreset: float    # sampling parameter (expected coreset size bound)
    dtype: str        # storage type of A: "f32" or "bf16"
    design: str       # "gauss", "gauss_colscale", "gauss_t2rows", "gauss_spiky"
    noise: str        # "laplace_outliers" or "cauchy1"
    seed: int = 0
    problem_id: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def q(self) -> int:
        return self.d + 1

    @property
    def r1(self) -> int:
        return r1_for(self.d)

    def with_n(self, n: int) -> "Workload":
        return replace(self, n=int(n))


WORKLOADS = {
    # n=65536, d=8, Gaussian design, Laplace noise with 5% Cauchy(0,100) outliers.
    "gauss_n65536_d8": Workload("gauss_n65536_d8", 65536, 8, 64, 16, 2000.0,
                                "f32", "gauss", "laplace_outliers"),
    # n=2^22, d=16, columns scaled by 10^U(-2,2); the measured workload.
    "colscale_n4M_d16": Workload("colscale_n4M_d16", 1 << 22, 16, 256, 16, 20000.0,
                                 "f32", "gauss_colscale", "laplace_outliers"),
    # n=2^24, d=32, rows scaled by |Student-t(2)| magnitudes, A stored BF16.
    "t2rows_n16M_d32_bf16": Workload("t2rows_n16M_d32_bf16", 1 << 24, 32, 256, 32,
                                     100000.0, "bf16", "gauss_t2rows",
                                     "laplace_outliers"),
    # n=2^26, d=64, 0.1% of rows scaled by 1e3, Cauchy(0,1) noise.
    "spiky_n64M_d64": Workload("spiky_n64M_d64", 1 << 26, 64, 1024, 32, 100000.0,
                               "f32", "gauss_spiky", "cauchy1"),
}


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (nearest, ties to even); return uint16 bits."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    return ((u + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_f32(bits: np.ndarray) -> np.ndarray:
    """Widen bfloat16 bit patterns to float32 (exact)."""
    return (bits.astype(np.uint32) << 16).view(np.float32)


def _design(rng: np.random.Generator, w: Workload, n: int) -> np.ndarray:
    a = rng.standard_normal((n, w.d), dtype=np.float32)
    if w.design == "gauss":
        pass
    elif w.design == "gauss_colscale":
        scale = 10.0 ** rng.uniform(-2.0, 2.0, size=w.d)
        a *= scale.astype(np.float32)[None, :]
    elif w.design == "gauss_t2rows":
        mag = np.abs(rng.standard_t(2.0, size=n)).astype(np.float32)
        a *= mag[:, None]
    elif w.design == "gauss_spiky":
        spike = rng.random(n) < 1e-3
        a[spike] *= np.float32(1e3)
    else:
        raise ValueError(f"unknown design {w.design}")
    return a


def _noise(rng: np.random.Generator, w: Workload, n: int) -> np.ndarray:
    if w.noise == "laplace_outliers":
        e = rng.laplace(0.0, 1.0, size=n)
        out = rng.random(n) < 0.05
        e[out] = 100.0 * rng.standard_cauchy(size=int(out.sum()))
    elif w.noise == "cauchy1":
        e = rng.standard_cauchy(size=n)
    else:
        raise ValueError(f"unknown noise {w.noise}")
    return e


# Workloads at least this tall are drawn chunk-parallel (see make_problem).
PARALLEL_ROWS = 1 << 25


def _chunk(rng, w: Workload, m: int, x_star: np.ndarray):
    a = _design(rng, w, m)
    if w.dtype == "bf16":
        bits = f32_to_bf16_bits(a)
        a_stored = bf16_bits_to_f32(bits)
        stored = bits
    elif w.dtype == "f32":
        a_stored = a
        stored = a
    else:
        raise ValueError(w.dtype)
    e = _noise(rng, w, m)
    b = a_stored.astype(np.float64) @ x_star + e
    return stored, b.astype(np.float32)


def _make_parallel(w: Workload, chunk: int) -> dict:
    """Rows in chunks of `chunk`; chunk k is drawn from the k-th child of
    SeedSequence(seed), x* from PCG64(seed), so the result does not depend on how many
    threads draw the chunks."""
    import concurrent.futures as cf
    import os

    x_star = np.random.Generator(np.random.PCG64(w.seed)).standard_normal(w.d)
    nchunks = -(-w.n // chunk)
    kids = np.random.SeedSequence(w.seed).spawn(nchunks)
    A = np.empty((w.n, w.d), dtype=np.uint16 if w.dtype == "bf16" else np.float32)
    b = np.empty(w.n, dtype=np.float32)

    def fill(k):
        lo = k * chunk
        m = min(chunk, w.n - lo)
        a_k, b_k = _chunk(np.random.Generator(np.random.PCG64(kids[k])), w, m, x_star)
        A[lo:lo + m] = a_k
        b[lo:lo + m] = b_k

    with cf.ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(fill, range(nchunks)))
    return {"A": A, "b": b, "x_star": x_star, "w": w}


def make_problem(w: Workload | str, n: int | None = None, seed: int | None = None,
                 chunk: int = 1 << 22) -> dict:
    """Generate (A, b) for a workload.

    Returns a dict with
      A      (n, d) float32, or uint16 bfloat16 bits when w.dtype == "bf16"
      b      (n,) float32, b = A·x* + noise computed in float64 from the stored A
      x_star (d,) float64 planted solution
      w      the Workload (with n overridden if given)

    Workloads of PARALLEL_ROWS rows or more are drawn chunk by chunk from independent
    child seeds on several threads (one sequential stream would take minutes at 2^26
    rows); smaller ones from one sequential PCG64 stream.
    """
    if isinstance(w, str):
        w = WORKLOADS[w]
    if n is not None:
        w = w.with_n(n)
    if seed is not None:
        w = replace(w, seed=int(seed))
    if w.n >= PARALLEL_ROWS:
        return _make_parallel(w, chunk)
    rng = np.random.Generator(np.random.PCG64(w.seed))
    x_star = rng.standard_normal(w.d)
    n_total = w.n
    a_parts, b_parts = [], []
    done = 0
    while done < n_total:
        m = min(chunk, n_total - done)
        a_k, b_k = _chunk(rng, w, m, x_star)
        a_parts.append(a_k)
        b_parts.append(b_k)
        done += m
    A = a_parts[0] if len(a_parts) == 1 else np.concatenate(a_parts, axis=0)
    b = b_parts[0] if len(b_parts) == 1 else np.concatenate(b_parts)
    return {"A": A, "b": b, "x_star": x_star, "w": w}


def batched_block_size(d: int) -> int:
    """Hadamard block size of a batch member (block_size_for)."""
    return block_size_for(d)


def make_batched_problems(count: int = 256, seed: int = 0,
                          log2n_range=(12.0, 20.0), dims=(4, 8, 16, 32, 64),
                          r2: int = 16, coreset: float = 2000.0) -> list[dict]:
    """Many independent regressions of uneven n and d.

    n is log-uniform on [2^12, 2^20], d uniform over {4, 8, 16, 32, 64}; the
    design is Gaussian and the noise Laplace with 5% Cauchy(0,100) outliers.
    Each problem gets its own data seed and problem id; s follows
    batched_block_size(d).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for p in range(count):
        n = int(round(2.0 ** rng.uniform(*log2n_range)))
        d = int(rng.choice(dims))
        s = batched_block_size(d)
        w = Workload(f"batched_{p}", n, d, s, r2, coreset, "f32", "gauss",
                     "laplace_outliers", seed=seed * 100003 + p + 1, problem_id=p)
        out.append(make_problem(w))
    return out


def kappa_test_matrix(kind: str, n: int, d: int, seed: int = 0) -> np.ndarray:
    """The randomly generated ill-conditioned test matrices of the conditioning study (§6.1),
    as float32 (n × d):

    A1 = D1·G1·D2·G2 with D1 = diag(linspace(1, 10^4, n)), G1 ∈ R^{n×d} and G2 ∈ R^{d×d}
         standard Gaussian, D2 = diag(linspace(1, 10^4, d)): ill-conditioned, and its bottom
         rows tend to have high leverage;
    A2 = E·G with G ∈ R^{d×d} standard Gaussian and E ∈ R^{n×d} whose first d−1 rows are
         e_1 … e_{d−1} and whose other n−d+1 rows are all e_d: the first d−1 rows have very
         high leverage, the rest identical and very low.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "A1":
        g1 = rng.standard_normal((n, d))
        g2 = rng.standard_normal((d, d))
        d1 = np.linspace(1.0, 1e4, n)
        d2 = np.linspace(1.0, 1e4, d)
        a = (d1[:, None] * g1) @ (d2[:, None] * g2)
    elif kind == "A2":
        g = rng.standard_normal((d, d))
        a = np.empty((n, d))
        a[: d - 1] = g[: d - 1]
        a[d - 1:] = g[d - 1]
    else:
        raise ValueError(f"unknown test matrix {kind}")
    return a.astype(np.float32)


def canonical_design(n: int, d: int = 15, seed: int = 0, corrupt: float = 1e-3,
                     corrupt_scale: float = 1000.0) -> dict:
    """The imbalanced, corrupted canonical-row design of the large-scale experiment (§6.3):

    x* ∈ R^d standard Gaussian; every row of A is a canonical vector e_j, coordinate j
    (from 0) receiving twice as many rows as coordinate j + 1 (counts ⌊n·2^{d−1−j}/(2^d − 1)⌋,
    the rounding remainder going to coordinate 0), in a seeded random row order;
    b_i = corrupt_scale·ε_i with probability `corrupt`, else x*_{c_i} + ε_i, ε i.i.d.
    standard Laplace.  The paper's instance has n ≈ 5.24e9 and d = 15.

    Returns {"cols": (n,) int8 coordinate of each row, "b": (n,) float32, "x_star": (d,)
    float64, "counts": (d,) int64}; A itself (n × d, one 1 per row) is formed by the caller.
    """
    if not 1 <= d <= 127:
        raise ValueError("d must be in [1, 127]")
    rng = np.random.Generator(np.random.PCG64(seed))
    x_star = rng.standard_normal(d)
    counts = np.array([(n << (d - 1 - j)) // ((1 << d) - 1) for j in range(d)], dtype=np.int64)
    counts[0] += n - int(counts.sum())
    cols = np.repeat(np.arange(d, dtype=np.int8), counts)
    cols = rng.permutation(cols)
    eps = rng.laplace(0.0, 1.0, size=n)
    bad = rng.random(n) < corrupt
    b = np.where(bad, corrupt_scale * eps, x_star[cols] + eps).astype(np.float32)
    return {"cols": cols, "b": b, "x_star": x_star, "counts": counts}
