"""Plain FP64 CPU oracle of the Fast Cauchy Transform ℓ1-regression hot path.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the tests, the package's
smoke check and the bench's CPU-baseline leg may import or run anything in
this package.  The CUDA library never calls it and shares no code, header,
table or constant generator with it; the two sides meet only through the
seeded input generators in `synth/` and through the published definition of
the counter-based generator, which each side implements on its own.

Modules, in the order of the method (Figure 2, FastCauchyRegression):
  rng        Philox4x32-10 draws: signs, hash buckets, Cauchy scales, Π2, uniforms, dense C
  fct        Π1·X = 4·B·C·H̃·D·X (§3.1), per block and as an explicit dense product
  sct        Π1·X = (4/r1)·C·X, the slow Cauchy transform (§3, used to condition in §6.3)
  condition  QR of Π1·X with positive diag(R), M = R⁻¹·Π2 (steps 2-3)
  leverage   λ_i = lower median_j |(X·M)_ij| and exact ‖U_(i)‖₁ (steps 4-5)
  sampling   p̂_i = min(1, τ·λ_i), τ = m_s/Σλ, Bernoulli keep u_i < p̂_i (steps 6-7)
  solve      weighted LAD by LP, brute force and weighted median (step 8)
  quality    κ̄₁(U), the conditioning metric of §6.1, from d exact ℓ1 regressions
  pipeline   the steps chained, with every intermediate returned

Parity status: every function above is pinned by the CPU tests in
tests/test_oracle_*.py against closed forms, invariants, brute force or the
paper's lemmas.  The exact bit pattern of Philox4x32-10 is pinned only
statistically and structurally (no published known-answer vectors are
available offline); the GPU side is checked against it bit for bit.
"""
