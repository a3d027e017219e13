// Conditioning (Figure 1, step 2; Figure 2, steps 2-3): FP64 QR of the small
// r1 × q matrix Π1·X with positive diag(R), then M = R⁻¹·Π2 with Π2 a q × r2
// matrix of independent standard Cauchys.  M is formed first (q × r2) so that
// phase 2 multiplies X by one skinny matrix, the order the paper's running-time
// argument uses (proof of the fast ℓ1 regression theorem: R⁻¹Π2 before X·(R⁻¹Π2)).
//
// The QR is CholeskyQR2 (below) in two launches over many thread blocks.  When
// its blocks do not fit in shared memory (q near 129), a single thread block runs
// Householder reflections on a column-major FP64 copy of Π1·X instead, held in
// shared memory when it fits (r1·q·8 bytes ≤ 160 KB) and in the workspace
// (L2-resident) otherwise.  CholeskyQR2 squares the condition number in its Gram
// matrices and breaks down when Π1·X is conditioned worse than about 1e7-1e8; a
// breakdown (a Cholesky pivot that is not positive, or a non-finite R or M) is recorded
// in the status block, and the Householder kernel, enqueued after the two passes, then
// redoes the step (it returns at once otherwise), so the decision stays on the device.
#include <stddef.h>

#include <algorithm>

#include "l1s_common.cuh"

namespace l1s {

constexpr int kCondThreads = 512;
constexpr size_t kCondSmemMax = 160 * 1024;

// Column k of Π1·X counts as dependent on columns 0..k−1 when |R_kk| ≤ kRankTol·‖(Π1X)_{:,k}‖₂:
// Π1·X carries FP32 rounding of about 1e-7 of its terms, so a smaller residual cannot be told apart
// from an exactly dependent column.
constexpr double kRankTol = 1e-5;

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Sum over the block in a fixed order (warp trees, then warp 0 over the warp sums).
__device__ double block_sum_f64(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_f64(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < nw ? scratch[lane] : 0.0;
    t = warp_sum_f64(t);
    if (lane == 0) scratch[32] = t;
  }
  __syncthreads();
  return scratch[32];
}


struct CondArgs {
  const float* pix;   // r1 × q row-major FP32
  int r1, q, r2;
  Key2 key;
  uint32_t problem;
  double* work;       // r1 × q column-major FP64 (workspace copy, used when it does not fit in shared memory)
  int in_smem;
  double* R;          // q × q row-major (workspace)
  double* M64;        // q × r2 row-major (workspace)
  float* M32;         // q × r2 row-major (workspace)
  double* pi2;        // q × r2 (workspace)
  double* R_user;     // optional copies
  double* M_user;
  uint32_t* flags;
  int pi2_gauss;      // 1: Gaussian Π2 (OptimizedFastCauchyRegression)
  const uint32_t* only_if;   // non-NULL: run only when *only_if != 0 (CholeskyQR2 broke down)
};

__global__ void __launch_bounds__(kCondThreads) condition_kernel(const CondArgs a) {
  if (a.only_if && *a.only_if == 0u) return;
  extern __shared__ __align__(16) double cond_smem[];
  __shared__ double scratch[33];
  __shared__ double s_vtv;
  __shared__ int s_rank_bad;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int r1 = a.r1, q = a.q;
  double* W = a.in_smem ? cond_smem : a.work;

  for (int i = tid; i < r1 * q; i += nthr) {
    const int r = i / q, c = i - r * q;
    W[static_cast<size_t>(c) * r1 + r] = static_cast<double>(a.pix[i]);
  }
  for (int e = tid; e < q * a.r2; e += nthr) a.pi2[e] = pi2_value(a.key, a.problem, e, a.pi2_gauss);
  if (tid == 0) s_rank_bad = 0;
  __syncthreads();

  // Householder: column k is reflected onto α_k·e_k, α_k = −sign(a_kk)·‖a_k[k:]‖.
  for (int k = 0; k < q; ++k) {
    double* col = W + static_cast<size_t>(k) * r1;
    double part = 0.0;
    for (int i = k + tid; i < r1; i += nthr) part += col[i] * col[i];
    const double nrm2 = block_sum_f64(part, scratch);
    if (tid == 0) {
      const double akk = col[k];
      const double nrm = sqrt(nrm2);
      const double alpha = akk >= 0.0 ? -nrm : nrm;
      const double vk = akk - alpha;
      s_vtv = nrm2 - akk * akk + vk * vk;  // ‖v‖² with v = a_k[k:] − α e_k
      col[k] = vk;
      a.R[k * q + k] = alpha;
      // The reflections are orthogonal, so ‖(Π1X)_{:,k}‖² = ‖a_k[k:]‖² + Σ_{i<k} R_ik².
      double col2 = nrm2;
      for (int i = 0; i < k; ++i) col2 += a.R[i * q + k] * a.R[i * q + k];
      if (!(nrm > kRankTol * sqrt(col2)) || !isfinite(col2)) s_rank_bad = 1;
    }
    __syncthreads();
    const double vtv = s_vtv;
    for (int j = k + 1 + warp; j < q; j += nwarps) {
      double* cj = W + static_cast<size_t>(j) * r1;
      double dot = 0.0;
      for (int i = k + lane; i < r1; i += 32) dot += col[i] * cj[i];
      dot = warp_sum_f64(dot);
      const double f = vtv > 0.0 ? 2.0 * dot / vtv : 0.0;
      for (int i = k + lane; i < r1; i += 32) cj[i] -= f * col[i];
    }
    __syncthreads();
    // Row k of R: entry k of each reflected trailing column.
    for (int j = k + 1 + tid; j < q; j += nthr) a.R[k * q + j] = W[static_cast<size_t>(j) * r1 + k];
    __syncthreads();
  }

  // Positive diagonal, strictly lower part zero, rank test.
  for (int i = tid; i < q * q; i += nthr) {
    const int r = i / q, c = i - r * q;
    if (c < r) a.R[i] = 0.0;
  }
  __syncthreads();
  for (int i = tid; i < q * q; i += nthr) {
    const int r = i / q, c = i - r * q;
    if (c >= r && a.R[r * q + r] < 0.0 && c != r) a.R[i] = -a.R[i];
  }
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < q; ++k) a.R[k * q + k] = fabs(a.R[k * q + k]);
    if (s_rank_bad) raise_flag(a.flags, L1S_ERR_RANK_DEFICIENT);
  }
  __syncthreads();

  // M = R⁻¹·Π2 by back substitution, one column of Π2 per thread.
  for (int c = tid; c < a.r2; c += nthr) {
    for (int k = q - 1; k >= 0; --k) {
      double acc = a.pi2[k * a.r2 + c];
      for (int j = k + 1; j < q; ++j) acc -= a.R[k * q + j] * a.M64[j * a.r2 + c];
      a.M64[k * a.r2 + c] = acc / a.R[k * q + k];
    }
  }
  __syncthreads();
  for (int e = tid; e < q * a.r2; e += nthr) {
    const double m = a.M64[e];
    a.M32[e] = static_cast<float>(m);
    if (a.M_user) a.M_user[e] = m;
  }
  if (a.R_user)
    for (int e = tid; e < q * q; e += nthr) a.R_user[e] = a.R[e];
}

// ----------------------------------------------------------------- CholeskyQR2
// R is also the Cholesky factor of the Gram matrix (Π1X)ᵀ(Π1X), and applying the
// Cholesky step twice (R1 from the Gram of Π1X, R2 from the Gram of Π1X·R1⁻¹,
// R = R2·R1) gives a QR factor accurate to FP64 rounding whenever the condition
// number is below about 1e7 — far past what an FP32-accumulated Π1X resolves (the
// rank test flags columns dependent to 1e-5).  The Gram products spread over thread
// blocks; the last block to finish (an atomic ticket, no waiting) sums the partials in
// a fixed order and factors the q×q matrix.  Two launches: pass 0 (Gram of Π1X → R1),
// pass 1 (rows of Π1X·R1⁻¹ by forward substitution, their Gram → R2, then R = R2·R1
// and M = R⁻¹Π2).  Π2 is drawn by the phase-1 reduction when the whole pass runs.
//
// FP64 arithmetic on this part is slow (a dependent FMA takes ~64 cycles, a division
// ~430, a square root ~670, and a full-warp FP64 instruction holds its sub-partition
// for ~80 cycles), so the serial parts avoid divisions and square roots — reciprocals
// and reciprocal square roots come from FP32 estimates refined by Newton steps in
// FP64, and every division by a diagonal entry is a multiplication by its stored
// reciprocal — and run right-looking (each step finishes one row or column and updates
// the rest in parallel), so the dependent chain per step is a few operations long.
constexpr int kGramThreads = 256;
// Blocks per first-level group of the partial sums: one group (a single level) for
// q ≤ 32, groups of 8 for wider X, whose partials are long.
__host__ __device__ __forceinline__ int cond2_group_size(int q, int blocks) { return q > 32 ? 8 : blocks; }

struct Cond2Args {
  const float* pix;      // r1 × q row-major FP32
  int r1, q, r2;
  int rows_per_block;
  Key2 key;
  uint32_t problem;
  double* partials;      // [gridDim.x][q(q+1)/2], then the group sums
  unsigned int* ticket;  // group tickets [groups], then the final ticket (zero before each pass)
  double* R1;            // q × q (pass 0 → pass 1)
  double* R1dinv;        // q: 1 / (R1)_kk
  double* colnorm;       // q: ‖(Π1X)_:k‖₂
  double* R;             // q × q row-major (output)
  double* M64;           // q × r2
  float* M32;
  double* pi2;
  double* R_user;
  double* M_user;
  uint32_t* flags;
  uint32_t* breakdown;   // set when a Cholesky factorisation fails or R, M are not finite
  int pi2_ready;         // 1: Π2 is already in pi2 (drawn by the phase-1 reduction)
  int pi2_gauss;         // 1: Gaussian Π2 (OptimizedFastCauchyRegression)
};

// On this part every FP64 warp instruction occupies its SM sub-partition for tens of
// cycles, so the serial steps below keep their FP64 chains short and spread the
// independent work over all warps of the block.

// 1/x and 1/√x for x > 0 in FP64: an FP32 estimate of the mantissa part (the exponent is
// split off first, so any normal FP64 x works), then Newton steps in FP64 — for 1/x
// y ← y + y·(1 − x·y), for 1/√x y ← y·(3/2 − (x/2)·y²).  Each step doubles the number of
// correct bits: one leaves a relative error near 1e-13, two reach FP64 rounding.
__device__ __forceinline__ double rcp_f64(double x, int steps) {
  int e;
  const double m = frexp(x, &e);                         // x = m·2^e, m ∈ [1/2, 1)
  double y = ldexp(static_cast<double>(__frcp_rn(static_cast<float>(m))), -e);
  for (int i = 0; i < steps; ++i) y = fma(y, fma(-x, y, 1.0), y);
  return y;
}

__device__ __forceinline__ double rsqrt_f64(double x, int steps) {
  int e;
  double m = frexp(x, &e);
  if (e & 1) {                                           // make the exponent even
    m *= 2.0;
    e -= 1;
  }
  double y = ldexp(static_cast<double>(rsqrtf(static_cast<float>(m))), -e / 2);
  const double h = 0.5 * x;
  for (int i = 0; i < steps; ++i) y = y * fma(-h, y * y, 1.5);
  return y;
}

// Cholesky of the symmetric q×q matrix G (row-major, upper triangle, shared memory) by
// all threads of the block, in the square-root-free form G = LᵀDL first: step k
// subtracts G_ki·G_kj/d_k from the trailing triangle (warps 1 and up, a row per warp)
// while thread 0 forms the next pivot — the same FMA the update would apply to
// G_{k+1,k+1} — and its reciprocal, so the serial chain per step is one reciprocal.  Then R_kj = G_kj/√d_k for all
// entries at once, and dinv[k] = 1/R_kk.  s_r holds q doubles.  Returns false when a
// pivot is not positive.
// chain_steps Newton steps refine the pivots' reciprocals on the serial chain (0 leaves
// them FP32-accurate, which only perturbs G by about 1e-7 relative: enough for a
// preconditioner); the final 1/√d_k always take two.
// Threads [0, nt) take part (nt a multiple of 32: 128 for q ≤ 32, where four warps are
// enough and a named barrier is cheaper, else the whole block).
__device__ __forceinline__ void sync_first(int nt) {
  if (nt == static_cast<int>(blockDim.x)) __syncthreads();
  else named_barrier(1, nt);
}

__device__ bool block_cholesky(double* G, double* R, double* dinv, double* s_r, int q, int chain_steps, int nt) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = nt >> 5;
  const int steps = chain_steps;
  bool ok = true;
  if (t == 0) {
    const double a = G[0];
    s_r[0] = rcp_f64(fmax(a, 1e-300), steps);
    if (!(a > 0.0) || !isfinite(a)) ok = false;
  }
  sync_first(nt);
  for (int k = 0; k + 1 < q; ++k) {
    const double r = s_r[k];
    if (t == 0) {
      const double g = G[k * q + k + 1];
      const double an = fma(-(g * r), g, G[(k + 1) * q + k + 1]);
      G[(k + 1) * q + k + 1] = an;   // the one trailing entry the other warps leave to thread 0
      s_r[k + 1] = rcp_f64(fmax(an, 1e-300), steps);
      if (!(an > 0.0) || !isfinite(an)) ok = false;
    } else if (warp > 0) {
      const int w = q - k - 1;
      if (q <= 32) {
        // small trailing block: its w×w entries spread flat over warps 1 and up
        for (int e = t - 32; e < w * w; e += nt - 32) {
          const int i = k + 1 + e / w, j = k + 1 + e % w;
          if (j >= i && (j != k + 1 || i != k + 1))
            G[i * q + j] = fma(-(G[k * q + i] * r), G[k * q + j], G[i * q + j]);
        }
      } else {
        // rows i = k+1.. of the trailing upper triangle, one row per warp, lanes over j ≥ i
        for (int i = k + warp; i < q; i += nw - 1) {
          const double gki = G[k * q + i] * r;
          for (int j = i + lane; j < q; j += 32)
            if (j != k + 1 || i != k + 1) G[i * q + j] = fma(-gki, G[k * q + j], G[i * q + j]);
        }
      }
    }
    sync_first(nt);
  }
  // R_kj = G_kj/√d_k (d_k = G_kk after its step), zero below the diagonal
  for (int k = t; k < q; k += nt) dinv[k] = rsqrt_f64(fmax(G[k * q + k], 1e-300), 2);
  sync_first(nt);
  for (int e = t; e < q * q; e += nt) {
    const int i = e / q, j = e - i * q;
    R[e] = j < i ? 0.0 : G[e] * dinv[i];
  }
  sync_first(nt);
  return ok;
}

// Right-looking back substitution in place, all threads of the block: on entry M holds
// B (q × r2), on return R⁻¹·B for the upper-triangular R (row-major q × q) with dinv[k] =
// 1/R_kk: step k finishes row k, then every row above subtracts R_jk·M_k·.
__device__ void block_back_subst(const double* R, const double* dinv, double* M, int q, int r2, int nt) {
  const int t = threadIdx.x;
  for (int k = q - 1; k >= 0; --k) {
    for (int c = t; c < r2; c += nt) M[k * r2 + c] *= dinv[k];
    sync_first(nt);
    for (int e = t; e < k * r2; e += nt) {
      const int j = e / r2, c = e - j * r2;
      M[e] = fma(-R[j * q + k], M[k * r2 + c], M[e]);
    }
    sync_first(nt);
  }
}

// Σ_{i<count} a[i·stride] with four independent accumulators, combined in a fixed order.
__device__ __forceinline__ double sum4(const double* a, int count, size_t stride) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = 0;
  for (; i + 3 < count; i += 4) {
    s0 += a[static_cast<size_t>(i) * stride];
    s1 += a[static_cast<size_t>(i + 1) * stride];
    s2 += a[static_cast<size_t>(i + 2) * stride];
    s3 += a[static_cast<size_t>(i + 3) * stride];
  }
  for (; i < count; ++i) s0 += a[static_cast<size_t>(i) * stride];
  return (s0 + s1) + (s2 + s3);
}

__device__ __forceinline__ void pair_index(int e, int q, int& j, int& l) {
  int row = 0, left = e;
  while (left >= q - row) {
    left -= q - row;
    ++row;
  }
  j = row;
  l = row + left;
}

// Shared memory of a cond2 block (doubles): rows | R1 | dinv | dn | Rc | inv | R | Π2 | M.
struct Cond2Smem {
  int rows, r1q, dinv, dn, Rc, inv, R, P, M, total;
  __host__ __device__ Cond2Smem(int rpb, int q, int r2) {
    rows = 0;
    r1q = rows + (rpb > q ? rpb : q) * q;
    dinv = r1q + q * q;
    dn = dinv + q;
    Rc = dn + q;
    inv = Rc + q * q;
    R = inv + 2 * q;
    P = R + q * q;
    M = P + q * r2;
    total = M + q * r2;
  }
};

template <int PASS>
__global__ void __launch_bounds__(kGramThreads) cond2_kernel(const Cond2Args a) {
  extern __shared__ __align__(16) double sm2[];
  __shared__ int s_last;
  __shared__ int s_ok;
  const int q = a.q, tid = threadIdx.x, lane = tid & 31;
  const int ne = q * (q + 1) / 2;
  const int r_lo = blockIdx.x * a.rows_per_block;
  const int r_hi = min(a.r1, r_lo + a.rows_per_block);
  const int nrows = r_hi - r_lo;
  const Cond2Smem L(a.rows_per_block, q, a.r2);
  double* rows = sm2 + L.rows;                // this block's rows, later the Gram
  double* R1s = sm2 + L.r1q;                  // pass 1: R1
  double* dinv = sm2 + L.dinv;                // pass 1: 1/(R1)_kk
  double* dn = sm2 + L.dn;                    // reciprocals of this pass's factor
  if (PASS == 0) {
    // Π2, unless the phase-1 reduction drew it, spread over all blocks.
    if (!a.pi2_ready)
      for (int e = blockIdx.x * blockDim.x + tid; e < q * a.r2; e += gridDim.x * blockDim.x)
        a.pi2[e] = pi2_value(a.key, a.problem, e, a.pi2_gauss);
  } else {
    for (int e = tid; e < q * q; e += blockDim.x) R1s[e] = a.R1[e];
    for (int e = tid; e < q; e += blockDim.x) dinv[e] = a.R1dinv[e];
  }
  for (int e = tid; e < nrows * q; e += blockDim.x)
    rows[e] = static_cast<double>(a.pix[static_cast<size_t>(r_lo) * q + e]);
  __syncthreads();
  if (PASS == 1) {
    // y·R1 = x by forward substitution, right-looking: lane c of a warp holds the running
    // value of column c of up to three rows; at step k the lane holding column k
    // finishes y_k (a shuffle broadcasts it) and every later column subtracts y_k·R1_kc.
    // The three rows of a warp are independent chains that overlap.  (q > 64: one row per
    // thread.)
    if (q <= 32) {
      const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
      for (int i0 = warp; i0 < nrows; i0 += 3 * nw) {
        double acc[3];
        bool live[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int i = i0 + u * nw;
          live[u] = i < nrows;
          acc[u] = (live[u] && lane < q) ? rows[i * q + lane] : 0.0;
        }
        for (int k = 0; k < q; ++k) {
          const double rk = lane < q ? R1s[k * q + lane] : 0.0;
          const double dk = dinv[k];
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            const double yk = __shfl_sync(0xffffffffu, acc[u], k) * dk;
            if (lane == k) acc[u] = yk;
            else if (lane > k) acc[u] = fma(-yk, rk, acc[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (live[u] && lane < q) rows[(i0 + u * nw) * q + lane] = acc[u];
      }
    } else if (q <= 64) {
      // lane c holds columns c and c + 32
      const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
      const int c1 = lane + 32;
      for (int i0 = warp; i0 < nrows; i0 += 3 * nw) {
        double acc[3], acc1[3];
        bool live[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int i = i0 + u * nw;
          live[u] = i < nrows;
          acc[u] = (live[u] && lane < q) ? rows[i * q + lane] : 0.0;
          acc1[u] = (live[u] && c1 < q) ? rows[i * q + c1] : 0.0;
        }
        for (int k = 0; k < q; ++k) {
          const double rk = lane < q ? R1s[k * q + lane] : 0.0;
          const double rk1 = c1 < q ? R1s[k * q + c1] : 0.0;
          const double dk = dinv[k];
          const bool hi = k >= 32;
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            const double src = hi ? acc1[u] : acc[u];
            const double yk = __shfl_sync(0xffffffffu, src, k & 31) * dk;
            if (!hi) {
              if (lane == k) acc[u] = yk;
              else if (lane > k) acc[u] = fma(-yk, rk, acc[u]);
            }
            if (c1 == k) acc1[u] = yk;
            else if (c1 > k) acc1[u] = fma(-yk, rk1, acc1[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          if (live[u] && lane < q) rows[(i0 + u * nw) * q + lane] = acc[u];
          if (live[u] && c1 < q) rows[(i0 + u * nw) * q + c1] = acc1[u];
        }
      }
    } else {
      for (int i = tid; i < nrows; i += blockDim.x) {
        double* y = rows + i * q;
        for (int c = 0; c < q; ++c) {
          double s0 = y[c], s1 = 0.0, s2 = 0.0, s3 = 0.0;
          int k = 0;
          for (; k + 3 < c; k += 4) {
            s0 = fma(-y[k], R1s[k * q + c], s0);
            s1 = fma(-y[k + 1], R1s[(k + 1) * q + c], s1);
            s2 = fma(-y[k + 2], R1s[(k + 2) * q + c], s2);
            s3 = fma(-y[k + 3], R1s[(k + 3) * q + c], s3);
          }
          for (; k < c; ++k) s0 = fma(-y[k], R1s[k * q + c], s0);
          y[c] = ((s0 + s1) + (s2 + s3)) * dinv[c];
        }
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < ne; e += blockDim.x) {
    int j, l;
    pair_index(e, q, j, l);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 3 < nrows; i += 4) {
      s0 = fma(rows[i * q + j], rows[i * q + l], s0);
      s1 = fma(rows[(i + 1) * q + j], rows[(i + 1) * q + l], s1);
      s2 = fma(rows[(i + 2) * q + j], rows[(i + 2) * q + l], s2);
      s3 = fma(rows[(i + 3) * q + j], rows[(i + 3) * q + l], s3);
    }
    for (; i < nrows; ++i) s0 = fma(rows[i * q + j], rows[i * q + l], s0);
    a.partials[static_cast<size_t>(blockIdx.x) * ne + e] = (s0 + s1) + (s2 + s3);
  }
  // Two-level fixed-order sum of the partials: the last block of each group of
  // kCondGroup blocks adds its group's partials; the last group to finish adds the
  // group sums (both in block order, so the result does not depend on scheduling).
  const int gsz = cond2_group_size(q, gridDim.x);
  const int groups = (gridDim.x + gsz - 1) / gsz;
  const int g = blockIdx.x / gsz;
  const int g_lo = g * gsz, g_n = min(gsz, static_cast<int>(gridDim.x) - g_lo);
  double* gsum = a.partials + static_cast<size_t>(gridDim.x) * ne;   // [groups][ne]
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(a.ticket + g, 1u) == static_cast<unsigned>(g_n - 1)) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (groups > 1) {
    for (int e = tid; e < ne; e += blockDim.x)
      gsum[static_cast<size_t>(g) * ne + e] = sum4(a.partials + static_cast<size_t>(g_lo) * ne + e, g_n, ne);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(a.ticket + groups, 1u) == static_cast<unsigned>(groups - 1)) ? 1 : 0;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
  }
  // ---- last group: the group sums (or, with one group, the partials), then the q×q work
  double* Gs = rows;
  const double* src = groups > 1 ? gsum : a.partials;
  const int nsrc = groups > 1 ? groups : static_cast<int>(gridDim.x);
  for (int e = tid; e < ne; e += blockDim.x) {
    const double v = sum4(src + e, nsrc, ne);
    int j, l;
    pair_index(e, q, j, l);
    Gs[j * q + l] = v;
    Gs[l * q + j] = v;
    if (PASS == 0 && j == l) a.colnorm[j] = sqrt(v);
  }
  double* Ps = sm2 + L.P;
  double* Rc = sm2 + L.Rc;                    // this pass's Cholesky factor
  if (PASS == 1)
    for (int e = tid; e < q * a.r2; e += blockDim.x) Ps[e] = a.pi2[e];
  __syncthreads();
  const int nt = q > 32 ? static_cast<int>(blockDim.x) : 128;
  if (tid < nt) {
    // FP32-accurate pivot reciprocals suffice for R1, which only preconditions pass 1
    const bool ok = block_cholesky(Gs, Rc, dn, sm2 + L.inv, q, PASS == 0 ? 0 : 2, nt);
    if (tid == 0) s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  if (PASS == 0) {
    if (tid == 0) *a.breakdown = s_ok ? 0u : 1u;     // the Householder kernel redoes the step
    for (int e = tid; e < q * q; e += blockDim.x) a.R1[e] = Rc[e];
    for (int e = tid; e < q; e += blockDim.x) a.R1dinv[e] = dn[e];
  } else {
    double* Rs = sm2 + L.R;
    double* Ms = sm2 + L.M;
    const bool broke0 = *a.breakdown != 0u || !s_ok;
    if (tid < 32) {
      // rank test over the columns, one lane per column: R_kk = (R2)_kk·(R1)_kk (skipped after a
      // breakdown: the Householder kernel runs its own)
      bool bad = false;
      for (int k = tid; k < q; k += 32) {
        const double rkk = Rc[k * q + k] * R1s[k * q + k];
        if (!(rkk > kRankTol * a.colnorm[k]) || !isfinite(rkk)) bad = true;
      }
      if (__any_sync(0xffffffffu, bad) && !broke0) {
        if (tid == 0) raise_flag(a.flags, L1S_ERR_RANK_DEFICIENT);
      }
      if (broke0 && tid == 0) *a.breakdown = 1u;
    }
    // M = R⁻¹·Π2.  q ≤ 32: R = R2·R1 first, then one right-looking back substitution;
    // wider X: R1⁻¹·(R2⁻¹·Π2) by two, which avoids the q³ product.
    const bool small = q <= 32;
    if (small) {
      for (int e = tid; e < q * q; e += blockDim.x) {
        const int i = e / q, j = e - i * q;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int k = i;
        for (; k + 3 <= j; k += 4) {
          s0 = fma(Rc[i * q + k], R1s[k * q + j], s0);
          s1 = fma(Rc[i * q + k + 1], R1s[(k + 1) * q + j], s1);
          s2 = fma(Rc[i * q + k + 2], R1s[(k + 2) * q + j], s2);
          s3 = fma(Rc[i * q + k + 3], R1s[(k + 3) * q + j], s3);
        }
        for (; k <= j; ++k) s0 = fma(Rc[i * q + k], R1s[k * q + j], s0);
        Rs[e] = j < i ? 0.0 : (s0 + s1) + (s2 + s3);
      }
      for (int k = tid; k < q; k += blockDim.x) dn[k] = dn[k] * dinv[k];   // 1/(R2_kk·R1_kk)
    }
    for (int e = tid; e < q * a.r2; e += blockDim.x) Ms[e] = Ps[e];
    __syncthreads();
    if (tid < nt) {
      if (small) {
        block_back_subst(Rs, dn, Ms, q, a.r2, nt);
      } else {
        block_back_subst(Rc, dn, Ms, q, a.r2, nt);
        block_back_subst(R1s, dinv, Ms, q, a.r2, nt);
      }
    }
    __syncthreads();
    for (int e = tid; e < q * a.r2; e += blockDim.x) {
      const double m = Ms[e];
      a.M64[e] = m;
      a.M32[e] = static_cast<float>(m);
      if (a.M_user) a.M_user[e] = m;
      if (!isfinite(m)) *a.breakdown = 1u;
    }
    if (a.R_user && small) {
      for (int e = tid; e < q * q; e += blockDim.x) {
        a.R[e] = Rs[e];
        a.R_user[e] = Rs[e];
      }
    } else if (a.R_user) {
      // R = R2·R1 (both upper triangular), only when the caller asks for it
      for (int e = tid; e < q * q; e += blockDim.x) {
        const int i = e / q, j = e - i * q;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int k = i;
        for (; k + 3 <= j; k += 4) {
          s0 = fma(Rc[i * q + k], R1s[k * q + j], s0);
          s1 = fma(Rc[i * q + k + 1], R1s[(k + 1) * q + j], s1);
          s2 = fma(Rc[i * q + k + 2], R1s[(k + 2) * q + j], s2);
          s3 = fma(Rc[i * q + k + 3], R1s[(k + 3) * q + j], s3);
        }
        for (; k <= j; ++k) s0 = fma(Rc[i * q + k], R1s[k * q + j], s0);
        const double v = j < i ? 0.0 : (s0 + s1) + (s2 + s3);
        Rs[e] = v;
        a.R[e] = v;
        a.R_user[e] = v;
      }
    }
  }
  for (int k = tid; k <= groups; k += blockDim.x) a.ticket[k] = 0u;   // ready for the next pass
}

__global__ void pi2_kernel(Key2 key, uint32_t problem, int total, int gaussian, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < total) out[e] = pi2_value(key, problem, e, gaussian);
}

// Rows of Π1X per block of the Gram passes: for q ≤ 32 at least q and at most 32
// blocks; wider X (whose Gram costs r1·q²/2 FP64 FMAs) spreads over about 128 blocks.
static int cond2_rows_per_block(int r1, int q) {
  if (q > 32) return std::max(4, (r1 + 127) / 128);
  return std::max(q, (r1 + 31) / 32);
}

size_t cond2_scratch_bytes(int r1, int q, int sms) {
  (void)sms;
  const int rpb = cond2_rows_per_block(r1, q);
  const int blocks = (r1 + rpb - 1) / rpb;
  const int groups = (blocks + cond2_group_size(q, blocks) - 1) / cond2_group_size(q, blocks);
  return sizeof(double) * (static_cast<size_t>(blocks + groups) * (q * (q + 1) / 2) + q * q + 2 * q) +
         sizeof(unsigned int) * (groups + 1) + 256;
}

bool launch_condition_householder(const Plan& pl, const float* pix, const l1s_params* p, double* R_user,
                                  double* M_user, unsigned char* ws, cudaStream_t st,
                                  const uint32_t* only_if = nullptr);

bool launch_condition(const Plan& pl, const float* pix, const l1s_params* p, double* R_user,
                      double* M_user, unsigned char* ws, cudaStream_t st, bool pi2_ready) {
  // Wide X (q near 129) does not fit the CholeskyQR2 blocks in shared memory: one block
  // of Householder reflections on a workspace copy handles it instead.
  if (sizeof(double) * static_cast<size_t>(Cond2Smem(cond2_rows_per_block(pl.r1, pl.q), pl.q, pl.r2).total) >
      static_cast<size_t>(device_info().max_smem_optin))
    return launch_condition_householder(pl, pix, p, R_user, M_user, ws, st);
  Cond2Args a;
  a.pix = pix;
  a.r1 = pl.r1;
  a.q = pl.q;
  a.r2 = pl.r2;
  a.rows_per_block = cond2_rows_per_block(pl.r1, pl.q);
  const int grid = (pl.r1 + a.rows_per_block - 1) / a.rows_per_block;
  a.key = make_key(p->seed);
  a.problem = p->problem_id;
  double* scratch = reinterpret_cast<double*>(ws + pl.off_qr);
  const int ne = pl.q * (pl.q + 1) / 2;
  const int groups = (grid + cond2_group_size(pl.q, grid) - 1) / cond2_group_size(pl.q, grid);
  a.partials = scratch;
  a.R1 = scratch + static_cast<size_t>(grid + groups) * ne;
  a.R1dinv = a.R1 + pl.q * pl.q;
  a.colnorm = a.R1dinv + pl.q;
  a.ticket = reinterpret_cast<unsigned int*>(a.colnorm + pl.q);
  a.R = reinterpret_cast<double*>(ws + pl.off_r);
  a.M64 = reinterpret_cast<double*>(ws + pl.off_m64);
  a.M32 = reinterpret_cast<float*>(ws + pl.off_m32);
  a.pi2 = reinterpret_cast<double*>(ws + pl.off_pi2);
  a.R_user = R_user;
  a.M_user = M_user;
  a.pi2_gauss = p->variant == 1 ? 1 : 0;
  a.flags = reinterpret_cast<uint32_t*>(ws + pl.off_status);
  a.pi2_ready = pi2_ready ? 1 : 0;
  a.pi2_gauss = p->variant == 1 ? 1 : 0;
  const size_t smem = sizeof(double) * static_cast<size_t>(Cond2Smem(a.rows_per_block, pl.q, pl.r2).total);
  if (!cuda_ok(cudaFuncSetAttribute(cond2_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)),
               "cond2 smem") ||
      !cuda_ok(cudaFuncSetAttribute(cond2_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)),
               "cond2 smem"))
    return false;
  if (!cuda_ok(cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int) * (groups + 1), st), "reset conditioning tickets"))
    return false;
  a.breakdown = &reinterpret_cast<StatusBlock*>(ws + pl.off_status)->qr_breakdown;
  cond2_kernel<0><<<grid, kGramThreads, smem, st>>>(a);
  cond2_kernel<1><<<grid, kGramThreads, smem, st>>>(a);
  count_launch(2);
  if (!cuda_ok(cudaGetLastError(), "launch condition")) return false;
  // After a breakdown (Π1·X too ill-conditioned for the Gram matrices), Householder QR.
  return launch_condition_householder(pl, pix, p, R_user, M_user, ws, st, a.breakdown);
}

// The one-block Householder variant (wide X, or after a CholeskyQR2 breakdown when only_if is set).
bool launch_condition_householder(const Plan& pl, const float* pix, const l1s_params* p, double* R_user,
                                  double* M_user, unsigned char* ws, cudaStream_t st, const uint32_t* only_if) {
  CondArgs a;
  a.only_if = only_if;
  a.pix = pix;
  a.r1 = pl.r1;
  a.q = pl.q;
  a.r2 = pl.r2;
  a.key = make_key(p->seed);
  a.problem = p->problem_id;
  a.work = reinterpret_cast<double*>(ws + pl.off_qr);
  a.R = reinterpret_cast<double*>(ws + pl.off_r);
  a.M64 = reinterpret_cast<double*>(ws + pl.off_m64);
  a.M32 = reinterpret_cast<float*>(ws + pl.off_m32);
  a.pi2 = reinterpret_cast<double*>(ws + pl.off_pi2);
  a.R_user = R_user;
  a.M_user = M_user;
  a.flags = reinterpret_cast<uint32_t*>(ws + pl.off_status);
  a.pi2_gauss = p->variant == 1 ? 1 : 0;
  const size_t bytes = sizeof(double) * static_cast<size_t>(pl.r1) * pl.q;
  a.in_smem = bytes <= kCondSmemMax ? 1 : 0;
  const size_t smem = a.in_smem ? bytes : 0;
  if (!cuda_ok(cudaFuncSetAttribute(condition_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)),
               "condition smem"))
    return false;
  condition_kernel<<<1, kCondThreads, smem, st>>>(a);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch condition");
}

bool launch_pi2(const l1s_params* p, int q, double* out, cudaStream_t st) {
  const int total = q * p->r2;
  pi2_kernel<<<(total + 127) / 128, 128, 0, st>>>(make_key(p->seed), p->problem_id, total, p->variant, out);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch pi2");
}

}  // namespace l1s
