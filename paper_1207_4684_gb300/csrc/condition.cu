// Conditioning (Figure 1, step 2; Figure 2, steps 2-3): FP64 QR of the small
// r1 × q matrix Π1·X with positive diag(R), then M = R⁻¹·Π2 with Π2 a q × r2
// matrix of independent standard Cauchys.  M is formed first (q × r2) so that
// phase 2 multiplies X by one skinny matrix, the order the paper's running-time
// argument uses (proof of the fast ℓ1 regression theorem: R⁻¹Π2 before X·(R⁻¹Π2)).
//
// The QR is CholeskyQR2 (below) in two launches over many thread blocks, and M comes
// from a third, one block per row of M.  When the blocks do not fit in shared memory
// (q above about 93), a single thread block runs
// Householder reflections on a column-major FP64 copy of Π1·X instead, held in
// shared memory when it fits (r1·q·8 bytes ≤ 160 KB) and in the workspace
// (L2-resident) otherwise.  CholeskyQR2 squares the condition number in its Gram
// matrices and breaks down when Π1·X is conditioned worse than about 1e7-1e8; a
// breakdown (a Cholesky pivot that is not positive, or a non-finite R or M) is recorded
// in the status block, and the Householder kernel, enqueued after those launches, then
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
// Cholesky step twice (R1 from the Gram of Π1X, R2 from the Gram of Y = Π1X·R1⁻¹,
// R = R2·R1) gives a QR factor accurate to FP64 rounding whenever the condition
// number is below about 1e7 — far past what an FP32-accumulated Π1X resolves (the
// rank test flags columns dependent to 1e-5).  Each Cholesky factorisation also yields
// the inverse of its factor (the elimination's row operations applied to the identity),
// so that everything else is a matrix product: the rows of Y = Π1X·R1⁻¹, and
// M = R⁻¹Π2 = R1⁻¹·(R2⁻¹·Π2).  The Gram products spread over thread blocks; the last
// block to finish (an atomic ticket, no waiting) sums the partials in a fixed order and
// factors the q×q matrix.  Two launches: pass 0 (Gram of Π1X → R1 and R1⁻¹), pass 1
// (rows of Y, their Gram → R2 and R2⁻¹, then M, and R = R2·R1 when the caller asks for
// it).  Π2 is drawn by the phase-1 reduction when the whole pass runs.
//
// FP64 arithmetic on this part is slow (a dependent FMA takes ~64 cycles, and a full-warp
// FP64 instruction holds its sub-partition for ~64-80 cycles however few of its lanes
// are active), so the factorisation keeps one short chain per step — a reciprocal from the
// hardware's FP64 approximation (refined by Newton steps where it enters R), no division or
// square root — and packs each step's independent updates densely over all threads; the
// products and the sums of the partials are independent dot products.
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
  double* Z1;            // q × q: R1⁻¹ (pass 0 → pass 1)
  double* R2;            // q × q (pass 1 → cond_m_kernel)
  double* Z2;            // q × q: R2⁻¹ (pass 1 → cond_m_kernel)
  double* colnorm;       // q: ‖(Π1X)_:k‖₂
  double* R;             // q × q row-major (output, when the caller asks for R)
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

// 1/√x for x > 0 in FP64: an FP32 estimate of the mantissa part (the exponent is split
// off first, so any normal FP64 x works), then Newton steps y ← y·(3/2 − (x/2)·y²) in FP64.
// Each step doubles the number of correct bits: one leaves a relative error near 1e-13,
// two reach FP64 rounding.
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

// 1/x for a positive normal FP64 x on the serial chain of the factorisation: the
// hardware's approximate FP64 reciprocal (PTX rcp.approx.ftz.f64; at most 2^-19.9 relative
// error over 4M random operands spanning 1e±260 on GB300, where two Newton steps need
// 2^-14) refined by two Newton steps y ← y + y·(1 − x·y), each of which squares the
// relative error, to FP64 rounding.
__device__ __forceinline__ double rcp_approx_f64(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

__device__ __forceinline__ double rcp_newton_f64(double x) {
  double y = rcp_approx_f64(x);
  y = fma(y, fma(-x, y, 1.0), y);
  return fma(y, fma(-x, y, 1.0), y);
}

// The pivot reciprocals of the two factorisations.  Pass 0 only preconditions: any r_k
// close to 1/d_k serves, because R1 and R1⁻¹ are both formed from the same r_k (they stay
// exact inverses of each other) and pass 1 corrects the rest — the hardware approximation
// alone.  Pass 1's R2 is part of R: two Newton steps.  A pivot that is not positive gives a
// meaningless reciprocal here and is reported after the loop.
template <int PASS>
__device__ __forceinline__ double pivot_rcp(double d) {
  return PASS == 0 ? rcp_approx_f64(d) : rcp_newton_f64(d);
}

// Threads [0, nt) take part in the factorisation (nt a multiple of 32: 128 for q ≤ 32,
// where four warps are enough and a named barrier is cheaper, else the whole block).
__device__ __forceinline__ void sync_first(int nt) {
  if (nt == static_cast<int>(blockDim.x)) __syncthreads();
  else named_barrier(1, nt);
}

// The entries (i, j), 1 ≤ i ≤ j < q, of an upper triangle, the rows nearest the bottom
// first: entry e lies in row i = q − 1 − w with w the largest integer of w(w+1)/2 ≤ e, so
// that the entries below row k form the prefix of length (q−1−k)(q−k)/2.  Packed i·2^16 + j.
__device__ void fill_tri(uint32_t* tri, int q) {
  for (int e = threadIdx.x; e < q * (q - 1) / 2; e += blockDim.x) {
    int w = static_cast<int>((sqrtf(8.0f * static_cast<float>(e) + 1.0f) - 1.0f) * 0.5f);
    while ((w + 1) * (w + 2) / 2 <= e) ++w;
    while (w * (w + 1) / 2 > e) --w;
    const int i = q - 1 - w;
    tri[e] = (static_cast<uint32_t>(i) << 16) | static_cast<uint32_t>(i + e - w * (w + 1) / 2);
  }
}

// Cholesky factor R of the symmetric positive definite q×q matrix G and its inverse Z,
// right-looking in the square-root-free form G = L·D·Lᵀ (L unit lower triangular) by the
// threads [0, nt).  Step k uses pivot d_k, its reciprocal r_k (pivot_rcp) and the multipliers
// u_i = l_ik = G_ki·r_k (i > k): the trailing upper triangle loses u_i·G_kj (k < i ≤ j), and
// the same row operations, applied to E (the identity at the start), leave E = L⁻¹ — its
// rows i > k lose u_i times row k.  Warp 0 updates row k+1, the next pivot among it, and
// from them forms r_{k+1} and the next step's multipliers (every lane the same values, so
// no exchange); the other warps update the rows below and E, flat over their threads (the
// triangle through the table of fill_tri).  One barrier per step; the serial chain per
// step is the pivot update, one reciprocal and one product.  Then R = D^½·Lᵀ (R_kk = √d_k,
// R_kj = √d_k·u_j of step k) overwrites the upper triangle of G, and Z = R⁻¹ = Eᵀ·D^-½ the
// upper triangle of E (the strictly lower parts of both become zero).  G and E are
// row-major q×q in shared memory; s_u holds 2q doubles (the multipliers of two steps), s_r,
// s_t and s_s q each (r_k, 1/√d_k, √d_k).  Returns false when a pivot is not positive.
template <int PASS>
__device__ bool block_chol_inv(double* G, double* E, const uint32_t* tri, double* s_u, double* s_r,
                               double* s_t, double* s_s, int q, int nt) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (warp == 0) {
    const double r = pivot_rcp<PASS>(G[0]);
    if (lane == 0) s_r[0] = r;
    for (int j = 1 + lane; j < q; j += 32) s_u[j] = G[j] * r;
  }
  sync_first(nt);
  for (int k = 0; k + 1 < q; ++k) {
    const double* u = s_u + (k & 1) * q;            // multipliers of step k
    const double* gk = G + k * q;
    if (warp == 0) {
      double* un = s_u + ((k + 1) & 1) * q;         // those of step k + 1
      double* g1 = G + (k + 1) * q;
      const double uk1 = u[k + 1];
      const double d1 = fma(-uk1, gk[k + 1], g1[k + 1]);
      const double r1 = pivot_rcp<PASS>(d1);
      if (lane == 0) {
        g1[k + 1] = d1;
        s_r[k + 1] = r1;
      }
      for (int j = k + 2 + lane; j < q; j += 32) {
        const double v = fma(-uk1, gk[j], g1[j]);
        g1[j] = v;
        un[j] = v * r1;
      }
    } else {
      // Four entries per thread at a time, all loads before the stores (the entries of a step
      // are distinct and none is read by another), so that their shared-memory and FP64
      // latencies overlap.  E's new column k is −u_i = fma(−u_i, 1, 0).
      const int w = q - 1 - k;
      const int ntri = (w - 1) * w / 2;              // trailing entries below row k+1
      const int total = ntri + w * (k + 1);          // and the entries (i, c) of E, k < i, c ≤ k
      const int step = nt - 32;
      for (int e0 = t - 32; e0 < total; e0 += 4 * step) {
        double* dst[4];
        double ua[4], bb[4], cc[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int e = e0 + m * step;
          dst[m] = nullptr;
          ua[m] = 0.0;
          bb[m] = 0.0;
          cc[m] = 0.0;
          if (e < ntri) {
            const uint32_t ij = tri[e];
            const int i = static_cast<int>(ij >> 16), j = static_cast<int>(ij & 0xFFFFu);
            dst[m] = G + i * q + j;
            ua[m] = u[i];
            bb[m] = gk[j];
            cc[m] = *dst[m];
          } else if (e < total) {
            const int f = e - ntri;
            const int di = f / (k + 1);
            const int i = k + 1 + di, c = f - di * (k + 1);
            dst[m] = E + i * q + c;
            ua[m] = u[i];
            bb[m] = c == k ? 1.0 : E[k * q + c];
            cc[m] = c == k ? 0.0 : *dst[m];
          }
        }
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (dst[m]) *dst[m] = fma(-ua[m], bb[m], cc[m]);
      }
    }
    sync_first(nt);
  }
  bool bad = false;
  for (int k = t; k < q; k += nt) {
    const double d0 = G[k * q + k];
    if (!(d0 > 0.0) || !isfinite(d0)) bad = true;
    const double d = fmax(d0, 1e-300);
    const double tk = rsqrt_f64(d, 2);
    s_t[k] = tk;
    s_s[k] = d * tk;
  }
  const bool ok = !named_barrier_any(1, nt, bad);
  // R in place (each entry reads only itself); Z's upper part from E's strictly lower part
  for (int e = t; e < q * q; e += nt) {
    const int i = e / q, j = e - i * q;
    if (j < i) {
      G[e] = 0.0;
    } else {
      G[e] = j == i ? s_s[i] : s_s[i] * (G[e] * s_r[i]);
      E[e] = j == i ? s_t[i] : E[j * q + i] * s_t[j];
    }
  }
  sync_first(nt);
  for (int e = t; e < q * q; e += nt)
    if (e % q < e / q) E[e] = 0.0;
  sync_first(nt);
  return ok;
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

// out(e, Σ_{p<count} src[p·stride + e]) for every e < ne, over the whole block: a thread
// takes RUN entries at a time and loads CHUNK partials of each before it adds them, so that
// their L2 round trips overlap, into four accumulators (p mod 4) combined at the end — the
// same order whatever the schedule.  The partials come from other blocks of the launch, so
// they are read at L2.
template <int RUN, int CHUNK, class Out>
__device__ __forceinline__ void sum_partials_t(const double* src, int count, size_t stride, int ne, Out out) {
  static_assert(CHUNK % 4 == 0, "chunks of whole accumulator rounds");
  const int nb = static_cast<int>(blockDim.x);
  for (int e0 = threadIdx.x; e0 < ne; e0 += RUN * nb) {
    double acc[RUN][4];
#pragma unroll
    for (int m = 0; m < RUN; ++m)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[m][c] = 0.0;
    for (int p0 = 0; p0 < count; p0 += CHUNK) {
      double v[RUN][CHUNK];
#pragma unroll
      for (int m = 0; m < RUN; ++m)
#pragma unroll
        for (int c = 0; c < CHUNK; ++c) {
          const int e = e0 + m * nb, p = p0 + c;
          v[m][c] = (e < ne && p < count) ? __ldcg(src + static_cast<size_t>(p) * stride + e) : 0.0;
        }
#pragma unroll
      for (int m = 0; m < RUN; ++m)
#pragma unroll
        for (int c = 0; c < CHUNK; ++c) acc[m][c & 3] += v[m][c];
    }
#pragma unroll
    for (int m = 0; m < RUN; ++m) {
      const int e = e0 + m * nb;
      if (e < ne) out(e, (acc[m][0] + acc[m][1]) + (acc[m][2] + acc[m][3]));
    }
  }
}

template <class Out>
__device__ __forceinline__ void sum_partials(const double* src, int count, size_t stride, int ne, Out out) {
  if (ne <= static_cast<int>(blockDim.x)) sum_partials_t<1, 32>(src, count, stride, ne, out);
  else sum_partials_t<4, 8>(src, count, stride, ne, out);
}

// dst[e] = src[e] for e < count over the whole block, kStageRun loads of a thread in flight
// before their stores (global loads at L2: the factors come from other blocks of earlier
// launches).
constexpr int kStageRun = 8;
template <typename TS>
__device__ __forceinline__ void stage_to_shared(double* dst, const TS* src, int count) {
  const int nb = static_cast<int>(blockDim.x);
  for (int e0 = threadIdx.x; e0 < count; e0 += kStageRun * nb) {
    TS v[kStageRun];
#pragma unroll
    for (int u = 0; u < kStageRun; ++u) {
      const int e = e0 + u * nb;
      v[u] = e < count ? __ldcg(src + e) : TS(0);
    }
#pragma unroll
    for (int u = 0; u < kStageRun; ++u) {
      const int e = e0 + u * nb;
      if (e < count) dst[e] = static_cast<double>(v[u]);
    }
  }
}

// Shared memory of a cond2 block (doubles): the rows of Π1X, later the Gram matrix and R in
// place | the rows of Y (pass 1), later E and the inverse factor in place | R1⁻¹ (pass 1) |
// the triangle table (uint32) | the multipliers of two steps | r_k | 1/√d_k | √d_k | diag R1.
struct Cond2Smem {
  int G, EZ, Z1, tri, su, sr, st, ss, r1d, total;
  __host__ __device__ Cond2Smem(int rpb, int q) {
    const int big = (rpb > q ? rpb : q) * q;
    G = 0;
    EZ = G + big;
    Z1 = EZ + big;
    tri = Z1 + q * q;
    su = tri + (q * (q - 1) / 2 + 1) / 2;
    sr = su + 2 * q;
    st = sr + q;
    ss = st + q;
    r1d = ss + q;
    total = r1d + q;
  }
};

template <int PASS>
__global__ void __launch_bounds__(kGramThreads) cond2_kernel(const Cond2Args a) {
  extern __shared__ __align__(16) double sm2[];
  __shared__ int s_last;
  __shared__ int s_ok;
  const int q = a.q, tid = threadIdx.x;
  const int ne = q * (q + 1) / 2;
  const int r_lo = blockIdx.x * a.rows_per_block;
  const int r_hi = min(a.r1, r_lo + a.rows_per_block);
  const int nrows = r_hi - r_lo;
  const Cond2Smem L(a.rows_per_block, q);
  double* rows = sm2 + L.G;                   // this block's rows of Π1X, later the Gram
  double* EZ = sm2 + L.EZ;                    // pass 1: the rows of Y; the tail: E, Z
  double* Z1s = sm2 + L.Z1;
  double* r1d = sm2 + L.r1d;
  if (PASS == 0) {
    // Π2, unless the phase-1 reduction drew it, spread over all blocks.
    if (!a.pi2_ready)
      for (int e = blockIdx.x * blockDim.x + tid; e < q * a.r2; e += gridDim.x * blockDim.x)
        a.pi2[e] = pi2_value(a.key, a.problem, e, a.pi2_gauss);
  } else {
    stage_to_shared(Z1s, a.Z1, q * q);
    for (int e = tid; e < q; e += blockDim.x) r1d[e] = a.R1[e * q + e];
  }
  stage_to_shared(rows, a.pix + static_cast<size_t>(r_lo) * q, nrows * q);
  __syncthreads();
  const double* src = rows;
  if (PASS == 1) {
    // Y = X·R1⁻¹ with R1⁻¹ upper triangular: Y_ic = Σ_{k≤c} X_ik·(R1⁻¹)_kc, an entry per thread
    for (int e = tid; e < nrows * q; e += blockDim.x) {
      const int i = e / q, c = e - i * q;
      const double* x = rows + i * q;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int k = 0;
      for (; k + 3 <= c; k += 4) {
        s0 = fma(x[k], Z1s[k * q + c], s0);
        s1 = fma(x[k + 1], Z1s[(k + 1) * q + c], s1);
        s2 = fma(x[k + 2], Z1s[(k + 2) * q + c], s2);
        s3 = fma(x[k + 3], Z1s[(k + 3) * q + c], s3);
      }
      for (; k <= c; ++k) s0 = fma(x[k], Z1s[k * q + c], s0);
      EZ[e] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
    src = EZ;
  }
  for (int e = tid; e < ne; e += blockDim.x) {
    int j, l;
    pair_index(e, q, j, l);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 3 < nrows; i += 4) {
      s0 = fma(src[i * q + j], src[i * q + l], s0);
      s1 = fma(src[(i + 1) * q + j], src[(i + 1) * q + l], s1);
      s2 = fma(src[(i + 2) * q + j], src[(i + 2) * q + l], s2);
      s3 = fma(src[(i + 3) * q + j], src[(i + 3) * q + l], s3);
    }
    for (; i < nrows; ++i) s0 = fma(src[i * q + j], src[i * q + l], s0);
    a.partials[static_cast<size_t>(blockIdx.x) * ne + e] = (s0 + s1) + (s2 + s3);
  }
  // Two-level fixed-order sum of the partials: the last block of each group of
  // cond2_group_size blocks adds its group's partials; the last group to finish adds the
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
    sum_partials(a.partials + static_cast<size_t>(g_lo) * ne, g_n, ne, ne,
                 [&](int e, double v) { gsum[static_cast<size_t>(g) * ne + e] = v; });
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(a.ticket + groups, 1u) == static_cast<unsigned>(groups - 1)) ? 1 : 0;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
  }
  // ---- last group: the group sums (or, with one group, the partials), then the q×q work
  double* Gs = rows;
  sum_partials(groups > 1 ? gsum : a.partials, groups > 1 ? groups : static_cast<int>(gridDim.x), ne, ne,
               [&](int e, double v) {
                 int j, l;
                 pair_index(e, q, j, l);
                 Gs[j * q + l] = v;
                 Gs[l * q + j] = v;
                 if (PASS == 0 && j == l) a.colnorm[j] = sqrt(v);
               });
  uint32_t* tri = reinterpret_cast<uint32_t*>(sm2 + L.tri);
  fill_tri(tri, q);
  __syncthreads();
  const int nt = q > 32 ? static_cast<int>(blockDim.x) : 128;
  if (tid < nt) {
    const bool ok = block_chol_inv<PASS>(Gs, EZ, tri, sm2 + L.su, sm2 + L.sr, sm2 + L.st, sm2 + L.ss, q, nt);
    if (tid == 0) s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  if (PASS == 0) {
    if (tid == 0) *a.breakdown = s_ok ? 0u : 1u;     // the Householder kernel redoes the step
    for (int e = tid; e < q * q; e += blockDim.x) {
      a.R1[e] = Gs[e];
      a.Z1[e] = EZ[e];
    }
  } else {
    const bool broke0 = *a.breakdown != 0u || !s_ok;
    if (tid < 32) {
      // rank test over the columns, one lane per column: R_kk = (R2)_kk·(R1)_kk (skipped after a
      // breakdown: the Householder kernel runs its own)
      bool bad = false;
      for (int k = tid; k < q; k += 32) {
        const double rkk = Gs[k * q + k] * r1d[k];
        if (!(rkk > kRankTol * a.colnorm[k]) || !isfinite(rkk)) bad = true;
      }
      if (__any_sync(0xffffffffu, bad) && !broke0) {
        if (tid == 0) raise_flag(a.flags, L1S_ERR_RANK_DEFICIENT);
      }
      if (broke0 && tid == 0) *a.breakdown = 1u;
    }
    for (int e = tid; e < q * q; e += blockDim.x) {
      a.R2[e] = Gs[e];
      a.Z2[e] = EZ[e];
    }
  }
  for (int k = tid; k <= groups; k += blockDim.x) a.ticket[k] = 0u;   // ready for the next pass
}

// After pass 1, one block per row i (Figure 2, step 3): row i of R⁻¹ = R1⁻¹·R2⁻¹, then
// M_i = (R⁻¹)_i·Π2 and, when the caller asks for R, R_i = (R2)_i·R1 — products of upper
// triangular factors, an entry per thread.  A non-finite entry of M records a breakdown, so
// that the Householder kernel enqueued next redoes the step.
constexpr int kCondMThreads = 128;

__global__ void __launch_bounds__(kCondMThreads) cond_m_kernel(const Cond2Args a) {
  // shared: R2⁻¹ (q×q), Π2 (q×r2), row i of R1⁻¹ and of R⁻¹ (q each), and for R the rows of
  // R1 (q×q) and row i of R2 (q)
  extern __shared__ __align__(16) double cm[];
  const int q = a.q, r2 = a.r2, i = blockIdx.x, tid = threadIdx.x;
  const bool want_r = a.R_user != nullptr;
  double* z2 = cm;
  double* pi = z2 + q * q;
  double* z1 = pi + q * r2;
  double* zr = z1 + q;
  double* r1 = zr + q;
  double* r2i = r1 + (want_r ? q * q : 0);
  stage_to_shared(z2, a.Z2, q * q);
  stage_to_shared(pi, a.pi2, q * r2);
  stage_to_shared(z1, a.Z1 + i * q, q);
  if (want_r) {
    stage_to_shared(r1, a.R1, q * q);
    stage_to_shared(r2i, a.R2 + i * q, q);
  }
  __syncthreads();
  for (int j = tid; j < q; j += blockDim.x) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = i;
    for (; k + 3 <= j; k += 4) {
      s0 = fma(z1[k], z2[k * q + j], s0);
      s1 = fma(z1[k + 1], z2[(k + 1) * q + j], s1);
      s2 = fma(z1[k + 2], z2[(k + 2) * q + j], s2);
      s3 = fma(z1[k + 3], z2[(k + 3) * q + j], s3);
    }
    for (; k <= j; ++k) s0 = fma(z1[k], z2[k * q + j], s0);
    zr[j] = j < i ? 0.0 : (s0 + s1) + (s2 + s3);
  }
  __syncthreads();
  for (int c = tid; c < r2; c += blockDim.x) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = i;
    for (; k + 3 < q; k += 4) {
      s0 = fma(zr[k], pi[k * r2 + c], s0);
      s1 = fma(zr[k + 1], pi[(k + 1) * r2 + c], s1);
      s2 = fma(zr[k + 2], pi[(k + 2) * r2 + c], s2);
      s3 = fma(zr[k + 3], pi[(k + 3) * r2 + c], s3);
    }
    for (; k < q; ++k) s0 = fma(zr[k], pi[k * r2 + c], s0);
    const double m = (s0 + s1) + (s2 + s3);
    a.M64[i * r2 + c] = m;
    a.M32[i * r2 + c] = static_cast<float>(m);
    if (a.M_user) a.M_user[i * r2 + c] = m;
    if (!isfinite(m)) *a.breakdown = 1u;
  }
  if (want_r) {
    for (int j = tid; j < q; j += blockDim.x) {
      double s0 = 0.0, s1 = 0.0;
      int k = i;
      for (; k + 1 <= j; k += 2) {
        s0 = fma(r2i[k], r1[k * q + j], s0);
        s1 = fma(r2i[k + 1], r1[(k + 1) * q + j], s1);
      }
      if (k <= j) s0 = fma(r2i[k], r1[k * q + j], s0);
      const double v = j < i ? 0.0 : s0 + s1;
      a.R[i * q + j] = v;
      a.R_user[i * q + j] = v;
    }
  }
}

static size_t cond_m_smem(int q, int r2, bool want_r) {
  return sizeof(double) * (static_cast<size_t>(q) * q + static_cast<size_t>(q) * r2 + 2 * q +
                           (want_r ? static_cast<size_t>(q) * q + q : 0));
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
  return sizeof(double) * (static_cast<size_t>(blocks + groups) * (q * (q + 1) / 2) + 4 * q * q + q) +
         sizeof(unsigned int) * (groups + 1) + 256;
}

bool launch_condition_householder(const Plan& pl, const float* pix, const l1s_params* p, double* R_user,
                                  double* M_user, unsigned char* ws, cudaStream_t st,
                                  const uint32_t* only_if = nullptr);

bool launch_condition(const Plan& pl, const float* pix, const l1s_params* p, double* R_user,
                      double* M_user, unsigned char* ws, cudaStream_t st, bool pi2_ready) {
  // Wide X (q above about 93) does not fit the CholeskyQR2 blocks in shared memory: one block
  // of Householder reflections on a workspace copy handles it instead.
  if (std::max(sizeof(double) * static_cast<size_t>(Cond2Smem(cond2_rows_per_block(pl.r1, pl.q), pl.q).total),
               cond_m_smem(pl.q, pl.r2, R_user != nullptr)) > static_cast<size_t>(device_info().max_smem_optin))
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
  a.Z1 = a.R1 + pl.q * pl.q;
  a.R2 = a.Z1 + pl.q * pl.q;
  a.Z2 = a.R2 + pl.q * pl.q;
  a.colnorm = a.Z2 + pl.q * pl.q;
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
  const size_t smem = sizeof(double) * static_cast<size_t>(Cond2Smem(a.rows_per_block, pl.q).total);
  const size_t msmem = cond_m_smem(pl.q, pl.r2, R_user != nullptr);
  if (!allow_dynamic_smem(reinterpret_cast<const void*>(cond2_kernel<0>), smem, "cond2 smem") ||
      !allow_dynamic_smem(reinterpret_cast<const void*>(cond2_kernel<1>), smem, "cond2 smem") ||
      !allow_dynamic_smem(reinterpret_cast<const void*>(cond_m_kernel), msmem, "cond_m smem"))
    return false;
  if (!cuda_ok(cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int) * (groups + 1), st), "reset conditioning tickets"))
    return false;
  a.breakdown = &reinterpret_cast<StatusBlock*>(ws + pl.off_status)->qr_breakdown;
  cond2_kernel<0><<<grid, kGramThreads, smem, st>>>(a);
  cond2_kernel<1><<<grid, kGramThreads, smem, st>>>(a);
  cond_m_kernel<<<pl.q, kCondMThreads, msmem, st>>>(a);
  count_launch(3);
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
  if (!allow_dynamic_smem(reinterpret_cast<const void*>(condition_kernel), smem, "condition smem"))
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
