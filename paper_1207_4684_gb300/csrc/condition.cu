// Conditioning (Figure 1, step 2; Figure 2, steps 2-3): FP64 QR of the small
// r1 × q matrix Π1·X with positive diag(R), then M = R⁻¹·Π2 with Π2 a q × r2
// matrix of independent standard Cauchys.  M is formed first (q × r2) so that
// phase 2 multiplies X by one skinny matrix, the order the paper's running-time
// argument uses (proof of the fast ℓ1 regression theorem: R⁻¹Π2 before X·(R⁻¹Π2)).
//
// A single thread block runs Householder reflections on a column-major FP64
// copy of Π1·X, held in shared memory when it fits (r1·q·8 bytes ≤ 160 KB) and
// in the workspace (L2-resident) otherwise.
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

// Π2 entry e (row-major q × r2): word e mod 4 of Philox call ⌊e/4⌋ on stream 1.
__device__ __forceinline__ double pi2_entry(Key2 key, uint32_t problem, int e) {
  const uint4 o = philox4x32_10(make_uint4(static_cast<uint32_t>(e >> 2), 0u, problem, kStreamPi2), key);
  const uint32_t w = (e & 3) == 0 ? o.x : (e & 3) == 1 ? o.y : (e & 3) == 2 ? o.z : o.w;
  return cauchy_f64(w >> 8);
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
};

__global__ void __launch_bounds__(kCondThreads) condition_kernel(const CondArgs a) {
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
  for (int e = tid; e < q * a.r2; e += nthr) a.pi2[e] = pi2_entry(a.key, a.problem, e);
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
// a fixed order and factors the q×q matrix in one warp.  Two launches: pass 0 (Gram of
// Π1X → R1), pass 1 (rows of Π1X·R1⁻¹ by forward substitution, their Gram → R2, then
// R = R2·R1 and M = R⁻¹Π2).
//
// FP64 arithmetic on this part has long latencies (a dependent FMA takes ~64 cycles,
// a division ~430, a square root ~670), so the serial parts avoid divisions and
// square roots: 1/√x comes from an FP32 estimate refined by two Newton steps in FP64,
// and every division by a diagonal entry is a multiplication by its stored reciprocal;
// sums keep four independent partial accumulators (combined in a fixed order).
constexpr int kGramThreads = 256;

struct Cond2Args {
  const float* pix;      // r1 × q row-major FP32
  int r1, q, r2;
  int rows_per_block;
  Key2 key;
  uint32_t problem;
  double* partials;      // [gridDim.x][q(q+1)/2]
  unsigned int* ticket;
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
};

// 1/√x for x > 0: FP32 estimate, then two Newton steps y ← y·(3 − x·y²)/2 in FP64.
__device__ __forceinline__ double rsqrt_f64(double x) {
  double y = static_cast<double>(rsqrtf(static_cast<float>(x)));
  y = y * fma(-0.5 * x * y, y, 1.5);
  y = y * fma(-0.5 * x * y, y, 1.5);
  return y;
}

// Cholesky of the symmetric q×q matrix G (row-major, upper triangle used) by one warp:
// on return the upper triangle of G holds R with RᵀR = G and dinv[k] = 1/R_kk.
// Returns false when a pivot is not positive.
__device__ bool warp_cholesky(double* G, double* dinv, int q) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int k = 0; k < q; ++k) {
    const double a = G[k * q + k];
    if (!(a > 0.0) || !isfinite(a)) ok = false;
    const double inv = rsqrt_f64(fmax(a, 1e-300));
    __syncwarp();
    for (int j = k + lane; j < q; j += 32) G[k * q + j] = (j == k) ? a * inv : G[k * q + j] * inv;
    if (lane == 0) dinv[k] = inv;
    __syncwarp();
    // trailing update of rows i > k, columns j ≥ i (upper triangle)
    for (int e = lane; e < (q - k - 1) * (q - k - 1); e += 32) {
      const int i = k + 1 + e / (q - k - 1), j = k + 1 + e % (q - k - 1);
      if (j >= i) G[i * q + j] = fma(-G[k * q + i], G[k * q + j], G[i * q + j]);
    }
    __syncwarp();
  }
  for (int e = lane; e < q * q; e += 32)
    if (e % q < e / q) G[e] = 0.0;
  __syncwarp();
  return ok;
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

template <int PASS>
__global__ void __launch_bounds__(kGramThreads) cond2_kernel(const Cond2Args a) {
  extern __shared__ __align__(16) double sm2[];
  __shared__ int s_last;
  const int q = a.q, tid = threadIdx.x;
  const int ne = q * (q + 1) / 2;
  const int r_lo = blockIdx.x * a.rows_per_block;
  const int r_hi = min(a.r1, r_lo + a.rows_per_block);
  const int nrows = r_hi - r_lo;
  double* rows = sm2;                         // max(rows_per_block, q) × q: this block's rows, later the Gram
  double* R1s = rows + max(a.rows_per_block, q) * q;   // q × q (pass 1: R1), then q reciprocals
  double* dinv = R1s + q * q;
  if (PASS == 1) {
    for (int e = tid; e < q * q; e += blockDim.x) R1s[e] = a.R1[e];
    for (int e = tid; e < q; e += blockDim.x) dinv[e] = a.R1dinv[e];
    __syncthreads();
  }
  if (PASS == 0) {
    for (int e = tid; e < nrows * q; e += blockDim.x)
      rows[e] = static_cast<double>(a.pix[static_cast<size_t>(r_lo) * q + e]);
  } else {
    // y·R1 = x by forward substitution, one row per thread
    for (int i = tid; i < nrows; i += blockDim.x) {
      const float* x = a.pix + static_cast<size_t>(r_lo + i) * q;
      double* y = rows + i * q;
      for (int c = 0; c < q; ++c) {
        double v = static_cast<double>(x[c]);
        for (int k = 0; k < c; ++k) v = fma(-y[k], R1s[k * q + c], v);
        y[c] = v * dinv[c];
      }
    }
  }
  __syncthreads();
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
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // ---- last block: fixed-order sum of the partials, then the q×q work
  double* Gs = rows;
  for (int e = tid; e < ne; e += blockDim.x) {
    const double v = sum4(a.partials + e, gridDim.x, ne);
    int j, l;
    pair_index(e, q, j, l);
    Gs[j * q + l] = v;
    Gs[l * q + j] = v;
  }
  if (PASS == 1)
    for (int e = tid; e < q * a.r2; e += blockDim.x) a.pi2[e] = pi2_entry(a.key, a.problem, e);
  __syncthreads();
  if (tid >= 32) return;
  if (PASS == 0)
    for (int k = tid; k < q; k += 32) a.colnorm[k] = sqrt(Gs[k * q + k]);
  double* dn = dinv + q;                      // reciprocals of this pass's factor
  const bool ok = warp_cholesky(Gs, dn, q);
  if (tid == 0 && !ok) raise_flag(a.flags, L1S_ERR_RANK_DEFICIENT);
  if (PASS == 0) {
    for (int e = tid; e < q * q; e += 32) a.R1[e] = Gs[e];
    for (int e = tid; e < q; e += 32) a.R1dinv[e] = dn[e];
  } else {
    // R = R2·R1 (both upper triangular) and the reciprocals of its diagonal
    for (int e = tid; e < q * q; e += 32) {
      const int i = e / q, j = e - i * q;
      double v = 0.0;
      for (int k = i; k <= j; ++k) v = fma(Gs[i * q + k], R1s[k * q + j], v);
      a.R[e] = j < i ? 0.0 : v;
    }
    __syncwarp();
    for (int k = tid; k < q; k += 32) dn[k] = dn[k] * dinv[k];   // 1/(R2_kk·R1_kk)
    __syncwarp();
    if (tid == 0) {
      bool bad = !ok;
      for (int k = 0; k < q; ++k) {
        const double rkk = a.R[k * q + k];
        if (!(rkk > kRankTol * a.colnorm[k]) || !isfinite(rkk)) bad = true;
      }
      if (bad) raise_flag(a.flags, L1S_ERR_RANK_DEFICIENT);
    }
    // M = R⁻¹·Π2 by back substitution with the stored reciprocals, one column per lane
    for (int c = tid; c < a.r2; c += 32) {
      for (int k = q - 1; k >= 0; --k) {
        double acc = a.pi2[k * a.r2 + c];
        for (int j = k + 1; j < q; ++j) acc = fma(-a.R[k * q + j], a.M64[j * a.r2 + c], acc);
        a.M64[k * a.r2 + c] = acc * dn[k];
      }
    }
    __syncwarp();
    for (int e = tid; e < q * a.r2; e += 32) {
      const double m = a.M64[e];
      a.M32[e] = static_cast<float>(m);
      if (a.M_user) a.M_user[e] = m;
    }
    if (a.R_user)
      for (int e = tid; e < q * q; e += 32) a.R_user[e] = a.R[e];
  }
  if (tid == 0) *a.ticket = 0u;   // ready for the next launch
}

__global__ void pi2_kernel(Key2 key, uint32_t problem, int total, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < total) out[e] = pi2_entry(key, problem, e);
}

// Rows of Π1X per block of the Gram pass: at least q, and at most 32 blocks.
static int cond2_rows_per_block(int r1, int q) { return std::max(q, (r1 + 31) / 32); }

size_t cond2_scratch_bytes(int r1, int q, int sms) {
  (void)sms;
  const int rpb = cond2_rows_per_block(r1, q);
  const int blocks = (r1 + rpb - 1) / rpb;
  return sizeof(double) * (static_cast<size_t>(blocks) * (q * (q + 1) / 2) + q * q + 2 * q) + 256;
}

bool launch_condition(const Plan& pl, const float* pix, const l1s_params* p, double* R_user,
                      double* M_user, unsigned char* ws, cudaStream_t st) {
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
  a.partials = scratch;
  a.R1 = scratch + static_cast<size_t>(grid) * ne;
  a.R1dinv = a.R1 + pl.q * pl.q;
  a.colnorm = a.R1dinv + pl.q;
  a.ticket = reinterpret_cast<unsigned int*>(ws + pl.off_status + offsetof(StatusBlock, cond_ticket));
  a.R = reinterpret_cast<double*>(ws + pl.off_r);
  a.M64 = reinterpret_cast<double*>(ws + pl.off_m64);
  a.M32 = reinterpret_cast<float*>(ws + pl.off_m32);
  a.pi2 = reinterpret_cast<double*>(ws + pl.off_pi2);
  a.R_user = R_user;
  a.M_user = M_user;
  a.flags = reinterpret_cast<uint32_t*>(ws + pl.off_status);
  const size_t smem = sizeof(double) * (static_cast<size_t>(std::max(a.rows_per_block, pl.q)) * pl.q + 2 * pl.q * pl.q + 2 * pl.q);
  if (!cuda_ok(cudaFuncSetAttribute(cond2_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)),
               "cond2 smem") ||
      !cuda_ok(cudaFuncSetAttribute(cond2_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)),
               "cond2 smem"))
    return false;
  if (!cuda_ok(cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int), st), "reset conditioning ticket")) return false;
  cond2_kernel<0><<<grid, kGramThreads, smem, st>>>(a);
  cond2_kernel<1><<<grid, kGramThreads, smem, st>>>(a);
  count_launch(2);
  return cuda_ok(cudaGetLastError(), "launch condition");
}

// The one-block Householder variant (kept for reference checks of the Cholesky route).
bool launch_condition_householder(const Plan& pl, const float* pix, const l1s_params* p, double* R_user,
                                  double* M_user, unsigned char* ws, cudaStream_t st) {
  CondArgs a;
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
  pi2_kernel<<<(total + 127) / 128, 128, 0, st>>>(make_key(p->seed), p->problem_id, total, out);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch pi2");
}

}  // namespace l1s
