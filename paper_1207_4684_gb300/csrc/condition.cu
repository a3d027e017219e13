// Conditioning (Figure 1, step 2; Figure 2, steps 2-3): FP64 QR of the small
// r1 × q matrix Π1·X with positive diag(R), then M = R⁻¹·Π2 with Π2 a q × r2
// matrix of independent standard Cauchys.  M is formed first (q × r2) so that
// phase 2 multiplies X by one skinny matrix, the order the paper's running-time
// argument uses (proof of the fast ℓ1 regression theorem: R⁻¹Π2 before X·(R⁻¹Π2)).
//
// A single thread block runs Householder reflections on a column-major FP64
// copy of Π1·X, held in shared memory when it fits (r1·q·8 bytes ≤ 160 KB) and
// in the workspace (L2-resident) otherwise.
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

__global__ void pi2_kernel(Key2 key, uint32_t problem, int total, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < total) out[e] = pi2_entry(key, problem, e);
}

bool launch_condition(const Plan& pl, const float* pix, const l1s_params* p, double* R_user,
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
  return cuda_ok(cudaGetLastError(), "launch condition");
}

bool launch_pi2(const l1s_params* p, int q, double* out, cudaStream_t st) {
  const int total = q * p->r2;
  pi2_kernel<<<(total + 127) / 128, 128, 0, st>>>(make_key(p->seed), p->problem_id, total, out);
  return cuda_ok(cudaGetLastError(), "launch pi2");
}

}  // namespace l1s
