// Phase 2 (Figure 2, steps 4-5): λ_i = median_j |Λ_ij|, Λ = X·M, M = R⁻¹·Π2.
//
// One thread per row: the q values of X_(i) are loaded (vectorised when A's
// rows allow it), the q × r2 product accumulates in FP32 registers with M read
// from the constant bank (every lane of a warp reads the same M entry, so the
// operand comes straight from the constant cache into the FMA), |·| is taken,
// and the lower median — the ((r2−1)/2)-th order statistic from 0 — is picked
// by a Batcher odd–even merge network whose unused comparators the compiler
// drops.  λ is written once (4 B/row) and each block adds its λ's into an FP64
// partial of Σλ through compensated FP32 pairs, so Σλ does not depend on the
// launch order.  X crosses HBM once.
//
// The kernels live in lambda_kernels.cuh and are instantiated per storage type and
// home of M in lambda_f32_const.cu, lambda_f32_smem.cu, lambda_bf16_const.cu and
// lambda_bf16_smem.cu (each with its own constant bank); this unit holds the Σλ
// finish, the FP32 copy of M and the dispatch.
#include <algorithm>

#include "l1s_common.cuh"

namespace l1s {

constexpr int kLamThreads = 256;

bool launch_lambda_f32_const(const Plan& pl, const void* A, int64_t lda, const float* b, float* lam, double* sums,
                         const float* m32, cudaStream_t st);
bool launch_lambda_f32_smem(const Plan& pl, const void* A, int64_t lda, const float* b, float* lam, double* sums,
                         const float* m32, cudaStream_t st);
bool launch_lambda_bf16_const(const Plan& pl, const void* A, int64_t lda, const float* b, float* lam, double* sums,
                         const float* m32, cudaStream_t st);
bool launch_lambda_bf16_smem(const Plan& pl, const void* A, int64_t lda, const float* b, float* lam, double* sums,
                         const float* m32, cudaStream_t st);

// Σλ over the block partials in a fixed order (strided per-thread sums, then a
// fixed shuffle tree and the warp sums in order); τ = m_s / Σλ.
__global__ void __launch_bounds__(256) lambda_finalize_kernel(const double* __restrict__ block_sums, int nblocks,
                                                              double coreset, StatusBlock* status, double* user_sum) {
  __shared__ double wsum[8];
  const double tot = lambda_total_256(block_sums, nblocks, wsum);
  if (threadIdx.x == 0) {
    status->lambda_total = tot;
    if (user_sum) *user_sum = tot;
    double tau;
    float tau32;
    if (!tau_of(tot, coreset, &tau, &tau32)) raise_flag(&status->flags, L1S_ERR_ZERO_MASS);
    status->tau = tau;
    status->tau32 = tau32;
  }
}

__global__ void m_to_f32_kernel(const double* __restrict__ m, int total, float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < total) out[e] = static_cast<float>(m[e]);
}

int lambda_threads() { return kLamThreads; }


bool lambda_tc_applies(int d, int r2, int64_t lda, const void* A, l1s_dtype dt);
bool launch_lambda_tc(int64_t n, int d, int r2, const void* A, int64_t lda, const float* b, const float* m32,
                      uint16_t* mt_bf16, float* lam, double* block_sums, int blocks, uint32_t* flags, cudaStream_t st);

// M (FP32, q × r2 in the workspace) → constant bank, then λ and Σλ.  BF16 A with d = r2 = 32
// runs on the tensor cores (M_A rounded to BF16; its transpose goes to the Π2 region, 2 KB).
// With nsums_out non-NULL the Σλ/τ step is left to the sampling kernel: the number of
// block partials is returned there instead of launching the finalize kernel.
bool launch_lambda(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b,
                   const float* m32, const l1s_params* p, float* lam, double* user_sum,
                   unsigned char* ws, cudaStream_t st, int* nsums_out) {
  const bool smem_m = pl.lam_m_in_smem != 0;
  const bool tc = lambda_tc_applies(pl.d, pl.r2, lda, A, dt);
  double* sums = reinterpret_cast<double*>(ws + pl.off_lamsum);
  int blocks = pl.lam_ctas;
  bool ok;
  if (tc) {
    blocks = std::min(pl.lam_ctas, 3 * device_info().sms);   // three resident per SM (64 TMEM columns each)
    ok = launch_lambda_tc(pl.n, pl.d, pl.r2, A, lda, b, m32, reinterpret_cast<uint16_t*>(ws + pl.off_pi2), lam, sums,
                          blocks, reinterpret_cast<uint32_t*>(ws + pl.off_status), st);
  } else {
    if (dt == L1S_BF16)
      ok = smem_m ? launch_lambda_bf16_smem(pl, A, lda, b, lam, sums, m32, st)
                  : launch_lambda_bf16_const(pl, A, lda, b, lam, sums, m32, st);
    else
      ok = smem_m ? launch_lambda_f32_smem(pl, A, lda, b, lam, sums, m32, st)
                  : launch_lambda_f32_const(pl, A, lda, b, lam, sums, m32, st);
  }
  if (!ok) return false;
  if (nsums_out) {
    *nsums_out = blocks;
    return true;
  }
  lambda_finalize_kernel<<<1, 256, 0, st>>>(sums, blocks, p->coreset_size,
                                           reinterpret_cast<StatusBlock*>(ws + pl.off_status), user_sum);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch lambda_finalize");
}

bool launch_m_to_f32(const double* m, int total, float* out, cudaStream_t st) {
  m_to_f32_kernel<<<(total + 255) / 256, 256, 0, st>>>(m, total, out);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch m_to_f32");
}

}  // namespace l1s
