// The ℓ1 well-conditioned basis itself (§4.1, Figure 1: U = X·R⁻¹ with R from the QR of
// Π1·X) and its exact ℓ1 row norms ‖U_(i)‖₁ — the ℓ1 leverage scores that Figure 2's λ
// estimates by medians over Π2 — in FP64.  One thread per row: U_(i) solves U_(i)·R = X_(i)
// by forward substitution with R (q × q, upper triangular) in shared memory, so R⁻¹ is
// never formed.  Σ_i ‖U_(i)‖₁ = ‖U‖₁ (the α of an (α, β)-conditioned basis, §6.1) is
// summed per block and the block partials are added in a fixed order.  This pass is a
// validation tool (the conditioning quality of §6.1); the sampling pass does not use it.
#include <algorithm>

#include "l1s_common.cuh"

namespace l1s {

constexpr int kBasisThreads = 128;
constexpr int kBasisMaxBlocks = 1024;

template <typename TA>
__global__ void __launch_bounds__(kBasisThreads) l1_basis_kernel(const TA* __restrict__ A, int64_t lda,
                                                                 const float* __restrict__ b, int64_t n, int d,
                                                                 const double* __restrict__ R, double* __restrict__ U,
                                                                 double* __restrict__ rownorm,
                                                                 double* __restrict__ block_sums) {
  extern __shared__ double sR[];                      // R, row-major q × q
  __shared__ double wsum[kBasisThreads / 32];
  const int q = d + 1;
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) sR[e] = R[e];
  __syncthreads();
  double total = 0.0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    double u[kMaxD + 1];
    double norm = 0.0;
    for (int k = 0; k < q; ++k) {
      double x = k < d ? static_cast<double>(load_elem<TA>(A + i * lda + k)) : -static_cast<double>(__ldg(b + i));
      for (int m = 0; m < k; ++m) x = fma(-u[m], sR[m * q + k], x);
      u[k] = x / sR[k * q + k];
      norm += fabs(u[k]);
      if (U) U[i * q + k] = u[k];
    }
    if (rownorm) rownorm[i] = norm;
    total += norm;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) total += __shfl_down_sync(0xffffffffu, total, off);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = total;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kBasisThreads / 32; ++w) s += wsum[w];
    block_sums[blockIdx.x] = s;
  }
}

__global__ void basis_total_kernel(const double* __restrict__ block_sums, int nblocks, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nblocks; ++k) s += block_sums[k];
    *out = s;
  }
}

size_t basis_workspace_bytes() { return 256 + sizeof(double) * kBasisMaxBlocks; }

bool launch_basis(const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n, int d, const double* R,
                  double* U, double* rownorm, double* total, unsigned char* ws, cudaStream_t st) {
  const int q = d + 1;
  const int blocks = static_cast<int>(
      std::max<int64_t>(1, std::min<int64_t>(kBasisMaxBlocks, (n + kBasisThreads - 1) / kBasisThreads)));
  double* sums = reinterpret_cast<double*>(ws + 256);
  const size_t smem = sizeof(double) * q * q;
  if (dt == L1S_BF16) {
    if (!allow_dynamic_smem(reinterpret_cast<const void*>(l1_basis_kernel<uint16_t>), smem, "cudaFuncSetAttribute(l1_basis)"))
      return false;
    l1_basis_kernel<uint16_t><<<blocks, kBasisThreads, smem, st>>>(static_cast<const uint16_t*>(A), lda, b, n, d, R,
                                                                    U, rownorm, sums);
  } else {
    if (!allow_dynamic_smem(reinterpret_cast<const void*>(l1_basis_kernel<float>), smem, "cudaFuncSetAttribute(l1_basis)"))
      return false;
    l1_basis_kernel<float><<<blocks, kBasisThreads, smem, st>>>(static_cast<const float*>(A), lda, b, n, d, R, U,
                                                                 rownorm, sums);
  }
  count_launch(1);
  if (!cuda_ok(cudaGetLastError(), "launch l1_basis")) return false;
  if (total) {
    basis_total_kernel<<<1, 32, 0, st>>>(sums, blocks, total);
    count_launch(1);
    return cuda_ok(cudaGetLastError(), "launch basis_total");
  }
  return true;
}

}  // namespace l1s

using namespace l1s;

extern "C" int l1_basis(const void* A, int64_t lda, l1s_dtype dtype, const float* b, int64_t n, int32_t d,
                        const double* R_dev, double* U_dev, double* rownorm_dev, double* total_dev, void* ws,
                        size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_basis");
  if (!A || !b || !R_dev) return set_error("A, b and R must not be NULL"), L1S_ERR_INVALID_ARG;
  if (n < 1 || d < 1 || d > kMaxD || lda < d) return set_error("bad n, d or lda"), L1S_ERR_INVALID_ARG;
  if (dtype != L1S_F32 && dtype != L1S_BF16) return set_error("dtype must be L1S_F32 or L1S_BF16"), L1S_ERR_INVALID_ARG;
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < basis_workspace_bytes())
    return set_error("l1_basis needs a 256-byte aligned workspace of %zu bytes", basis_workspace_bytes()),
           L1S_ERR_WORKSPACE;
  if (!launch_basis(A, lda, dtype, b, n, d, R_dev, U_dev, rownorm_dev, total_dev, static_cast<unsigned char*>(ws),
                    static_cast<cudaStream_t>(stream)))
    return L1S_ERR_CUDA;
  return L1S_OK;
}
