// Phase 2 (Figure 2, steps 4-5), FP32 CUDA-core λ kernels for BF16 rows, M in the constant bank.
#include "lambda_kernels.cuh"

namespace l1s {

bool launch_lambda_bf16_const(const Plan& pl, const void* A, int64_t lda, const float* b, float* lam, double* sums,
                         const float* m32, cudaStream_t st) {
  return launch_lambda_t<uint16_t, false>(pl, static_cast<const uint16_t*>(A), lda, b, lam, sums, m32, st);
}

}  // namespace l1s
