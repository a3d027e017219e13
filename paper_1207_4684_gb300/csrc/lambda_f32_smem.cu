// Phase 2 (Figure 2, steps 4-5), FP32 CUDA-core λ kernels for FP32 rows, M in shared memory.
#include "lambda_kernels.cuh"

namespace l1s {

bool launch_lambda_f32_smem(const Plan& pl, const void* A, int64_t lda, const float* b, float* lam, double* sums,
                         const float* m32, cudaStream_t st) {
  return launch_lambda_t<float, true>(pl, static_cast<const float*>(A), lda, b, lam, sums, m32, st);
}

}  // namespace l1s
