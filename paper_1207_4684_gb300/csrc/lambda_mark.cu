// OptimizedFastCauchyRegression: λ̂ and the keep decision in one pass (Figure "mainOpt",
// steps 5-7), FP32 rows; kernels in lambda_kernels.cuh.
#include "lambda_kernels.cuh"

namespace l1s {

bool lambda_mark_applies(const Plan& pl, l1s_dtype dt, const l1s_params* p) {
  if (p->variant != 1 || dt != L1S_F32 || (pl.r2 != 8 && pl.r2 != 16)) return false;
  return pl.d == 4 || pl.d == 8 || pl.d == 16 || pl.d == 32;
}

// λ̂ and the keep mask of OptimizedFastCauchyRegression in one launch over pl.smp_ctas
// chunks of pl.smp_chunk rows (the compaction kernel then gathers the kept rows).
bool launch_lambda_mark(const Plan& pl, const void* A, int64_t lda, const float* b, const float* m32,
                        const l1s_params* p, float* lam_out, unsigned char* ws, cudaStream_t st) {
  const bool smem_m = pl.lam_m_in_smem != 0;
  if (!smem_m && !load_const_m(m32, pl.d, pl.r2, 0, st)) return false;
  LamMarkArgs a;
  a.A = A;
  a.lda = lda;
  a.b = b;
  a.n = pl.n;
  a.chunk = pl.smp_chunk;
  a.mg = m32;
  a.lam_out = lam_out;
  a.key = make_key(p->seed);
  a.problem = p->problem_id;
  a.row_offset = p->global_row_offset;
  a.tau = p->sample_scale;
  a.mask = reinterpret_cast<uint64_t*>(ws + pl.off_mask);
  a.counts = reinterpret_cast<int64_t*>(ws + pl.off_counts);
  a.status = reinterpret_cast<StatusBlock*>(ws + pl.off_status);
  const bool aligned = (reinterpret_cast<uintptr_t>(A) % 16 == 0) && ((lda * 4) % 16 == 0);
  const int grid = pl.smp_ctas;
#define L1S_LM_CASE(DD, RR)                                                                        \
  if (pl.d == DD && pl.r2 == RR) {                                                                 \
    if (smem_m) launch_lambda_mark_case<DD, RR, float, true>(grid, st, aligned, a);                \
    else launch_lambda_mark_case<DD, RR, float, false>(grid, st, aligned, a);                      \
    count_launch(1);                                                                               \
    return cuda_ok(cudaGetLastError(), "launch lambda_mark");                                      \
  }
  L1S_LM_CASE(4, 8)
  L1S_LM_CASE(8, 8)
  L1S_LM_CASE(16, 8)
  L1S_LM_CASE(32, 8)
  L1S_LM_CASE(4, 16)
  L1S_LM_CASE(8, 16)
  L1S_LM_CASE(16, 16)
  L1S_LM_CASE(32, 16)
#undef L1S_LM_CASE
  return set_error("lambda_mark: no kernel for d = %d, r2 = %d", pl.d, pl.r2), false;
}

}  // namespace l1s
