// l1_lambda_noalloc: the λ pass for callers that cannot allocate device memory.
//
// The ordinary entry points take a caller-allocated workspace.  Some callers
// cannot provide one: cudaMalloc may synchronise the whole device, which a
// latency-bound loop cannot afford once it is running, and some host programs
// hand all device memory to their own pool at start-up and give plug-in code no
// way to allocate.  This entry point needs no workspace: its scratch (the FP32
// copy of M, the per-block Σλ partials and a status block) lives in one
// file-scope __device__ array of kScratchBytes bytes, which every GPU that
// loads the library holds until the process exits.
//
// The device address of that array is looked up once per device with
// cudaGetSymbolAddress, on the first call made with that device current; make
// that first call before any stream capture.  All calls share the array, and
// it keeps whatever the last call left in it: the status block is cleared at
// the start of every call, the rest is overwritten before it is read.  Calls
// whose work overlaps on the GPU (different streams, or threads) race on the
// array and on M's constant bank.  Nothing here calls cudaMalloc, cudaFree or
// an allocating library routine.
#include <mutex>

#include "l1s_common.cuh"

namespace l1s {

bool launch_lambda(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b,
                   const float* m32, const l1s_params* p, float* lam, double* user_sum,
                   unsigned char* ws, cudaStream_t st, int* nsums_out = nullptr);
bool launch_m_to_f32(const double* m, int total, float* out, cudaStream_t st);

constexpr size_t kScratchBytes = 40 * 1024;  // holds q·r2 up to 65·64 with 1216 partial sums

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch on the current device (looked up once per device).
static bool scratch_on_current_device(unsigned char** out) {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = 0;
  if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return false;
  if (dev < 0 || dev >= 64) return set_error("device ordinal out of range"), false;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (!cuda_ok(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(no-alloc scratch)"))
      return false;
    addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(addr[dev]);
  return true;
}

}  // namespace l1s

using namespace l1s;

extern "C" int l1_lambda_noalloc(const void* A, int64_t lda, l1s_dtype dtype, const float* b, int64_t n,
                                 int32_t d, const double* M, const l1s_params* params, float* lambda,
                                 double* lambda_sum, void* stream) {
  Plan pl;
  if (!make_plan(params, n, d, dtype, false, &pl)) return L1S_ERR_INVALID_ARG;
  if (!A || !b || !M || !lambda || lda < d) return set_error("A, b, M, lambda must be given and lda >= d"), L1S_ERR_INVALID_ARG;
  // Scratch layout: status block | Σλ block partials | M in FP32 | M_Aᵀ in BF16 (tensor-core form).
  const size_t off_sums = 256;
  const size_t off_m32 = align_up(off_sums + sizeof(double) * static_cast<size_t>(pl.lam_ctas));
  const size_t off_mt = align_up(off_m32 + sizeof(float) * static_cast<size_t>(pl.q) * pl.r2);
  const size_t need = off_mt + 4096;                        // M_Aᵀ of the tensor-core form: r2 × 64 BF16 at most
  if (need > kScratchBytes)
    return set_error("l1_lambda_noalloc: q·r2 = %d and %d partial sums need %zu bytes, more than its %zu-byte scratch",
                     pl.q * pl.r2, pl.lam_ctas, need, kScratchBytes),
           L1S_ERR_INVALID_ARG;
  unsigned char* scratch = nullptr;
  if (!scratch_on_current_device(&scratch)) return L1S_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Plan local = pl;
  local.off_status = 0;
  local.off_lamsum = off_sums;
  local.off_m32 = off_m32;
  local.off_pi2 = off_mt;
  float* m32 = reinterpret_cast<float*>(scratch + off_m32);
  if (!cuda_ok(cudaMemsetAsync(scratch, 0, sizeof(StatusBlock), st), "clear no-alloc status")) return L1S_ERR_CUDA;
  if (!launch_m_to_f32(M, pl.q * pl.r2, m32, st)) return L1S_ERR_CUDA;
  if (!launch_lambda(local, A, lda, dtype, b, m32, params, lambda, lambda_sum, scratch, st)) return L1S_ERR_CUDA;
  return L1S_OK;
}
