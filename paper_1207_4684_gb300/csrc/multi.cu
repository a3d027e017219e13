// Multiple ℓ1 regression (§4.2.1): min_W ‖A·W − B‖₁ with B ∈ R^{n×k}, by the same steps
// on X = [A, −B] (q = d + k columns), one coreset for all k right-hand sides, then k
// weighted ℓ1 problems on it.
//
// The caller's matrix holds [A | B] row by row (n × (d + k), leading dimension ldx).  The
// passes of the single right-hand-side path read an "A" of d + k − 1 columns and a
// separate FP32 "b" that they negate; here that A is the caller's first d + k − 1 columns
// (so B_1 … B_{k−1} enter with a + sign) and b is B_k, gathered once into the workspace.
// With D = diag(1_d, −1_{k−1}, 1) the passes therefore see X·D.  Π1(X·D) = (Π1X)·D, its R
// factor is D·R·D, and with Π2's rows d … d+k−2 drawn negated (D·Π2) the conditioning gives
// M' = (D R D)⁻¹·D·Π2 = D·R⁻¹·Π2, so (X·D)·M' = X·R⁻¹·Π2: λ, p̂ and the coreset are those
// of X = [A, −B] with the same draws.  The gathered coreset rows negate the same columns
// back, so they are rows of X.
#include <math.h>
#include <stdlib.h>

#include <algorithm>

#include "l1s_common.cuh"

namespace l1s {

int64_t coreset_capacity_of(const l1s_params* p);
bool check_ws(const Plan& pl, const void* ws, size_t ws_bytes);
int first_error(uint32_t flags);
int coreset_impl(const Plan& pl, const void* A, int64_t lda, l1s_dtype dtype, const float* b,
                 const l1s_params* params, int64_t capacity, int64_t* idx, double* wts, double* coreset,
                 int64_t* count, unsigned char* w, cudaStream_t st);
bool launch_objective(const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n, int d,
                      const double* x, double* out, int nblocks, double* partials, cudaStream_t st);

// Column c of the caller's matrix as contiguous FP32 (exact for FP32 and BF16 storage).
template <typename TA>
__global__ void column_to_f32_kernel(const TA* __restrict__ X, int64_t ldx, int c, int64_t n, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = load_elem<TA>(X + i * ldx + c);
}

// Coreset rows of one right-hand side: [X_i(0..d−1), X_i(d + j)] = [A_i, −B_ij].
__global__ void coreset_select_kernel(const double* __restrict__ core, int q, int d, int j, int64_t capacity,
                                      double* __restrict__ out) {
  const int64_t total = capacity * (d + 1);
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / (d + 1);
    const int c = static_cast<int>(e - r * (d + 1));
    out[e] = core[r * q + (c < d ? c : d + j)];
  }
}

struct MultiLayout {
  Plan pl;           // the single right-hand-side plan with d + k − 1 columns in "A"
  int64_t cap;
  size_t off_bcol;   // n FP32: B_k for the passes, then B_j for objective j
  size_t off_core;   // the coreset (cap × (d + k) FP64), its weights and indices
  size_t off_sel;    // cap × (d + 1) FP64: coreset rows of one right-hand side
  size_t off_out;    // k × (d + 1) FP64: x_j and the coreset objective of each j; k full objectives
  size_t total;
};

static bool multi_layout(const l1s_params* p, int64_t n, int d, int k, l1s_dtype dt, MultiLayout* L) {
  if (d < 1 || k < 1 || d + k - 1 > kMaxD)
    return set_error("multiple regression needs d >= 1, k >= 1 and d + k - 1 <= %d", kMaxD), false;
  if (!make_plan(p, n, d + k - 1, dt, false, &L->pl)) return false;
  L->pl.pi2_neg_lo = d;
  L->pl.pi2_neg_hi = d + k - 1;
  L->cap = coreset_capacity_of(p);
  size_t off = L->pl.total;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const int q = d + k;
  L->off_bcol = take(sizeof(float) * static_cast<size_t>(n));
  L->off_core = take(static_cast<size_t>(L->cap) * (sizeof(int64_t) + sizeof(double) + sizeof(double) * q));
  L->off_sel = take(static_cast<size_t>(L->cap) * sizeof(double) * (d + 1));
  L->off_out = take(sizeof(double) * static_cast<size_t>(k) * (d + 2));
  L->total = off;
  return true;
}

static bool launch_column(const void* X, int64_t ldx, l1s_dtype dt, int c, int64_t n, float* out, cudaStream_t st) {
  const int blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, 4 * device_info().sms));
  if (dt == L1S_BF16)
    column_to_f32_kernel<uint16_t><<<blocks, 256, 0, st>>>(static_cast<const uint16_t*>(X), ldx, c, n, out);
  else
    column_to_f32_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(X), ldx, c, n, out);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch column_to_f32");
}

static bool check_x(const void* X, int64_t ldx, int d, int k) {
  if (!X) return set_error("X must not be NULL"), false;
  if (ldx < static_cast<int64_t>(d) + k) return set_error("ldx must be >= d + k"), false;
  return true;
}

static int coreset_multi_impl(const MultiLayout& M, const void* X, int64_t ldx, l1s_dtype dtype, int d, int k,
                              const l1s_params* params, int64_t capacity, int64_t* idx, double* wts,
                              double* coreset, int64_t* count, unsigned char* w, cudaStream_t st) {
  float* bcol = reinterpret_cast<float*>(w + M.off_bcol);
  if (!launch_column(X, ldx, dtype, d + k - 1, M.pl.n, bcol, st)) return L1S_ERR_CUDA;
  return coreset_impl(M.pl, X, ldx, dtype, bcol, params, capacity, idx, wts, coreset, count, w, st);
}

}  // namespace l1s

using namespace l1s;

extern "C" {

int l1s_multi_workspace_size(const l1s_params* params, int64_t n, int32_t d, int32_t k, l1s_dtype dtype,
                             size_t* bytes) {
  if (!bytes) return set_error("bytes is NULL"), L1S_ERR_INVALID_ARG;
  MultiLayout M;
  if (!multi_layout(params, n, d, k, dtype, &M)) return L1S_ERR_INVALID_ARG;
  *bytes = M.total;
  return L1S_OK;
}

int l1_coreset_multi(const void* X, int64_t ldx, l1s_dtype dtype, int64_t n, int32_t d, int32_t k,
                     const l1s_params* params, int64_t capacity, int64_t* idx, double* wts, double* coreset,
                     int64_t* count, void* ws, size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_coreset_multi");
  MultiLayout M;
  if (!multi_layout(params, n, d, k, dtype, &M)) return L1S_ERR_INVALID_ARG;
  if (!check_x(X, ldx, d, k)) return L1S_ERR_INVALID_ARG;
  if (capacity < 0 || (capacity > 0 && (!idx || !wts)) || !count)
    return set_error("idx, w (capacity > 0) and count must not be NULL"), L1S_ERR_INVALID_ARG;
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < M.total)
    return set_error("workspace too small or misaligned: %zu bytes needed", M.total), L1S_ERR_WORKSPACE;
  return coreset_multi_impl(M, X, ldx, dtype, d, k, params, capacity, idx, wts, coreset, count,
                            static_cast<unsigned char*>(ws), static_cast<cudaStream_t>(stream));
}

int l1_regress_multi(const void* X, int64_t ldx, l1s_dtype dtype, int64_t n, int32_t d, int32_t k,
                     const l1s_params* params, int32_t max_iter, double* W_host, double* objectives_host,
                     int64_t* coreset_rows_host, void* ws, size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_regress_multi");
  MultiLayout M;
  if (!multi_layout(params, n, d, k, dtype, &M)) return L1S_ERR_INVALID_ARG;
  if (!check_x(X, ldx, d, k) || !W_host || !objectives_host) return set_error("NULL argument"), L1S_ERR_INVALID_ARG;
  if (max_iter < 0 || max_iter > 100000) return set_error("max_iter must be in [0, 100000]"), L1S_ERR_INVALID_ARG;
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < M.total)
    return set_error("workspace too small or misaligned: %zu bytes needed", M.total), L1S_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  const int q = d + k;
  const int64_t cap = M.cap;
  int64_t* idx = reinterpret_cast<int64_t*>(w + M.off_core);
  double* wts = reinterpret_cast<double*>(idx + cap);
  double* core = wts + cap;
  double* sel = reinterpret_cast<double*>(w + M.off_sel);
  double* outs = reinterpret_cast<double*>(w + M.off_out);   // [k][d + 1], then k full objectives
  double* full = outs + static_cast<size_t>(k) * (d + 1);
  StatusBlock* sb = reinterpret_cast<StatusBlock*>(w + M.pl.off_status);
  int rc = coreset_multi_impl(M, X, ldx, dtype, d, k, params, cap, idx, wts, core, &sb->count, w, st);
  if (rc != L1S_OK) return rc;
  float* bcol = reinterpret_cast<float*>(w + M.off_bcol);
  const int sel_blocks = static_cast<int>(std::min<int64_t>((cap * (d + 1) + 255) / 256, 1024));
  for (int j = 0; j < k; ++j) {
    double* xj = outs + static_cast<size_t>(j) * (d + 1);
    coreset_select_kernel<<<sel_blocks, 256, 0, st>>>(core, q, d, j, cap, sel);
    count_launch(1);
    if (!cuda_ok(cudaGetLastError(), "launch coreset_select")) return L1S_ERR_CUDA;
    rc = l1_solve(sel, wts, &sb->count, cap, d, max_iter, xj, xj + d, ws, ws_bytes, stream);
    if (rc != L1S_OK) return rc;
    if (!launch_column(X, ldx, dtype, d + j, n, bcol, st) ||
        !launch_objective(X, ldx, dtype, bcol, n, d, xj, full + j, M.pl.lam_ctas,
                          reinterpret_cast<double*>(w + M.pl.off_lamsum), st))
      return L1S_ERR_CUDA;
  }
  const size_t nres = static_cast<size_t>(k) * (d + 2);
  double* res = static_cast<double*>(malloc(sizeof(double) * nres));
  if (!res) return set_error("host allocation failed"), L1S_ERR_INVALID_ARG;
  int64_t cnt = 0;
  if (!cuda_ok(cudaMemcpyAsync(res, outs, sizeof(double) * nres, cudaMemcpyDeviceToHost, st), "copy W") ||
      !cuda_ok(cudaMemcpyAsync(&cnt, &sb->count, sizeof(cnt), cudaMemcpyDeviceToHost, st), "copy count")) {
    free(res);
    return L1S_ERR_CUDA;
  }
  uint32_t flags = 0;
  if (l1s_status_read(ws, ws_bytes, stream, &flags) != L1S_OK) {
    free(res);
    return L1S_ERR_CUDA;
  }
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < d; ++i) W_host[static_cast<size_t>(i) * k + j] = res[static_cast<size_t>(j) * (d + 1) + i];
    objectives_host[j] = res[static_cast<size_t>(k) * (d + 1) + j];
  }
  free(res);
  if (coreset_rows_host) *coreset_rows_host = cnt;
  return first_error(flags);
}

}  // extern "C"
