// C ABI of libl1fct: argument checks, workspace layout, and the order in which
// the kernels of each entry point are enqueued.  See include/l1fct.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>

#include "l1s_common.cuh"

namespace l1s {

// kernels (defined in the other translation units)
const void* fct_kernel(int log2s, l1s_dtype dt, bool staged);
size_t fct_smem_bytes(int s, int d, l1s_dtype dt, int r1, int width, bool staged);
int fct_threads_for(int log2s, int width);
int fct_ws_width(int log2s, int d);
int fct_ws_tile_log2(int log2s);
const void* fct_ws_kernel(int log2t, int log2s, l1s_dtype dt, int w, bool lean);
int fct_ws_threads(int w);
size_t fct_ws_smem_bytes(int s, int d, l1s_dtype dt, int r1, int w, bool lean);
int fct_sorted_width(int log2s, int d);
const void* fct_sorted_kernel(int log2s, l1s_dtype dt, int w);
int fct_sorted_threads(int w);
size_t fct_sorted_smem_bytes(int s, int d, l1s_dtype dt, int r1, int w);
int fct_cols_slices(int log2s, int d, int r1, int max_smem);
int sct_width(int q);
int sct_ctas(int64_t n, int r1, int q, int sms);
size_t fct_cols_smem_bytes(int r1);
int fct_cols_threads();
int fct_cols_tile();
const void* fct_cols_kernel(l1s_dtype dt, bool full);
size_t fct_cols_partial_floats(int slices, int ctas, int r1, int64_t n);
bool launch_fct(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b,
                const l1s_params* p, float* pix, unsigned char* ws, cudaStream_t st, double* pi2_out = nullptr);
bool launch_fct_streamed(const Plan& pl, const void* A_host, int64_t lda_host, l1s_dtype dt, const float* b_host,
                         void* A_dev, float* b_dev, const l1s_params* p, float* pix, unsigned char* ws,
                         cudaStream_t st, cudaStream_t cp, const cudaEvent_t* evs, double* pi2_out);
bool launch_condition(const Plan& pl, const float* pix, const l1s_params* p, double* R_user,
                      double* M_user, unsigned char* ws, cudaStream_t st, bool pi2_ready = false);
bool launch_pi2(const l1s_params* p, int q, double* out, cudaStream_t st);
size_t cond2_scratch_bytes(int r1, int q, int sms);
int lambda_threads();
bool launch_lambda(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b,
                   const float* m32, const l1s_params* p, float* lam, double* user_sum,
                   unsigned char* ws, cudaStream_t st, int* nsums_out = nullptr);
bool launch_m_to_f32(const double* m, int total, float* out, cudaStream_t st);
bool lambda_mark_applies(const Plan& pl, l1s_dtype dt, const l1s_params* p);
bool launch_debug_wait(uint32_t* flags, long long max_cycles, cudaStream_t st);
bool launch_replacement(const Plan& pl, const float* lam, const l1s_params* prm, const void* A, int64_t lda,
                        l1s_dtype dt, const float* b, int64_t capacity, int64_t* idx, double* w, double* coreset,
                        int64_t* count_out, unsigned char* ws, cudaStream_t st);
bool launch_lambda_mark(const Plan& pl, const void* A, int64_t lda, const float* b, const float* m32,
                        const l1s_params* p, float* lam_out, unsigned char* ws, cudaStream_t st);
bool launch_compact(const Plan& pl, const float* lam, const float* m32, const void* A, int64_t lda, l1s_dtype dt,
                    const float* b, int64_t capacity, int64_t* idx, double* w, double* coreset, int64_t* count_out,
                    unsigned char* ws, cudaStream_t st);
int sample_threads();
bool launch_sample(const Plan& pl, const float* lam, const double* p, const l1s_params* prm,
                   const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t capacity,
                   int64_t* idx, double* w, double* coreset, int64_t* count_out, unsigned char* ws,
                   cudaStream_t st, int lam_nsums = 0);
size_t sample_many_extra_bytes(const Plan& pl, int k);
bool launch_sample_many(const Plan& pl, const float* lam, const double* lam_total, const l1s_params* prm, int k,
                        const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t capacity, int64_t* idx,
                        double* w, double* coreset, int64_t* count_out, unsigned char* ws, cudaStream_t st);
bool launch_debug_variates(const l1s_params* p, int64_t row_start, int64_t count, int32_t* bh,
                           int32_t* bi, int32_t* kh, int32_t* ki, float* ch, float* ci, int8_t* sg,
                           uint64_t* ub, cudaStream_t st);
int irls_entries(int q);
size_t irls_state_bytes();
size_t solve_scratch_bytes(int64_t capacity);
bool launch_solve(const double* X, const double* w, const int64_t* count, int64_t capacity, int d,
                  int max_iter, double* x_out, double* obj_out, int nblocks, double* partials,
                  void* state, float* scratch, StatusBlock* status, cudaStream_t st, int k,
                  uint32_t* flags_out);
bool launch_objective(const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n, int d,
                      const double* x, double* out, int nblocks, double* partials, cudaStream_t st);

static thread_local char g_err[512] = "";
static std::atomic<uint64_t> g_launches{0};

void count_launch(int k) { g_launches.fetch_add(static_cast<uint64_t>(k), std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

bool cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return false;
}

bool allow_dynamic_smem(const void* fn, size_t bytes, const char* what) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> granted;
  int dev = 0;
  if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return false;
  std::lock_guard<std::mutex> lock(mu);
  size_t& g = granted[std::make_pair(dev, fn)];
  if (bytes <= g) return true;
  if (!cuda_ok(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)), what))
    return false;
  g = bytes;
  return true;
}

DeviceInfo device_info() {
  static std::mutex mu;
  static DeviceInfo cache[64];
  static bool have[64] = {};
  DeviceInfo di{-1, 0, 0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return di;
  std::lock_guard<std::mutex> lock(mu);
  if (!have[dev]) {
    cache[dev].device = dev;
    cudaDeviceGetAttribute(&cache[dev].sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&cache[dev].max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    have[dev] = true;
  }
  return cache[dev];
}

static bool check_params(const l1s_params* p, int64_t n, int d) {
  if (!p) return set_error("params is NULL"), false;
  if (n < 1) return set_error("n must be >= 1 (got %lld)", (long long)n), false;
  if (d < 1 || d > kMaxD) return set_error("d must be in [1, %d] (got %d)", kMaxD, d), false;
  const int l2 = log2_exact(p->s);
  if (p->s < 1 || l2 < 0 || l2 > kMaxLog2S)
    return set_error("s must be a power of two in [1, 4096] (got %d)", p->s), false;
  if (p->r1 < d + 1 || p->r1 > 65535)
    return set_error("r1 must be in [q, 65535] with q = d+1 = %d (got %d)", d + 1, p->r1), false;
  if (p->r2 < 1 || p->r2 > kMaxR2) return set_error("r2 must be in [1, %d] (got %d)", kMaxR2, p->r2), false;
  if (!(p->coreset_size > 0.0) || !isfinite(p->coreset_size))
    return set_error("coreset_size must be positive and finite"), false;
  if (p->global_row_offset < 0 || p->global_row_offset % p->s != 0)
    return set_error("global_row_offset must be a non-negative multiple of s"), false;
  if (p->sign_flip != 0 && p->sign_flip != 1) return set_error("sign_flip must be 0 or 1"), false;
  if (p->variant < 0 || p->variant > 2) return set_error("variant must be 0, 1 or 2"), false;
  if (p->variant != 1 && p->sample_scale != 0.0) return set_error("sample_scale must be 0 for variants 0 and 2"), false;
  if (p->variant == 2 && (p->coreset_size != floor(p->coreset_size) || p->coreset_size > 1e9))
    return set_error("variant 2 draws coreset_size rows: it must be an integer in [1, 1e9]"), false;
  if (p->variant == 1 && (!(p->sample_scale > 0.0) || !isfinite(p->sample_scale)))
    return set_error("variant 1 needs a positive, finite sample_scale"), false;
  if (p->transform < 0 || p->transform > 2) return set_error("transform must be 0, 1 or 2"), false;
  if (p->transform == 2 && (p->fjlt_rows < 0 || p->fjlt_rows > p->s))
    return set_error("transform 2: fjlt_rows must be in [0, s] (got %d)", p->fjlt_rows), false;
  return true;
}


int64_t coreset_capacity_of(const l1s_params* p) {
  return static_cast<int64_t>(ceil(2.0 * p->coreset_size)) + 64;
}

bool check_ws(const Plan& pl, const void* ws, size_t ws_bytes) {
  if (!ws) return set_error("workspace is NULL"), false;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return set_error("workspace must be 256-byte aligned"), false;
  if (ws_bytes < pl.total)
    return set_error("workspace too small: %zu bytes given, %zu needed", ws_bytes, pl.total), false;
  return true;
}

bool check_a(const void* A, int64_t lda, const float* b, int d) {
  if (!A || !b) return set_error("A and b must not be NULL"), false;
  if (lda < d) return set_error("lda must be >= d"), false;
  return true;
}

int first_error(uint32_t flags) {
  for (int code = L1S_ERR_RANK_DEFICIENT; code <= L1S_ERR_CAPACITY; ++code)
    if (flags & L1S_FLAG(code)) return code;
  if (flags & L1S_FLAG(L1S_ERR_TIMEOUT)) return L1S_ERR_TIMEOUT;
  return L1S_OK;
}

int sample_impl(const Plan& pl, const void* A, int64_t lda, l1s_dtype dtype, const float* b,
                       const float* m32, const l1s_params* params, int64_t capacity, int64_t* idx,
                       double* wts, double* coreset, int64_t* count, float* lambda, unsigned char* w,
                       cudaStream_t st) {
  // OptimizedFastCauchyRegression needs no Σλ: λ̂ and the keep mask come from one pass,
  // and the compaction recomputes λ̂ of the kept rows unless the caller wants every λ̂.
  if (lambda_mark_applies(pl, dtype, params)) {
    Plan pf = pl;
    pf.smp_chunk = pl.lm_chunk;
    pf.smp_ctas = pl.lm_ctas;
    if (!launch_lambda_mark(pf, A, lda, b, m32, params, lambda, w, st) ||
        !launch_compact(pf, lambda, m32, A, lda, dtype, b, capacity, idx, wts, coreset, count, w, st))
      return L1S_ERR_CUDA;
    return L1S_OK;
  }
  float* lam = lambda ? lambda : reinterpret_cast<float*>(w + pl.off_lam);
  if (params->variant == 2) {
    int nsums = 0;
    if (!launch_lambda(pl, A, lda, dtype, b, m32, params, lam, nullptr, w, st, &nsums) ||
        !launch_replacement(pl, lam, params, A, lda, dtype, b, capacity, idx, wts, coreset, count, w, st))
      return L1S_ERR_CUDA;
    return L1S_OK;
  }
  // Σλ and τ are formed at the start of the sampling kernel; OptimizedFastCauchyRegression
  // (variant 1) needs no Σλ at all.
  int nsums = 0;
  if (!launch_lambda(pl, A, lda, dtype, b, m32, params, lam, nullptr, w, st, &nsums)) return L1S_ERR_CUDA;
  if (!launch_sample(pl, lam, nullptr, params, A, lda, dtype, b, capacity, idx, wts, coreset, count, w, st,
                     params->variant == 1 ? 0 : nsums))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

int coreset_impl(const Plan& pl, const void* A, int64_t lda, l1s_dtype dtype, const float* b,
                        const l1s_params* params, int64_t capacity, int64_t* idx, double* wts,
                        double* coreset, int64_t* count, unsigned char* w, cudaStream_t st) {
  if (!cuda_ok(cudaMemsetAsync(w + pl.off_status, 0, sizeof(StatusBlock), st), "status reset"))
    return L1S_ERR_CUDA;
  float* pix = reinterpret_cast<float*>(w + pl.off_pix);
  // Π2 is drawn by the phase-1 reduction, off the conditioning's serial path.
  if (!launch_fct(pl, A, lda, dtype, b, params, pix, w, st, reinterpret_cast<double*>(w + pl.off_pi2)))
    return L1S_ERR_CUDA;
  if (!launch_condition(pl, pix, params, nullptr, nullptr, w, st, true)) return L1S_ERR_CUDA;
  return sample_impl(pl, A, lda, dtype, b, reinterpret_cast<float*>(w + pl.off_m32), params, capacity, idx,
                     wts, coreset, count, nullptr, w, st);
}

// Geometry of one phase-1 kernel variant for a shape: which kernel, its column slicing,
// shared memory, threads, and the resident blocks per SM that occupancy allows.
struct FctGeometry {
  bool ok;
  bool staged;
  int ws;                 // column width of the narrow-X kernel, 0 otherwise
  int tile_log2;          // its tile
  bool lean;              // its one-stage, one-copy form
  int sorted;             // column width of the bucket-sorted kernel, 0 otherwise
  int cols;               // slices of the column-sliced wide-X kernel, 0 otherwise
  int slices, width, threads, per_sm;
  size_t smem;
};

static FctGeometry fct_geometry(int variant, const Plan& P, l1s_dtype dt, const DeviceInfo& di) {
  FctGeometry g{};
  const size_t budget2 = std::min<size_t>(110 * 1024, di.max_smem_optin);
  const size_t budget1 = di.max_smem_optin;
  int width = P.q;
  bool staged = false;
  if (variant == 7) {
    // The column-sliced wide-X kernel: 16 columns of A per block, one block per SM.
    const int sl = P.d > 16 ? fct_cols_slices(P.log2s, P.d, P.r1, di.max_smem_optin) : 0;
    if (!sl) return g;
    g.cols = sl;
    g.tile_log2 = 10;
    g.slices = sl;
    g.width = 16;
    g.smem = fct_cols_smem_bytes(P.r1);
    g.threads = fct_cols_threads();
    const void* fn = fct_cols_kernel(dt, P.log2s == 10);
    if (!allow_dynamic_smem(reinterpret_cast<const void*>(fn), g.smem, "cudaFuncSetAttribute(fct_embed_cols)"))
      return g;
    int per_sm = 0;
    if (!cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, g.threads, g.smem), "occupancy(fct_cols)") ||
        per_sm < 1)
      return g;
    g.per_sm = per_sm;
    g.ok = true;
    return g;
  }
  if (variant == 4) {
    const int w = fct_sorted_width(P.log2s, P.d);
    if (!w || fct_sorted_smem_bytes(P.s, P.d, dt, P.r1, w) > budget1) return g;
    g.sorted = w;
    staged = true;
  } else if (variant == 1 || variant == 5) {
    const int w = fct_ws_width(P.log2s, P.d);
    const bool lean = variant == 5;
    if (!w || (lean && w != 16) ||
        fct_ws_smem_bytes(1 << fct_ws_tile_log2(P.log2s), P.d, dt, P.r1, w, lean) > budget1)
      return g;
    g.ws = w;
    g.lean = lean;
    g.tile_log2 = fct_ws_tile_log2(P.log2s);
    staged = true;
  } else if (variant == 2) {
    if (fct_smem_bytes(P.s, P.d, dt, P.r1, P.q, true) > budget1) return g;
    staged = true;
  } else {
    // Direct loads: the widest column slice whose shared-memory footprint allows two
    // blocks per SM, or failing that one (variant 6: the widest for one block per SM,
    // fewer slices re-reading X and redrawing the row variates).
    int slices = 1;
    for (;; ++slices) {
      width = (P.q + slices - 1) / slices;
      if (fct_smem_bytes(P.s, P.d, dt, P.r1, width, false) <= budget2 || width == 1) break;
    }
    if (variant == 6 || fct_smem_bytes(P.s, P.d, dt, P.r1, width, false) > budget2) {
      for (slices = 1;; ++slices) {
        width = (P.q + slices - 1) / slices;
        if (fct_smem_bytes(P.s, P.d, dt, P.r1, width, false) <= budget1) break;
        if (width == 1) return g;
      }
    }
  }
  g.staged = staged;
  g.slices = (P.q + width - 1) / width;
  g.width = width;
  g.smem = g.sorted ? fct_sorted_smem_bytes(P.s, P.d, dt, P.r1, g.sorted)
                    : (g.ws ? fct_ws_smem_bytes(1 << g.tile_log2, P.d, dt, P.r1, g.ws, g.lean)
                            : fct_smem_bytes(P.s, P.d, dt, P.r1, width, staged));
  g.threads = g.sorted ? fct_sorted_threads(g.sorted) : (g.ws ? fct_ws_threads(g.ws) : fct_threads_for(P.log2s, width));
  const void* fn = g.sorted ? fct_sorted_kernel(P.log2s, dt, g.sorted)
                            : (g.ws ? fct_ws_kernel(g.tile_log2, P.log2s, dt, g.ws, g.lean)
                                    : fct_kernel(P.log2s, dt, staged));
  if (!allow_dynamic_smem(reinterpret_cast<const void*>(fn), g.smem, "cudaFuncSetAttribute(fct_embed)"))
    return g;
  int per_sm = 0;
  if (!cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, g.threads, g.smem),
               "occupancy(fct_embed)"))
    return g;
  g.per_sm = std::max(per_sm, 1);
  g.ok = true;
  return g;
}

static int64_t fct_ctas_of(const FctGeometry& g, const Plan& P, const DeviceInfo& di, int per_sm) {
  const int64_t want = std::max<int64_t>(1, static_cast<int64_t>(di.sms) * per_sm / g.slices);
  const int64_t tiles = (g.ws || g.cols) ? (P.n + (int64_t{1} << g.tile_log2) - 1) >> g.tile_log2 : P.nblocks;
  return std::min<int64_t>(tiles, want);
}

// Bounds of the schedule fields (the workspace is sized for the largest).
constexpr int kMaxLamPerSm = 32;
constexpr int kMaxSmpPerSm = 16;
constexpr int kMaxChunks = 8;

bool make_plan(const l1s_params* p, int64_t n, int d, l1s_dtype dt, bool host_staging, Plan* pl,
               const l1s_schedule* override_sch) {
  if (!check_params(p, n, d)) return false;
  if (dt != L1S_F32 && dt != L1S_BF16) return set_error("dtype must be L1S_F32 or L1S_BF16"), false;
  const DeviceInfo di = device_info();
  if (di.device < 0 || di.sms <= 0) return set_error("no CUDA device"), false;
  Plan& P = *pl;
  memset(&P, 0, sizeof(P));
  P.n = n;
  P.d = d;
  P.q = d + 1;
  P.s = p->s;
  P.log2s = log2_exact(p->s);
  P.r1 = p->r1;
  P.r2 = p->r2;
  P.nblocks = (n + P.s - 1) / P.s;
  l1s_schedule sch{};
  if (override_sch)
    sch = *override_sch;
  else
    schedule_lookup(d, dt, P.log2s, &sch);

  // Phase 1.  Default: the warp-specialised narrow-X kernel where it applies, else all q
  // columns in one block with TMA-staged X tiles, else direct loads over column slices.
  // The bucket-sorted kernel is a schedule choice (slower than the narrow-X kernel on the
  // shapes measured so far).
  FctGeometry geo[8];
  for (int v = 1; v <= 7; ++v) geo[v] = fct_geometry(v, P, dt, di);
  if (!geo[3].ok) return set_error("r1 and s too large for shared memory"), false;
  // Wide X (d > 32): the column-sliced kernel where it fits.
  int variant = geo[1].ok ? 1 : (geo[2].ok ? 2 : (P.d > 32 && geo[7].ok ? 7 : 3));
  if (sch.fct_variant >= 1 && sch.fct_variant <= 7 && geo[sch.fct_variant].ok) variant = sch.fct_variant;
  const FctGeometry& g = geo[variant];
  P.fct_ws = g.ws;
  P.fct_tile_log2 = g.tile_log2;
  P.fct_lean = g.lean ? 1 : 0;
  P.fct_sorted = g.sorted;
  P.fct_cols = g.cols;
  P.fct_staged = g.staged ? 1 : 0;
  P.fct_slices = g.slices;
  P.fct_width = g.width;
  P.fct_smem = g.smem;
  P.fct_threads = g.threads;
  const int per_sm = sch.fct_ctas_per_sm > 0 ? std::min(sch.fct_ctas_per_sm, g.per_sm) : g.per_sm;
  P.fct_ctas = static_cast<int>(fct_ctas_of(g, P, di, per_sm));
  if (p->transform == 2) {
    // FCT2: ⌈n/s⌉·fjlt_rows rows of H̃X, then the slow transform on them.
    P.fjlt_rows = p->fjlt_rows > 0
                      ? p->fjlt_rows
                      : static_cast<int>(std::min<double>(p->s, std::max(1.0, ceil(2.0 * d * log(static_cast<double>(d))))));
    P.fjlt_n = P.nblocks * P.fjlt_rows;
  }
  if (p->transform == 1 || p->transform == 2) {
    // The slow Cauchy transform: column slices of sct_width(q) columns, blocks along the rows.
    const int64_t rows = p->transform == 2 ? P.fjlt_n : n;
    P.fct_ws = P.fct_tile_log2 = P.fct_lean = P.fct_sorted = P.fct_cols = P.fct_staged = 0;
    P.fct_width = sct_width(P.q);
    P.fct_slices = (P.q + P.fct_width - 1) / P.fct_width;
    P.fct_ctas = sct_ctas(rows, P.r1, P.q, di.sms);
  }
  // Inputs in host memory arrive in up to kMaxChunks row chunks of at least two waves of
  // tiles each, so that phase 1 on one chunk overlaps the copy of the next.
  P.fct_chunks = 1;
  if (host_staging && p->transform != 2) {       // FCT2's blocks of s rows need one chunk
    const int64_t tiles = (g.ws || g.cols) ? (n + (int64_t{1} << g.tile_log2) - 1) >> g.tile_log2 : P.nblocks;
    P.fct_chunks = static_cast<int>(
        std::max<int64_t>(1, std::min<int64_t>(kMaxChunks, tiles / (2 * static_cast<int64_t>(P.fct_ctas)))));
  }
  // Partial sums sized for the largest variant at full occupancy.
  size_t partial_floats = 0;
  for (int v = 1; v <= 7; ++v)
    if (geo[v].ok)
      partial_floats = std::max<size_t>(
          partial_floats,
          geo[v].cols ? fct_cols_partial_floats(geo[v].cols, static_cast<int>(fct_ctas_of(geo[v], P, di, geo[v].per_sm)),
                                                P.r1, n)
                      : static_cast<size_t>(geo[v].slices) * fct_ctas_of(geo[v], P, di, geo[v].per_sm) * P.r1 *
                            geo[v].width);
  if (p->transform == 1 || p->transform == 2)
    partial_floats = std::max<size_t>(partial_floats, static_cast<size_t>(P.fct_slices) * P.fct_ctas * P.r1 * P.fct_width);

  // Phase 2: a persistent-style grid, 8 blocks per SM by default.
  P.lam_threads = lambda_threads();
  const int lam_per_sm = sch.lam_ctas_per_sm > 0 ? std::min(sch.lam_ctas_per_sm, kMaxLamPerSm) : 8;
  const int64_t lam_rows_ctas = (n + P.lam_threads - 1) / P.lam_threads;
  P.lam_ctas = static_cast<int>(
      std::max<int64_t>(1, std::min<int64_t>(lam_rows_ctas, static_cast<int64_t>(di.sms) * lam_per_sm)));
  const int lam_ctas_max = static_cast<int>(
      std::max<int64_t>(1, std::min<int64_t>(lam_rows_ctas, static_cast<int64_t>(di.sms) * kMaxLamPerSm)));

  // Phase 3: contiguous chunks (multiples of 64 rows), 4 per SM by default.
  P.smp_threads = sample_threads();
  auto chunk_for = [&](int per) {
    const int64_t target = static_cast<int64_t>(di.sms) * per;
    int64_t chunk = (n + target - 1) / target;
    return std::max<int64_t>(64, (chunk + 63) / 64 * 64);
  };
  const int smp_per_sm = sch.smp_chunks_per_sm > 0 ? std::min(sch.smp_chunks_per_sm, kMaxSmpPerSm) : 4;
  P.smp_chunk = chunk_for(smp_per_sm);
  P.smp_ctas = static_cast<int>((n + P.smp_chunk - 1) / P.smp_chunk);
  // The fused λ-and-mark pass (OptimizedFastCauchyRegression) is a λ pass: its chunks
  // follow the λ residency.
  P.lm_chunk = chunk_for(lam_per_sm);
  P.lm_ctas = static_cast<int>((n + P.lm_chunk - 1) / P.lm_chunk);
  const int max_per_sm = std::max(kMaxSmpPerSm, kMaxLamPerSm);
  const int64_t smp_ctas_max = (n + chunk_for(max_per_sm) - 1) / chunk_for(max_per_sm);
  P.irls_ctas = di.sms;

  const int64_t cap = coreset_capacity_of(p);
  const size_t esz = dt == L1S_BF16 ? 2 : 4;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  P.off_status = take(256);
  // IRLS region first, so that l1_solve can use the same offsets with only (d, capacity).
  P.off_irls = take(sizeof(double) * static_cast<size_t>(P.irls_ctas) * (irls_entries(P.q) + 1));
  P.off_x = take(irls_state_bytes());
  P.off_objp = take(solve_scratch_bytes(cap));  // residuals and breakpoints of the solve
  P.off_partials = take(sizeof(float) * partial_floats);
  P.off_pix = take(sizeof(float) * P.r1 * P.q);
  P.off_qr = take(std::max(sizeof(double) * P.r1 * P.q, cond2_scratch_bytes(P.r1, P.q, di.sms)));
  P.off_r = take(sizeof(double) * P.q * P.q);
  P.off_m64 = take(sizeof(double) * P.q * P.r2);
  P.off_m32 = take(sizeof(float) * P.q * P.r2);
  P.off_pi2 = take(sizeof(double) * P.q * P.r2);
  P.off_lam = take(sizeof(float) * static_cast<size_t>(n));
  P.off_lamsum = take(sizeof(double) * std::max(lam_ctas_max, P.irls_ctas));
  P.off_mask = take(sizeof(uint64_t) * static_cast<size_t>((n + 63) / 64));
  P.off_counts = take(sizeof(int64_t) * static_cast<size_t>(smp_ctas_max));
  P.off_idx_tmp = take(static_cast<size_t>(cap) * (sizeof(int64_t) + sizeof(double) + sizeof(double) * P.q) +
                       2 * sizeof(double) * (P.q + 1));
  if (p->variant == 2) P.off_cdf = take(sizeof(double) * static_cast<size_t>(n));   // running sum of λ
  // The column-sliced phase-1 kernel reads every row's draws from a per-launch table
  // (16 bytes a row, whole 1024-row tiles).
  if (p->transform == 2) P.off_fjlt = take(sizeof(float) * static_cast<size_t>(P.fjlt_n) * P.q);   // H̃X: d columns, then G·b
  if (geo[7].ok) P.off_draws = take(16 * static_cast<size_t>((n + fct_cols_tile() - 1) / fct_cols_tile()) * fct_cols_tile());
  if (host_staging) {
    P.off_stage_a = take(esz * static_cast<size_t>(n) * d);
    P.off_stage_b = take(sizeof(float) * static_cast<size_t>(n));
  }
  P.total = off;
  return true;
}



}  // namespace l1s

using namespace l1s;

extern "C" {

const char* l1s_last_error(void) { return g_err; }

const char* l1s_version(void) { return "l1fct 0.1 (sm_103a)"; }

uint64_t l1s_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int l1s_workspace_size(const l1s_params* params, int64_t n, int32_t d, l1s_dtype dtype,
                       int32_t host_staging, size_t* bytes) {
  if (!bytes) return set_error("bytes is NULL"), L1S_ERR_INVALID_ARG;
  Plan pl;
  if (!make_plan(params, n, d, dtype, host_staging != 0, &pl)) return L1S_ERR_INVALID_ARG;
  *bytes = pl.total;
  return L1S_OK;
}

int l1s_status_reset(void* ws, size_t ws_bytes, void* stream) {
  if (!ws || ws_bytes < sizeof(StatusBlock)) return set_error("workspace too small"), L1S_ERR_WORKSPACE;
  if (!cuda_ok(cudaMemsetAsync(ws, 0, sizeof(StatusBlock), static_cast<cudaStream_t>(stream)),
               "status reset"))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

int l1s_status_read(const void* ws, size_t ws_bytes, void* stream, uint32_t* flags) {
  if (!ws || ws_bytes < sizeof(StatusBlock) || !flags) return set_error("bad arguments"), L1S_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!cuda_ok(cudaStreamSynchronize(st), "stream synchronize")) return L1S_ERR_CUDA;
  uint32_t v = 0;
  if (!cuda_ok(cudaMemcpy(&v, ws, sizeof(v), cudaMemcpyDeviceToHost), "status read")) return L1S_ERR_CUDA;
  *flags = v;
  return L1S_OK;
}

int fct_embed(const void* A, int64_t lda, l1s_dtype dtype, const float* b, int64_t n, int32_t d,
              const l1s_params* params, float* PiX, void* ws, size_t ws_bytes, void* stream) {
  TraceRange trace_("fct_embed");
  Plan pl;
  if (!make_plan(params, n, d, dtype, false, &pl)) return L1S_ERR_INVALID_ARG;
  if (!check_a(A, lda, b, d) || !PiX) return L1S_ERR_INVALID_ARG;
  if (!check_ws(pl, ws, ws_bytes)) return L1S_ERR_WORKSPACE;
  if (!launch_fct(pl, A, lda, dtype, b, params, PiX, static_cast<unsigned char*>(ws),
                  static_cast<cudaStream_t>(stream)))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

int l1_condition(const float* PiX, int32_t r1, int32_t q, const l1s_params* params, double* R,
                 double* M, void* ws, size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_condition");
  if (!params || !PiX) return set_error("params and PiX must not be NULL"), L1S_ERR_INVALID_ARG;
  if (r1 != params->r1) return set_error("r1 must equal params->r1"), L1S_ERR_INVALID_ARG;
  Plan pl;
  // Only the status block and the conditioning regions are used.  The plan of one row is
  // the smallest for these (r1, q, r2): a workspace that l1s_workspace_size gave for any
  // n ≥ 1 holds it (a plan of n = r1 rows asked more than one sized for n < r1 rows had).
  if (!make_plan(params, 1, q - 1, L1S_F32, false, &pl)) return L1S_ERR_INVALID_ARG;
  if (!check_ws(pl, ws, ws_bytes)) return L1S_ERR_WORKSPACE;
  if (!launch_condition(pl, PiX, params, R, M, static_cast<unsigned char*>(ws),
                        static_cast<cudaStream_t>(stream)))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

int l1_lambda(const void* A, int64_t lda, l1s_dtype dtype, const float* b, int64_t n, int32_t d,
              const double* M, const l1s_params* params, float* lambda, double* lambda_sum, void* ws,
              size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_lambda");
  Plan pl;
  if (!make_plan(params, n, d, dtype, false, &pl)) return L1S_ERR_INVALID_ARG;
  if (!check_a(A, lda, b, d) || !M || !lambda) return set_error("M and lambda must not be NULL"), L1S_ERR_INVALID_ARG;
  if (!check_ws(pl, ws, ws_bytes)) return L1S_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  float* m32 = reinterpret_cast<float*>(w + pl.off_m32);
  if (!launch_m_to_f32(M, pl.q * pl.r2, m32, st)) return L1S_ERR_CUDA;
  if (!launch_lambda(pl, A, lda, dtype, b, m32, params, lambda, lambda_sum, w, st)) return L1S_ERR_CUDA;
  return L1S_OK;
}


int l1_sample(const void* A, int64_t lda, l1s_dtype dtype, const float* b, int64_t n, int32_t d,
              const double* M, const l1s_params* params, int64_t capacity, int64_t* idx, double* wts,
              double* coreset, int64_t* count, float* lambda, void* ws, size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_sample");
  Plan pl;
  if (!make_plan(params, n, d, dtype, false, &pl)) return L1S_ERR_INVALID_ARG;
  if (!check_a(A, lda, b, d) || !M) return set_error("M must not be NULL"), L1S_ERR_INVALID_ARG;
  if (capacity < 0 || (capacity > 0 && (!idx || !wts)) || !count)
    return set_error("idx, w (capacity > 0) and count must not be NULL"), L1S_ERR_INVALID_ARG;
  if (!check_ws(pl, ws, ws_bytes)) return L1S_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  float* m32 = reinterpret_cast<float*>(w + pl.off_m32);
  if (!launch_m_to_f32(M, pl.q * pl.r2, m32, st)) return L1S_ERR_CUDA;
  return sample_impl(pl, A, lda, dtype, b, m32, params, capacity, idx, wts, coreset, count, lambda, w, st);
}

int l1s_sample_lambda_workspace_size(const l1s_params* params, int64_t n, int32_t d, l1s_dtype dtype, int32_t k,
                                     size_t* bytes) {
  Plan pl;
  if (!bytes) return set_error("bytes must not be NULL"), L1S_ERR_INVALID_ARG;
  if (k < 1 || k > kMaxCoresets) return set_error("k must be in [1, %d]", kMaxCoresets), L1S_ERR_INVALID_ARG;
  if (!make_plan(params, n, d, dtype, false, &pl)) return L1S_ERR_INVALID_ARG;
  *bytes = pl.total + sample_many_extra_bytes(pl, k);
  return L1S_OK;
}

int l1_sample_lambda(const void* A, int64_t lda, l1s_dtype dtype, const float* b, int64_t n, int32_t d,
                     const float* lambda, const double* lambda_total, const l1s_params* params, int32_t k,
                     int64_t capacity, int64_t* idx, double* wts, double* coreset, int64_t* count, void* ws,
                     size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_sample_lambda");
  Plan pl;
  if (!make_plan(params, n, d, dtype, false, &pl)) return L1S_ERR_INVALID_ARG;
  if (k < 1 || k > kMaxCoresets) return set_error("k must be in [1, %d]", kMaxCoresets), L1S_ERR_INVALID_ARG;
  if (params->variant == 2)
    return set_error("l1_sample_lambda samples without replacement (params.variant 0 or 1)"), L1S_ERR_INVALID_ARG;
  if (coreset && !check_a(A, lda, b, d)) return L1S_ERR_INVALID_ARG;
  if (!lambda || (params->variant == 0 && !lambda_total))
    return set_error("lambda (and lambda_total for variant 0) must not be NULL"), L1S_ERR_INVALID_ARG;
  if (capacity < 0 || (capacity > 0 && (!idx || !wts)) || !count)
    return set_error("idx, w (capacity > 0) and count must not be NULL"), L1S_ERR_INVALID_ARG;
  const size_t need = pl.total + sample_many_extra_bytes(pl, k);
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 || ws_bytes < need)
    return set_error("workspace too small for l1_sample_lambda: %zu needed", need), L1S_ERR_WORKSPACE;
  if (!launch_sample_many(pl, lambda, lambda_total, params, k, A, lda, dtype, b, capacity, idx, wts, coreset, count,
                          static_cast<unsigned char*>(ws), static_cast<cudaStream_t>(stream)))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

int l1_sample_from_p(const double* p, int64_t n, const l1s_params* params, int64_t capacity, int64_t* idx,
                     int64_t* count, void* ws, size_t ws_bytes, void* stream) {
  Plan pl;
  if (!make_plan(params, n, 1, L1S_F32, false, &pl)) return L1S_ERR_INVALID_ARG;
  if (!p || !count || capacity < 0 || (capacity > 0 && !idx))
    return set_error("p, count (and idx when capacity > 0) must not be NULL"), L1S_ERR_INVALID_ARG;
  if (!check_ws(pl, ws, ws_bytes)) return L1S_ERR_WORKSPACE;
  unsigned char* w = static_cast<unsigned char*>(ws);
  if (!launch_sample(pl, nullptr, p, params, nullptr, 0, L1S_F32, nullptr, capacity, idx, nullptr, nullptr,
                     count, w, static_cast<cudaStream_t>(stream)))
    return L1S_ERR_CUDA;
  return L1S_OK;
}


int l1_coreset(const void* A, int64_t lda, l1s_dtype dtype, const float* b, int64_t n, int32_t d,
               const l1s_params* params, int64_t capacity, int64_t* idx, double* wts, double* coreset,
               int64_t* count, void* ws, size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_coreset");
  Plan pl;
  if (!make_plan(params, n, d, dtype, false, &pl)) return L1S_ERR_INVALID_ARG;
  if (!check_a(A, lda, b, d)) return L1S_ERR_INVALID_ARG;
  if (capacity < 0 || (capacity > 0 && (!idx || !wts)) || !count)
    return set_error("idx, w (capacity > 0) and count must not be NULL"), L1S_ERR_INVALID_ARG;
  if (!check_ws(pl, ws, ws_bytes)) return L1S_ERR_WORKSPACE;
  return coreset_impl(pl, A, lda, dtype, b, params, capacity, idx, wts, coreset, count,
                      static_cast<unsigned char*>(ws), static_cast<cudaStream_t>(stream));
}


// Copy stream and events (per device) for inputs that arrive from host memory.  A call
// holds the pool's mutex while it enqueues.
struct CopyPool {
  bool ready = false;
  cudaStream_t cp;
  cudaEvent_t start;
  cudaEvent_t chunk[kMaxChunks];
  std::mutex mu;
};
static CopyPool g_copy_pools[64];
static std::mutex g_copy_pools_mu;

static CopyPool* copy_pool() {
  int dev = 0;
  if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice") || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_copy_pools_mu);
  CopyPool& P = g_copy_pools[dev];
  if (!P.ready) {
    if (!cuda_ok(cudaStreamCreateWithFlags(&P.cp, cudaStreamNonBlocking), "create copy stream") ||
        !cuda_ok(cudaEventCreateWithFlags(&P.start, cudaEventDisableTiming), "create copy event"))
      return nullptr;
    for (int k = 0; k < kMaxChunks; ++k)
      if (!cuda_ok(cudaEventCreateWithFlags(&P.chunk[k], cudaEventDisableTiming), "create copy event"))
        return nullptr;
    P.ready = true;
  }
  return &P;
}

// The coreset of inputs in host memory: the rows are copied into the workspace's staging
// region chunk by chunk, overlapping phase 1, and phases 2 and 3 read the staged rows.
static int coreset_impl_host(const Plan& pl, const void* A_host, int64_t lda, l1s_dtype dtype,
                             const float* b_host, const l1s_params* params, int64_t capacity, int64_t* idx,
                             double* wts, double* coreset, int64_t* count, unsigned char* w, cudaStream_t st) {
  CopyPool* cpool = copy_pool();
  if (!cpool) return L1S_ERR_CUDA;
  void* A_dev = w + pl.off_stage_a;
  float* b_dev = reinterpret_cast<float*>(w + pl.off_stage_b);
  {
    std::lock_guard<std::mutex> lock(cpool->mu);
    if (!cuda_ok(cudaMemsetAsync(w + pl.off_status, 0, sizeof(StatusBlock), st), "status reset") ||
        !cuda_ok(cudaEventRecord(cpool->start, st), "record copy start") ||
        !cuda_ok(cudaStreamWaitEvent(cpool->cp, cpool->start, 0), "copy stream wait"))
      return L1S_ERR_CUDA;
    if (!launch_fct_streamed(pl, A_host, lda, dtype, b_host, A_dev, b_dev, params,
                             reinterpret_cast<float*>(w + pl.off_pix), w, st, cpool->cp, cpool->chunk,
                             reinterpret_cast<double*>(w + pl.off_pi2)))
      return L1S_ERR_CUDA;
  }
  if (!launch_condition(pl, reinterpret_cast<float*>(w + pl.off_pix), params, nullptr, nullptr, w, st, true))
    return L1S_ERR_CUDA;
  return sample_impl(pl, A_dev, pl.d, dtype, b_dev, reinterpret_cast<float*>(w + pl.off_m32), params, capacity,
                     idx, wts, coreset, count, nullptr, w, st);
}

int l1_coreset_host(const void* A_host, int64_t lda, l1s_dtype dtype, const float* b_host, int64_t n,
                    int32_t d, const l1s_params* params, int64_t capacity, int64_t* idx_host, double* w_host,
                    int64_t* count_host, void* ws, size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_coreset_host");
  Plan pl;
  if (!make_plan(params, n, d, dtype, true, &pl)) return L1S_ERR_INVALID_ARG;
  if (!check_a(A_host, lda, b_host, d) || !count_host || capacity < 0 ||
      (capacity > 0 && (!idx_host || !w_host)))
    return set_error("bad host buffers"), L1S_ERR_INVALID_ARG;
  if (!check_ws(pl, ws, ws_bytes)) return L1S_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  const int64_t cap_ws = coreset_capacity_of(params);
  const int64_t cap = std::min(capacity, cap_ws);
  int64_t* idx_dev = reinterpret_cast<int64_t*>(w + pl.off_idx_tmp);
  double* w_dev = reinterpret_cast<double*>(idx_dev + cap_ws);
  StatusBlock* sb = reinterpret_cast<StatusBlock*>(w + pl.off_status);
  int rc = coreset_impl_host(pl, A_host, lda, dtype, b_host, params, cap, idx_dev, w_dev, nullptr, &sb->count, w,
                             st);
  if (rc != L1S_OK) return rc;
  int64_t cnt = 0;
  if (!cuda_ok(cudaMemcpyAsync(&cnt, &sb->count, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "copy count") ||
      !cuda_ok(cudaMemcpyAsync(idx_host, idx_dev, sizeof(int64_t) * cap, cudaMemcpyDeviceToHost, st),
               "copy idx") ||
      !cuda_ok(cudaMemcpyAsync(w_host, w_dev, sizeof(double) * cap, cudaMemcpyDeviceToHost, st), "copy w"))
    return L1S_ERR_CUDA;
  uint32_t flags = 0;
  if (l1s_status_read(ws, ws_bytes, stream, &flags) != L1S_OK) return L1S_ERR_CUDA;
  *count_host = cnt;
  if (cnt > capacity) flags |= L1S_FLAG(L1S_ERR_CAPACITY);
  return first_error(flags);
}

int l1_solve(const double* coreset, const double* wts, const int64_t* count, int64_t capacity, int32_t d,
             int32_t max_iter, double* x, double* objective, void* ws, size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_solve");
  if (!coreset || !wts || !count || !x || !objective) return set_error("NULL argument"), L1S_ERR_INVALID_ARG;
  if (d < 1 || d > kMaxD || capacity < 1 || max_iter < 0 || max_iter > 100000)
    return set_error("bad d, capacity or max_iter"), L1S_ERR_INVALID_ARG;
  const DeviceInfo di = device_info();
  if (di.device < 0) return set_error("no CUDA device"), L1S_ERR_CUDA;
  // Same leading layout as make_plan: status, IRLS partials, IRLS state, residual scratch.
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const int q = d + 1;
  const size_t o_status = take(256);
  const size_t o_part = take(sizeof(double) * static_cast<size_t>(di.sms) * (irls_entries(q) + 1));
  const size_t o_state = take(irls_state_bytes());
  const size_t o_scr = take(solve_scratch_bytes(capacity));
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 || ws_bytes < off)
    return set_error("workspace too small for l1_solve: %zu needed", off), L1S_ERR_WORKSPACE;
  unsigned char* w = static_cast<unsigned char*>(ws);
  if (!launch_solve(coreset, wts, count, capacity, d, max_iter, x, objective, di.sms,
                    reinterpret_cast<double*>(w + o_part), w + o_state, reinterpret_cast<float*>(w + o_scr),
                    reinterpret_cast<StatusBlock*>(w + o_status), static_cast<cudaStream_t>(stream), 1, nullptr))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

// Workspace layout of l1_solve_many: k status blocks, then per coreset the IRLS partials,
// state and residual scratch.
struct SolveManyLayout {
  int nblocks;
  size_t o_status, o_part, o_state, o_scr, total;
};

static SolveManyLayout solve_many_layout(int64_t capacity, int d, int k, int sms) {
  SolveManyLayout L;
  // About four accumulation blocks per SM over all k coresets, at most one per SM each.
  L.nblocks = std::max(1, std::min(sms, (4 * sms + k - 1) / k));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const int q = d + 1;
  L.o_status = take(std::max<size_t>(256, sizeof(StatusBlock) * static_cast<size_t>(k)));
  L.o_part = take(sizeof(double) * static_cast<size_t>(L.nblocks) * (irls_entries(q) + 1) * k);
  L.o_state = take(irls_state_bytes() * static_cast<size_t>(k));
  L.o_scr = take(solve_scratch_bytes(capacity) * static_cast<size_t>(k));
  L.total = off;
  return L;
}

int l1s_solve_many_workspace_size(int64_t capacity, int32_t d, int32_t k, size_t* bytes) {
  if (!bytes || d < 1 || d > kMaxD || capacity < 1 || k < 1 || k > kMaxCoresets)
    return set_error("bad capacity, d or k"), L1S_ERR_INVALID_ARG;
  const DeviceInfo di = device_info();
  if (di.device < 0) return set_error("no CUDA device"), L1S_ERR_CUDA;
  *bytes = solve_many_layout(capacity, d, k, di.sms).total;
  return L1S_OK;
}

int l1_solve_many(const double* coreset, const double* wts, const int64_t* count, int64_t capacity, int32_t d,
                  int32_t k, int32_t max_iter, double* x, double* objective, uint32_t* flags, void* ws,
                  size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_solve_many");
  if (!coreset || !wts || !count || !x || !objective) return set_error("NULL argument"), L1S_ERR_INVALID_ARG;
  if (d < 1 || d > kMaxD || capacity < 1 || max_iter < 0 || max_iter > 100000 || k < 1 || k > kMaxCoresets)
    return set_error("bad d, capacity, k or max_iter"), L1S_ERR_INVALID_ARG;
  const DeviceInfo di = device_info();
  if (di.device < 0) return set_error("no CUDA device"), L1S_ERR_CUDA;
  const SolveManyLayout L = solve_many_layout(capacity, d, k, di.sms);
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 || ws_bytes < L.total)
    return set_error("workspace too small for l1_solve_many: %zu needed", L.total), L1S_ERR_WORKSPACE;
  unsigned char* w = static_cast<unsigned char*>(ws);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!cuda_ok(cudaMemsetAsync(w + L.o_status, 0, sizeof(StatusBlock) * static_cast<size_t>(k), st),
               "status reset"))
    return L1S_ERR_CUDA;
  if (!launch_solve(coreset, wts, count, capacity, d, max_iter, x, objective, L.nblocks,
                    reinterpret_cast<double*>(w + L.o_part), w + L.o_state, reinterpret_cast<float*>(w + L.o_scr),
                    reinterpret_cast<StatusBlock*>(w + L.o_status), st, k, flags))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

int l1_objective(const void* A, int64_t lda, l1s_dtype dtype, const float* b, int64_t n, int32_t d,
                 const double* x, double* objective, void* ws, size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_objective");
  if (!check_a(A, lda, b, d) || !x || !objective || n < 1 || d < 1 || d > kMaxD)
    return set_error("bad arguments"), L1S_ERR_INVALID_ARG;
  const DeviceInfo di = device_info();
  if (di.device < 0) return set_error("no CUDA device"), L1S_ERR_CUDA;
  const int nb = di.sms * 4;
  if (!ws || ws_bytes < 256 + sizeof(double) * nb) return set_error("workspace too small"), L1S_ERR_WORKSPACE;
  double* partials = reinterpret_cast<double*>(static_cast<unsigned char*>(ws) + 256);
  if (!launch_objective(A, lda, dtype, b, n, d, x, objective, nb, partials, static_cast<cudaStream_t>(stream)))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

int l1_regress(const void* A, int64_t lda, l1s_dtype dtype, const float* b, int64_t n, int32_t d,
               const l1s_params* params, int32_t inputs_on_host, double* x_host, double* objective_host,
               int64_t* coreset_rows_host, void* ws, size_t ws_bytes, void* stream) {
  TraceRange trace_("l1_regress");
  Plan pl;
  if (!make_plan(params, n, d, dtype, inputs_on_host != 0, &pl)) return L1S_ERR_INVALID_ARG;
  if (!check_a(A, lda, b, d) || !x_host || !objective_host) return set_error("NULL argument"), L1S_ERR_INVALID_ARG;
  if (!check_ws(pl, ws, ws_bytes)) return L1S_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  const void* Ad = A;
  const float* bd = b;
  int64_t ld = lda;
  if (inputs_on_host) {
    Ad = w + pl.off_stage_a;
    bd = reinterpret_cast<const float*>(w + pl.off_stage_b);
    ld = d;
  }
  const int64_t cap = coreset_capacity_of(params);
  const int q = d + 1;
  int64_t* idx = reinterpret_cast<int64_t*>(w + pl.off_idx_tmp);
  double* wts = reinterpret_cast<double*>(idx + cap);
  double* core = wts + cap;
  double* xd = core + cap * q;
  double* objd = xd + q + 1;
  StatusBlock* sb = reinterpret_cast<StatusBlock*>(w + pl.off_status);
  int rc = inputs_on_host ? coreset_impl_host(pl, A, lda, dtype, b, params, cap, idx, wts, core, &sb->count, w, st)
                          : coreset_impl(pl, Ad, ld, dtype, bd, params, cap, idx, wts, core, &sb->count, w, st);
  if (rc != L1S_OK) return rc;
  rc = l1_solve(core, wts, &sb->count, cap, d, 100, xd, objd, ws, ws_bytes, stream);
  if (rc != L1S_OK) return rc;
  if (!launch_objective(Ad, ld, dtype, bd, n, d, xd, objd + 1, pl.lam_ctas,
                        reinterpret_cast<double*>(w + pl.off_lamsum), st))
    return L1S_ERR_CUDA;
  double res[2];
  int64_t cnt = 0;
  if (!cuda_ok(cudaMemcpyAsync(x_host, xd, sizeof(double) * d, cudaMemcpyDeviceToHost, st), "copy x") ||
      !cuda_ok(cudaMemcpyAsync(res, objd, sizeof(res), cudaMemcpyDeviceToHost, st), "copy objective") ||
      !cuda_ok(cudaMemcpyAsync(&cnt, &sb->count, sizeof(cnt), cudaMemcpyDeviceToHost, st), "copy count"))
    return L1S_ERR_CUDA;
  uint32_t flags = 0;
  if (l1s_status_read(ws, ws_bytes, stream, &flags) != L1S_OK) return L1S_ERR_CUDA;
  *objective_host = res[1];
  if (coreset_rows_host) *coreset_rows_host = cnt;
  return first_error(flags);
}

int l1s_debug_wait_timeout(void* ws, size_t ws_bytes, int64_t max_cycles, void* stream) {
  if (!ws || ws_bytes < sizeof(StatusBlock)) return set_error("workspace too small"), L1S_ERR_WORKSPACE;
  if (max_cycles < 1000 || max_cycles > kWaitCycles) return set_error("max_cycles out of range"), L1S_ERR_INVALID_ARG;
  if (!launch_debug_wait(&static_cast<StatusBlock*>(ws)->flags, max_cycles, static_cast<cudaStream_t>(stream)))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

int l1s_debug_variates(const l1s_params* params, int64_t row_start, int64_t count, int32_t* bucket_h,
                       int32_t* bucket_i, int32_t* k_h, int32_t* k_i, float* cauchy_h, float* cauchy_i,
                       int8_t* sign, uint64_t* u_bits, void* stream) {
  if (!params || row_start < 0 || count < 0) return set_error("bad arguments"), L1S_ERR_INVALID_ARG;
  if (params->r1 < 1 || params->r1 > 65535) return set_error("bad r1"), L1S_ERR_INVALID_ARG;
  if (count == 0) return L1S_OK;
  if (!launch_debug_variates(params, row_start, count, bucket_h, bucket_i, k_h, k_i, cauchy_h, cauchy_i, sign,
                             u_bits, static_cast<cudaStream_t>(stream)))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

int l1s_debug_pi2(const l1s_params* params, int32_t q, double* pi2, void* stream) {
  if (!params || !pi2 || q < 1 || params->r2 < 1 || params->r2 > kMaxR2)
    return set_error("bad arguments"), L1S_ERR_INVALID_ARG;
  if (!launch_pi2(params, q, pi2, static_cast<cudaStream_t>(stream))) return L1S_ERR_CUDA;
  return L1S_OK;
}

}  // extern "C"
