/*
 * l1fct — Fast Cauchy Transform ℓ1 regression on NVIDIA GB300 (sm_103a).
 *
 * C ABI of the library libl1fct.so.  The method is FastCauchyRegression
 * (Clarkson, Drineas, Magdon-Ismail, Mahoney, Meng, Woodruff, "The Fast
 * Cauchy Transform and Faster Robust Linear Regression", Figure 2) for the
 * problem statement min_x ‖A·x − b‖₁ (§4.2, eq. (original_prob)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - A is n × d, row-major with leading dimension lda ≥ d (elements), stored
 *   FP32 or BF16 (l1s_dtype); b is n FP32 values.  X = [A, −b] (n × q,
 *   q = d + 1) is never materialised; −b is applied on load.
 * - Pointers named *_dev are device pointers; *_host are host pointers.  All
 *   arrays are owned by the caller.  The library allocates no memory: every
 *   call that needs scratch takes a caller-allocated device workspace
 *   (`ws`, `ws_bytes`), sized by l1s_workspace_size and aligned to 256 bytes.
 *   One workspace must not be used by two calls that overlap on the GPU.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Unless stated otherwise a call only enqueues work on `stream` and returns.
 * - Return value: L1S_OK when the arguments were valid and the work was
 *   enqueued; otherwise an error code and nothing was enqueued.  Conditions
 *   that only the GPU can see (rank deficiency, non-finite input, zero mass,
 *   capacity overflow) are OR-ed into a status word inside the workspace and
 *   read back with l1s_status_read.  l1s_last_error() returns the text of the
 *   calling thread's last host-side error.
 * - Random draws come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *   params.seed, with counters built from the global row id, params.problem_id
 *   and a stream number (0: signs/buckets/Cauchy scales of Π1, 1: Π2,
 *   2: sampling uniforms, 3: draws with replacement, 4: the slow transform's C,
 *   5: FCT2's block G).  Row ids are global: row r of A has id
 *   params.global_row_offset + r, so shards of one problem reproduce the
 *   unsharded draws.
 * - Not thread-safe per workspace; distinct workspaces may be used from
 *   distinct threads (the kernels' dynamic shared-memory limits only ever rise,
 *   under a lock, so calls of different shapes do not undo each other's).
 *   l1_lambda, l1_sample, l1_coreset, l1_coreset_host and
 *   l1_regress load M into a per-device constant bank: calls of these on
 *   different streams of one device must not overlap (l1_regress_batched
 *   keeps M in shared memory and has no such limit).
 */
#ifndef L1FCT_H
#define L1FCT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define L1S_API __attribute__((visibility("default")))
#else
#define L1S_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  L1S_OK = 0,
  L1S_ERR_INVALID_ARG = 1,   /* an argument violates the documented constraints */
  L1S_ERR_WORKSPACE = 2,     /* workspace missing, misaligned or too small */
  L1S_ERR_CUDA = 3,          /* a CUDA runtime call failed (see l1s_last_error) */
  L1S_ERR_RANK_DEFICIENT = 4,/* status bit: |R_kk| <= 1e-5·‖(Π1X)_{:,k}‖₂ for some k, or R non-finite */
  L1S_ERR_NONFINITE = 5,     /* status bit: NaN/Inf met in A, b or Π1X */
  L1S_ERR_ZERO_MASS = 6,     /* status bit: Σλ is zero or not finite */
  L1S_ERR_CAPACITY = 7,      /* status bit: coreset larger than the caller's capacity */
  L1S_ERR_NOT_CONVERGED = 8, /* status bit: IRLS stopped at its iteration cap */
  L1S_ERR_TIMEOUT = 9        /* status bit: a bounded wait inside a kernel gave up */
} l1s_status;

/* Bits of the device status word (bit = 1 << (code − 1)). */
#define L1S_FLAG(code) (1u << ((code) - 1))

typedef enum { L1S_F32 = 0, L1S_BF16 = 1 } l1s_dtype;

typedef struct {
  uint64_t seed;              /* key of every Philox draw */
  uint32_t problem_id;        /* counter word 2: independent draws per problem */
  int32_t s;                  /* Hadamard block size of FCT1, power of two, 1..4096 (§3.1) */
  int32_t r1;                 /* rows of Π1·X, q ≤ r1 ≤ 65535 (§3.1, r1 = O(d log d)) */
  int32_t r2;                 /* columns of Π2, 1..64 (Figure 2, step 3) */
  double coreset_size;        /* m_s > 0: expected coreset size bound (Figure 2, step 6) */
  int64_t global_row_offset;  /* global id of A's first row; a multiple of s */
  int32_t sign_flip;          /* 1: Π1·D·X with random ±1 diagonal D; 0: Π1·X as in §3.1 */
  int32_t variant;            /* 0: FastCauchyRegression (Figure 2): Π2 Cauchy, p̂ = min(1, m_s·λ/Σλ).
                                 1: OptimizedFastCauchyRegression (Figure "mainOpt"): Π2 Gaussian
                                 (Box–Muller on stream 1), p̂ = min(1, sample_scale·λ̂), no Σλ;
                                 coreset_size then only bounds the expected coreset size
                                 (it sizes the workspace's coreset buffers).
                                 2: FastCauchyRegression drawing exactly coreset_size rows
                                 (an integer) independently with replacement, p̂_i = λ_i/Σλ,
                                 weight 1/(coreset_size·p̂_i) (caption of Figure 2); the
                                 kept rows are listed in draw order, with repeats. */
  double sample_scale;        /* variant 1: the sampling size s of p̂ = min{1, s·λ̂}; variants 0, 2: 0 */
  int32_t transform;          /* Π1 of phase 1: 0 FCT1 (§3.1); 1 the slow Cauchy transform
                                 (4/r1)·C with C an r1 × n matrix of i.i.d. standard Cauchys
                                 (§3, the theorem of Sohler and Woodruff; the conditioning of
                                 §6.3), entry (r, i), r = 4g + w, from word w of the Philox call
                                 with counter (i_lo, (i_hi mod 2^16) + g·2^16, problem_id, 4);
                                 s and sign_flip are then unused.  2: FCT2 (§3.2),
                                 (8/r1)·√(πt/(2·fjlt_rows))·C·H̃ with t = s (a power of two) and
                                 H̃ block diagonal, one fjlt_rows × t block
                                 G = √(t/fjlt_rows)·S·H_t·D per t rows (a subsampled randomized
                                 Hadamard transform: D_i = −1 when bit 0 of word 0 of Philox call
                                 (i, 0, problem_id, 5) is set, G's row r the Hadamard row
                                 ⌊word1·t/2^32⌋ of call r), then the slow transform above on the
                                 rows of H̃X (row k of H̃X has Cauchy row id k, counted from
                                 (global_row_offset/t)·fjlt_rows); sign_flip is unused */
  int32_t fjlt_rows;          /* transform 2: rows of G kept per t-row block (1 ≤ fjlt_rows ≤ s);
                                 0 takes ⌈2·d·ln d⌉ (at least 1, at most s); otherwise unused */
} l1s_params;

/* Text of the calling thread's last host-side error ("" if none). */
L1S_API const char* l1s_last_error(void);

/* Library version string. */
L1S_API const char* l1s_version(void);

/* Number of kernels this process has launched through the library so far.  A
 * CUDA graph counts its kernels once, when they are captured; its replays
 * re-run them without counting. */
L1S_API uint64_t l1s_kernel_launches(void);

/* Bytes of device workspace that every entry point below needs for a problem
 * of n rows and d columns with these params on the current device.  With
 * host_staging = 1 the size also covers the device copies of A and b used by
 * l1_coreset_host and l1_regress with host inputs. */
L1S_API int l1s_workspace_size(const l1s_params* params, int64_t n, int32_t d, l1s_dtype dtype,
                       int32_t host_staging, size_t* bytes);

/* Clear the workspace status word (enqueued on stream). */
L1S_API int l1s_status_reset(void* ws, size_t ws_bytes, void* stream);

/* Synchronise `stream` and read the workspace status word: *flags is an OR of
 * L1S_FLAG(code) bits (0 = no device-side error since the last reset). */
L1S_API int l1s_status_read(const void* ws, size_t ws_bytes, void* stream, uint32_t* flags);

/* Phase 1 — the FCT1 embedding (§3.1; Figure 2, steps 1-2), or with
 * params.transform = 1 the slow Cauchy transform Π1·X = (4/r1)·C·X (§3), whose
 * r1·n variates are drawn inside the kernel (its cost is the drawing, not the bytes),
 * or with params.transform = 2 FCT2 (§3.2): a subsampled randomized Hadamard block per
 * s rows (fjlt_rows of them kept, H̃X kept in the workspace) followed by the slow
 * transform on the rows of H̃X, scaled by (8/r1)·√(πs/(2·fjlt_rows)).  FCT1:
 *   PiX_dev = Π1·X = 4·B·C·H̃·D·[A, −b]          (r1 × q, FP32, row-major)
 * H̃ is block diagonal with blocks [H_s; I_s] (H_s the Sylvester Hadamard
 * matrix scaled by 1/√s), C a diagonal of standard Cauchys, B a hash of each
 * of the 2n virtual rows into r1 buckets, D a ±1 diagonal (params.sign_flip).
 * n need not be a multiple of s: X is padded with zero rows to the next
 * multiple of s, and the padded rows' Hadamard virtual rows take the draws of
 * their row ids.  The r1 × q sums are formed per thread block in shared
 * memory and combined in a fixed order; float rounding still depends on the
 * order of shared-memory additions, so repeated calls may differ in the last
 * bits.  Requires n ≥ 1, 1 ≤ d ≤ 128, lda ≥ d. */
L1S_API int fct_embed(const void* A_dev, int64_t lda, l1s_dtype dtype, const float* b_dev,
              int64_t n, int32_t d, const l1s_params* params, float* PiX_dev,
              void* ws, size_t ws_bytes, void* stream);

/* Conditioning (Figure 2, steps 2-3; Figure 1): FP64 QR of Π1·X (r1 × q,
 * FP32 row-major input) with positive diag(R), then M = R⁻¹·Π2 where Π2 is
 * q × r2 of standard Cauchys.  Outputs (device, FP64, row-major, may be NULL):
 * R_dev (q × q, upper triangular) and M_dev (q × r2).  Rank deficiency sets
 * the RANK_DEFICIENT status bit: column k counts as dependent on the columns
 * before it when |R_kk| ≤ 1e-5·‖(Π1X)_{:,k}‖₂, the resolution of an FP32 Π1X.
 * Any workspace that l1s_workspace_size gives for these params, d = q − 1 and some
 * n ≥ 1 serves. */
L1S_API int l1_condition(const float* PiX_dev, int32_t r1, int32_t q, const l1s_params* params,
                 double* R_dev, double* M_dev, void* ws, size_t ws_bytes, void* stream);

/* Phase 2 (Figure 2, steps 4-5): λ_i = lower median_j |(X·M)_ij| with M the
 * q × r2 FP64 matrix (rounded to FP32 for the product; FP32 accumulation;
 * BF16 A is widened to FP32 exactly).  Mixed-precision form: for BF16 A with
 * 16 < d ≤ 64, r2 ∈ {16, 32}, a 16-byte aligned A and lda·2 a multiple of 16,
 * A·M_A runs on the tensor cores with M_A (the first d rows of M, rounded to
 * FP32 then to BF16, nearest-even) and FP32 accumulation; the b column's term
 * −b_i·M_{d,j} is added in FP32.  The lower median
 * is the ((r2−1)/2)-th order statistic counting from 0.  Writes lambda_dev
 * (n floats) and *lambda_sum_dev (FP64 sum of the written λ, fixed order). */
L1S_API int l1_lambda(const void* A_dev, int64_t lda, l1s_dtype dtype, const float* b_dev,
              int64_t n, int32_t d, const double* M_dev, const l1s_params* params,
              float* lambda_dev, double* lambda_sum_dev, void* ws, size_t ws_bytes,
              void* stream);

/* l1_lambda without a workspace, for callers that cannot allocate device
 * memory (the paper has no counterpart: this is a property of the library).
 * cudaMalloc may synchronise the whole device, which a latency-bound loop cannot
 * afford once it runs, and some host programs give all device memory to their own
 * pool at start-up and let plug-in code allocate none.  Arguments and results are
 * those of l1_lambda minus ws/ws_bytes.  Scratch (M in FP32, the per-block Σλ
 * partials, a status block) lives in one library-owned 40 KiB device array per GPU,
 * held until the process exits; 4·q·r2 bytes, 8 bytes per Σλ partial (one per block
 * of the λ grid: 8 per SM by default, more when a schedule installed with
 * l1s_schedule_set asks for more) and 4 KiB for the BF16 copy of M must fit in it,
 * else L1S_ERR_INVALID_ARG.  Under the default grid every d ≤ 64 with r2 ≤ 64 fits;
 * whether a shape fits therefore depends on the installed λ grid.  The first
 * call on a device looks up that array's address (cudaGetSymbolAddress); make it
 * before any stream capture.  Every call shares the array and clears what must
 * start at zero; calls that overlap on the GPU race on it.  The FP32 form also loads
 * M into the per-device constant bank that l1_lambda, l1_sample, l1_coreset and
 * l1_regress use, so a no-alloc call that overlaps any of those on the same device
 * races with it too.  Allocates nothing: no cudaMalloc, cudaFree or allocating
 * library call. */
L1S_API int l1_lambda_noalloc(const void* A_dev, int64_t lda, l1s_dtype dtype, const float* b_dev,
                              int64_t n, int32_t d, const double* M_dev, const l1s_params* params,
                              float* lambda_dev, double* lambda_sum_dev, void* stream);

/* The ℓ1 well-conditioned basis U = X·R⁻¹ of §4.1 (Figure 1) with R the q × q upper
 * triangular factor from l1_condition (device, FP64, row-major), and its exact ℓ1 row
 * norms ‖U_(i)‖₁, the ℓ1 leverage scores that λ estimates (Figure 2, step 5); FP64, one
 * forward substitution per row (R⁻¹ is not formed).  Outputs (device, may be NULL):
 * U_dev (n × q FP64, row-major), rownorm_dev (n FP64) and *total_dev = Σ_i ‖U_(i)‖₁ = ‖U‖₁
 * (the α of an (α, β)-conditioned basis, §6.1), summed in a fixed order.  The workspace
 * needs 256 + 8·1024 bytes (256-byte aligned).  Asynchronous on `stream`. */
L1S_API int l1_basis(const void* A_dev, int64_t lda, l1s_dtype dtype, const float* b_dev, int64_t n,
                     int32_t d, const double* R_dev, double* U_dev, double* rownorm_dev,
                     double* total_dev, void* ws, size_t ws_bytes, void* stream);

/* Phases 2-3 (Figure 2, steps 4-7): λ as in l1_lambda, Σλ, τ = m_s/Σλ in FP64,
 * p̂_i = min(1, τ·λ_i) in FP64, row i kept iff u_i < p̂_i with its 53-bit
 * uniform u_i (exact FP64 comparison).  Kept rows are written in ascending
 * order: idx_dev (row index into A, int64), w_dev (1/p̂_i, FP64) and
 * coreset_dev (the row of X = [A_i, −b_i] in FP64, row-major, q per row), up to
 * `capacity` rows; *count_dev receives the number kept (which may exceed
 * capacity: the CAPACITY status bit is then set).  lambda_dev (n floats) and
 * coreset_dev may be NULL. */
L1S_API int l1_sample(const void* A_dev, int64_t lda, l1s_dtype dtype, const float* b_dev,
              int64_t n, int32_t d, const double* M_dev, const l1s_params* params,
              int64_t capacity, int64_t* idx_dev, double* w_dev, double* coreset_dev,
              int64_t* count_dev, float* lambda_dev, void* ws, size_t ws_bytes, void* stream);

/* Figure 2, steps 6-7 from a caller-given λ (lambda_dev, n floats, e.g. from l1_lambda)
 * and a caller-given Σλ (*lambda_total_dev, FP64 on the device), k times over:
 * τ = m_s/Σλ, p̂_i = min(1, τ·λ_i) in FP64, and coreset j (0 ≤ j < k) keeps row i iff
 * u_i < p̂_i with the sampling uniforms of problem id params.problem_id + j (the same
 * exact FP64 decision as l1_sample).  Σλ being an input, row shards of one problem
 * (each with its global_row_offset) sample with the sum of the shards' Σλ and together
 * keep exactly the rows the unsharded call keeps; with Σλ from l1_lambda and k = 1 the
 * result is l1_sample's.  k coresets cost one read of λ and k Philox calls per two rows
 * (the k approximate solutions of one pass over the data, §6.3).  params.variant 1
 * (OptimizedFastCauchyRegression) uses p̂ = min(1, sample_scale·λ_i) and ignores
 * lambda_total_dev (may then be NULL); variant 2 (with replacement) is refused.
 * Outputs of coreset j, rows in ascending order: idx_dev[j·capacity + t], w_dev[j·capacity
 * + t] (1/p̂), coreset_dev[(j·capacity + t)·q + c] (FP64 [A_i, −b_i]; may be NULL, and
 * then A_dev and b_dev are not read) for t < min(count, capacity), and count_dev[j]
 * (the number kept; above capacity the CAPACITY status bit is set).  1 ≤ k ≤ 1024.
 * The workspace is sized by l1s_sample_lambda_workspace_size (for k = 1 it is the
 * l1s_workspace_size of the same arguments). */
L1S_API int l1_sample_lambda(const void* A_dev, int64_t lda, l1s_dtype dtype, const float* b_dev,
                             int64_t n, int32_t d, const float* lambda_dev,
                             const double* lambda_total_dev, const l1s_params* params, int32_t k,
                             int64_t capacity, int64_t* idx_dev, double* w_dev, double* coreset_dev,
                             int64_t* count_dev, void* ws, size_t ws_bytes, void* stream);
L1S_API int l1s_sample_lambda_workspace_size(const l1s_params* params, int64_t n, int32_t d,
                                             l1s_dtype dtype, int32_t k, size_t* bytes);

/* The Bernoulli step alone (Figure 2, step 7) from caller-given probabilities
 * p_dev (n FP64 values in [0,1]): row i kept iff u_i < p_i.  Writes up to
 * capacity ascending indices and *count_dev. */
L1S_API int l1_sample_from_p(const double* p_dev, int64_t n, const l1s_params* params,
                     int64_t capacity, int64_t* idx_dev, int64_t* count_dev,
                     void* ws, size_t ws_bytes, void* stream);

/* The whole sampling pass (Figure 2, steps 1-7): fct_embed, l1_condition,
 * l1_sample, enqueued back to back with intermediates in the workspace.
 * Resets the status word first.  Outputs as in l1_sample. */
L1S_API int l1_coreset(const void* A_dev, int64_t lda, l1s_dtype dtype, const float* b_dev,
               int64_t n, int32_t d, const l1s_params* params, int64_t capacity,
               int64_t* idx_dev, double* w_dev, double* coreset_dev, int64_t* count_dev,
               void* ws, size_t ws_bytes, void* stream);

/* l1_coreset from host memory: copies A (n rows of lda elements) and b from
 * host buffers (pinned memory gives asynchronous copies) into the workspace
 * (sized with host_staging = 1), runs the sampling pass, copies the kept
 * indices and weights (up to capacity) and the count back to host memory and
 * synchronises `stream`.  Returns the first device-side error code, if any. */
L1S_API int l1_coreset_host(const void* A_host, int64_t lda, l1s_dtype dtype, const float* b_host,
                    int64_t n, int32_t d, const l1s_params* params, int64_t capacity,
                    int64_t* idx_host, double* w_host, int64_t* count_host,
                    void* ws, size_t ws_bytes, void* stream);

/* Weighted ℓ1 regression on a coreset (Figure 2, step 8): x̂ minimising
 * Σ_k w_k·|X_k·[x; 1]| over rows X_k = [A_k, −b_k] (coreset_dev, FP64, q per
 * row, count from *count_dev, at most capacity) by FP64 iteratively
 * reweighted least squares, finished by simplex pivots of the LAD linear
 * program from the vertex of the d rows with the smallest residuals whose A
 * parts are linearly independent, up to a vertex whose optimality the dual
 * multipliers certify.  Writes x_dev (d
 * FP64) and *objective_dev (the weighted objective at x_dev).  The status bit
 * L1S_ERR_NOT_CONVERGED is raised when neither the iteration converged nor the
 * vertex was certified optimal. */
L1S_API int l1_solve(const double* coreset_dev, const double* w_dev, const int64_t* count_dev,
             int64_t capacity, int32_t d, int32_t max_iter, double* x_dev,
             double* objective_dev, void* ws, size_t ws_bytes, void* stream);

/* l1_solve for k coresets side by side (the k approximate solutions of §6.3): coreset j
 * is rows coreset_dev + j·capacity·q, weights w_dev + j·capacity and count_dev[j], the
 * layout l1_sample_lambda writes.  Each is solved as l1_solve solves one (its
 * accumulation spread over fewer blocks, so sums may round differently); writes x_dev
 * (k × d FP64), objective_dev (k) and, when flags_dev is not NULL, flags_dev[j] = the
 * status flags of coreset j's solve (L1S_FLAG(L1S_ERR_NOT_CONVERGED) as in l1_solve).
 * 1 ≤ k ≤ 1024; workspace sized by l1s_solve_many_workspace_size. */
L1S_API int l1_solve_many(const double* coreset_dev, const double* w_dev, const int64_t* count_dev,
                          int64_t capacity, int32_t d, int32_t k, int32_t max_iter, double* x_dev,
                          double* objective_dev, uint32_t* flags_dev, void* ws, size_t ws_bytes,
                          void* stream);
L1S_API int l1s_solve_many_workspace_size(int64_t capacity, int32_t d, int32_t k, size_t* bytes);

/* ‖A·x − b‖₁ in FP64 over all n rows (problem statement, §4.2). */
L1S_API int l1_objective(const void* A_dev, int64_t lda, l1s_dtype dtype, const float* b_dev,
                 int64_t n, int32_t d, const double* x_dev, double* objective_dev,
                 void* ws, size_t ws_bytes, void* stream);

/* FastCauchyRegression end to end (Figure 2, steps 1-8): l1_coreset with a
 * coreset capacity of 2·m_s + 64 rows, l1_solve, l1_objective.  A and b are
 * device pointers (inputs_on_host = 0) or host pointers (inputs_on_host = 1,
 * workspace sized with host_staging = 1).  Synchronises `stream`; writes
 * x_host (d FP64), *objective_host and *coreset_rows_host (may be NULL) and
 * returns the first device-side error code, if any. */
L1S_API int l1_regress(const void* A, int64_t lda, l1s_dtype dtype, const float* b,
               int64_t n, int32_t d, const l1s_params* params, int32_t inputs_on_host,
               double* x_host, double* objective_host, int64_t* coreset_rows_host,
               void* ws, size_t ws_bytes, void* stream);

/* Multiple ℓ1 regression (§4.2.1): min_W ‖A·W − B‖₁ with A ∈ R^{n×d} and B ∈ R^{n×k},
 * FastCauchyRegression(A, B): the steps of Figure 2 on X = [A, −B] (q = d + k columns)
 * give one coreset for all k right-hand sides.  X_dev holds [A | B] row by row (n rows
 * of d + k values, leading dimension ldx ≥ d + k, FP32 or BF16 storage; device memory,
 * caller-owned).  d ≥ 1, k ≥ 1, d + k − 1 ≤ 128; the other limits are those of
 * l1s_workspace_size with d + k − 1 columns.  The workspace is sized by
 * l1s_multi_workspace_size. */
L1S_API int l1s_multi_workspace_size(const l1s_params* params, int64_t n, int32_t d, int32_t k,
                                     l1s_dtype dtype, size_t* bytes);

/* Steps 1-7 on X = [A, −B]: writes the kept row indices (ascending), weights 1/p̂ and,
 * when coreset_dev is not NULL, the kept rows of X (FP64, d + k values per row: A_i then
 * −B_i) for up to `capacity` rows, and *count_dev (all kept rows; L1S_ERR_CAPACITY is
 * raised in the status word when it exceeds capacity).  Asynchronous on `stream`. */
L1S_API int l1_coreset_multi(const void* X_dev, int64_t ldx, l1s_dtype dtype, int64_t n, int32_t d,
                             int32_t k, const l1s_params* params, int64_t capacity, int64_t* idx_dev,
                             double* w_dev, double* coreset_dev, int64_t* count_dev,
                             void* ws, size_t ws_bytes, void* stream);

/* FastCauchyRegression(A, B) end to end: l1_coreset_multi with a capacity of
 * 2·m_s + 64 rows, then for each right-hand side j the weighted ℓ1 problem
 * min_w Σ_i w_i·|A_i·w − B_ij| on the coreset (as l1_solve, max_iter IRLS steps) and
 * its objective ‖A·w_j − B_j‖₁ over all n rows.  Synchronises `stream`; writes W_host
 * (d × k row-major FP64: column j solves right-hand side j), objectives_host (k FP64)
 * and *coreset_rows_host (may be NULL); returns the first device-side error code. */
L1S_API int l1_regress_multi(const void* X_dev, int64_t ldx, l1s_dtype dtype, int64_t n, int32_t d,
                             int32_t k, const l1s_params* params, int32_t max_iter, double* W_host,
                             double* objectives_host, int64_t* coreset_rows_host,
                             void* ws, size_t ws_bytes, void* stream);

/* Debug: one thread waits, at most max_cycles SM clock cycles (1000 … 4e9), on a
 * barrier that nothing completes — the bounded wait of the pipelined kernels — and then
 * raises L1S_ERR_TIMEOUT in the status word of `ws` and returns, leaving the context
 * usable.  Lets a test exercise the timeout path without faulting or hanging the GPU. */
L1S_API int l1s_debug_wait_timeout(void* ws, size_t ws_bytes, int64_t max_cycles, void* stream);

/* Debug: the Philox draws of global rows [row_start, row_start + count) as the
 * kernels use them (device outputs, any may be NULL): bucket_h/bucket_i in
 * [0, r1), k_h/k_i the 24-bit integers of the Cauchy scales, cauchy_h/cauchy_i
 * the FP32 Cauchy variates, sign (±1), u_bits the 53-bit sampling integers. */
L1S_API int l1s_debug_variates(const l1s_params* params, int64_t row_start, int64_t count,
                       int32_t* bucket_h, int32_t* bucket_i, int32_t* k_h, int32_t* k_i,
                       float* cauchy_h, float* cauchy_i, int8_t* sign, uint64_t* u_bits,
                       void* stream);

/* Debug: Π2 (q × r2, FP64, row-major) as l1_condition draws it. */
L1S_API int l1s_debug_pi2(const l1s_params* params, int32_t q, double* pi2_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Launch schedules and the autotuner
 *
 * A schedule fixes how the kernels of one (d, dtype, s) tile the work; it never
 * changes what they compute (s itself is a parameter of Π1, §3.1, and is not
 * tuned here).  Zero fields mean "the default rule".
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t fct_variant;       /* phase 1 kernel: 0 default, 1 warp-specialised narrow-X kernel
                                (d ≤ 32, 2 ≤ s ≤ 512), 2 all columns with TMA-staged tiles,
                                3 direct loads over column slices sized for two blocks per SM,
                                4 bucket-sorted scatter (d ≤ 32, 32 ≤ s ≤ 512), 5 the narrow-X
                                kernel with one stage buffer and one copy of its partial
                                (d ≤ 16), 6 direct loads over the widest column slices that one
                                block per SM allows, 7 the column-sliced wide-X kernel (16
                                columns of A per block, one block per SM, s ≤ 1024, the b column
                                in a kernel of its own; the default for d > 32).  A variant that
                                does not apply to the shape falls back to the default. */
  int32_t fct_ctas_per_sm;   /* phase 1 resident blocks per SM (capped by occupancy); 0 = most */
  int32_t lam_ctas_per_sm;   /* λ pass blocks per SM, 1..32; 0 = 8 */
  int32_t smp_chunks_per_sm; /* sampling row chunks per SM, 1..16; 0 = 4 */
} l1s_schedule;

/* Install `sch` for every later call on this process with this d, dtype and s
 * (NULL removes the entry).  Workspace sizes do not depend on the schedule. */
L1S_API int l1s_schedule_set(int32_t d, l1s_dtype dtype, int32_t s, const l1s_schedule* sch);

/* The schedule installed for (d, dtype, s); all zeros when none is. */
L1S_API int l1s_schedule_get(int32_t d, l1s_dtype dtype, int32_t s, l1s_schedule* sch);

/* One problem of a batch (device pointers).  idx/w/coreset/count, x and
 * objective may be NULL: the coreset then stays in the workspace, and the
 * solve (Figure 2, step 8) runs only when x is non-NULL. */
typedef struct {
  const void* A_dev;         /* n × d, leading dimension lda, FP32 or BF16 */
  const float* b_dev;        /* n */
  int64_t lda;
  int64_t n;
  int32_t d;
  l1s_dtype dtype;
  l1s_params params;
  int64_t capacity;          /* rows of idx_dev / w_dev / coreset_dev */
  int64_t* idx_dev;          /* kept row ids, ascending */
  double* w_dev;             /* weights 1/p̂ */
  double* coreset_dev;       /* capacity × q FP64 rows w·X_i (may be NULL) */
  int64_t* count_dev;        /* number of kept rows */
  double* x_dev;             /* d: the coreset solution x̂ (NULL: no solve) */
  double* objective_dev;     /* 1: ‖A·x̂ − b‖₁ over all n rows (needs x_dev) */
} l1s_problem;

/* Time the schedules that apply to `prob`'s shape (l1_coreset on its data,
 * median of `trials` runs per candidate, CUDA events on `stream`), install
 * the fastest with l1s_schedule_set, and return it in *best (and its time in
 * *best_ms when non-NULL).  The workspace is sized by l1s_workspace_size for
 * the problem.  Synchronises `stream`; not for use inside stream capture. */
L1S_API int l1s_autotune(const l1s_problem* prob, int32_t trials, l1s_schedule* best, double* best_ms,
                         void* ws, size_t ws_bytes, void* stream);

/* Device workspace for l1_regress_batched over these problems. */
L1S_API int l1s_batched_workspace_size(const l1s_problem* probs, int32_t count, size_t* bytes);

/* Many independent regressions (Figure 2 per problem, each with its own n, d,
 * dtype and params) in one call.  The problems are spread over a pool of
 * library-owned streams (longest first, each onto the least loaded stream)
 * that fork from `stream` and join back into it, so the whole batch can be
 * captured into one CUDA graph and replayed.  λ reads M from shared memory
 * here, so concurrent problems do not share the constant bank.  flags_dev
 * (count uint32, may be NULL) receives each problem's status word.  Enqueues
 * only; `stream` sees every problem finished.  The caller keeps every member's
 * buffers alive until then. */
L1S_API int l1_regress_batched(const l1s_problem* probs, int32_t count, uint32_t* flags_dev, void* ws,
                               size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* L1FCT_H */
