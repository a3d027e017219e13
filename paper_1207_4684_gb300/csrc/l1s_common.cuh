// Shared device helpers and host plumbing of libl1fct (CUDA side only).
//
// Random draws: Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw
// (SC'11), written here for the device.  Each 10-round call maps a 128-bit
// counter and a 64-bit key to four 32-bit words; the method's random objects
// (§3.1: the ±1 diagonal, the Cauchy diagonal C and the hash matrix B;
// Figure 2: Π2 and the sampling uniforms) are read from those words as
// described in include/l1fct.h.
#pragma once

#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/l1fct.h"

namespace l1s {

// ----------------------------------------------------------------- limits
constexpr int kMaxLog2S = 12;       // s ≤ 4096
constexpr int kMaxD = 128;          // d ≤ 128 (q ≤ 129)
constexpr int kMaxCoresets = 1024;  // coresets per l1_sample_lambda / l1_solve_many call
constexpr int kMaxR2 = 64;
constexpr int kMaxConstM = 129 * 64;

// Draw streams (counter word 3).
constexpr uint32_t kStreamFct = 0;
constexpr uint32_t kStreamPi2 = 1;
constexpr uint32_t kStreamSample = 2;
constexpr uint32_t kStreamReplace = 3;   // with-replacement draws (params.variant = 2)

// Status word layout inside the workspace (first 256 bytes).
struct StatusBlock {
  uint32_t flags;        // OR of L1S_FLAG(code)
  uint32_t pad0;
  int64_t count;         // coreset rows kept (before capacity clipping)
  double lambda_total;   // Σλ
  double tau;            // m_s / Σλ
  float tau32;           // τ rounded to FP32 (fast pre-test in phase 3)
  uint32_t irls_done;    // IRLS convergence flag
  double irls_prev_obj;  // IRLS objective of the previous iterate
  double irls_obj;       // IRLS objective of the current iterate
  double irls_eta;       // IRLS smoothing floor
  int32_t irls_iters;
  uint32_t cond_ticket;  // blocks of the conditioning pass that have finished
  uint32_t qr_breakdown; // 1: CholeskyQR2 broke down (the Householder QR then redoes the step)
};

__device__ __forceinline__ void raise_flag(uint32_t* flags, int code) {
  atomicOr(flags, L1S_FLAG(code));
}

// ----------------------------------------------------------------- Philox4x32-10
struct Key2 {
  uint32_t k0, k1;
};

__host__ __device__ __forceinline__ Key2 make_key(uint64_t seed) {
  return Key2{static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)};
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, Key2 k) {
  constexpr uint32_t kMulA = 0xD2511F53u;  // multiplies counter word 0
  constexpr uint32_t kMulB = 0xCD9E8D57u;  // multiplies counter word 2
  constexpr uint32_t kWeylA = 0x9E3779B9u;
  constexpr uint32_t kWeylB = 0xBB67AE85u;
  uint32_t k0 = k.k0, k1 = k.k1;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hiA = __umulhi(kMulA, c.x);
    const uint32_t loA = kMulA * c.x;
    const uint32_t hiB = __umulhi(kMulB, c.z);
    const uint32_t loB = kMulB * c.z;
    c = make_uint4(hiB ^ c.y ^ k0, loB, hiA ^ c.w ^ k1, loA);
    k0 += kWeylA;
    k1 += kWeylB;
  }
  return c;
}

__device__ __forceinline__ uint4 draw_row(Key2 key, uint64_t row, uint32_t problem, uint32_t stream) {
  return philox4x32_10(make_uint4(static_cast<uint32_t>(row), static_cast<uint32_t>(row >> 32),
                                  problem, stream), key);
}

// Bucket in [0, r) from a 32-bit word: high half of word·r.
__device__ __forceinline__ int bucket_of(uint32_t word, uint32_t r) {
  return static_cast<int>(__umulhi(word, r));
}

// Standard Cauchy from the 24-bit integer k: tan(π(u − ½)) at u = (k + ½)/2^24,
// evaluated through the reflection w = ½ − |u − ½| = j·2^-25 (j odd, exact in FP32) as
// ±cot(πw), which keeps full relative accuracy near the poles.  With a = min(w, ½ − w) ≤ ¼
// (exact), sin(πa) = a·P(a²) and cos(πa) = Q(a²), P and Q the Taylor series of sin(πa)/a and
// cos(πa) about 0 truncated after the a⁸ terms (on |πa| ≤ π/4 the truncation is below 3e-8
// relative), coefficients (−1)^k π^{2k+1}/(2k+1)! and (−1)^k π^{2k}/(2k)! rounded to FP32;
// cot(πw) = Q/(a·P) when w ≤ ¼ and a·P/Q otherwise (cos(πw) = sin(π(½ − w))).  With the
// correctly rounded quotient the variate is within 2.5e-7 relative of cot(πw) for every k.
__device__ __forceinline__ float cauchy_f32(uint32_t k) {
  const int m = 2 * static_cast<int>(k) + 1 - (1 << 24);
  const int j = (1 << 24) - abs(m);
  const bool low = j <= (1 << 23);                       // w ≤ ¼
  const float a = static_cast<float>(low ? j : (1 << 24) - j) * 0x1p-25f;
  const float a2 = a * a;
  float p = 0.08214588463306427f;                        //  π⁹/9!
  p = fmaf(p, a2, -0.5992645025253296f);                 // −π⁷/7!
  p = fmaf(p, a2, 2.550163984298706f);                   //  π⁵/5!
  p = fmaf(p, a2, -5.167712688446045f);                  // −π³/3!
  p = fmaf(p, a2, 3.1415927410125732f);                  //  π
  const float sn = a * p;
  float c = 0.23533062636852264f;                        //  π⁸/8!
  c = fmaf(c, a2, -1.3352627754211426f);                 // −π⁶/6!
  c = fmaf(c, a2, 4.058712005615234f);                   //  π⁴/4!
  c = fmaf(c, a2, -4.934802055358887f);                  // −π²/2!
  c = fmaf(c, a2, 1.0f);
  const float r = low ? __fdiv_rn(c, sn) : __fdiv_rn(sn, c);
  return m > 0 ? r : -r;
}

__device__ __forceinline__ double cauchy_f64(uint32_t k) {
  const int m = 2 * static_cast<int>(k) + 1 - (1 << 24);
  const int j = (1 << 24) - abs(m);
  const double w = static_cast<double>(j) * 0x1p-25;
  double sn, cs;
  sincospi(w, &sn, &cs);
  const double r = cs / sn;
  return m > 0 ? r : -r;
}

// 53-bit sampling integer of row `row` from its stream-2 words (a, b).
__device__ __forceinline__ uint64_t u53_of(uint32_t wa, uint32_t wb) {
  return (static_cast<uint64_t>(wa >> 5) << 26) | static_cast<uint64_t>(wb >> 6);
}

// ----------------------------------------------------------------- packed FP32 pairs
// Two FP32 values in one 64-bit register, for the packed add/sub/fma of sm_100-class
// parts: each lane is rounded as the scalar instruction rounds it, so a butterfly on a
// pair gives exactly the two scalar results.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t p, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Stages t of a register butterfly run on row bit first + t, and only below log2 s: the
// mask of the stages that run.
__device__ __forceinline__ uint32_t f2_stage_mask(int first, int lg) {
  const int k = lg - first;
  return k <= 0 ? 0u : (k >= 32 ? 0xFFFFFFFFu : ((1u << k) - 1u));
}

// Radix-2 butterflies over the index bits of a register column v[0..N) held as the pairs
// p[k] = (v[k], v[k + N/2]), in the order of the bits: stages over the low log2(N/2) bits
// run on pairs, the top stage inside each pair.  Stage t runs when bit t of `stages` is set.
template <int N>
__device__ __forceinline__ void f2_butterflies(uint64_t (&p)[N / 2], uint32_t stages) {
  constexpr int H = N / 2;
  constexpr int LH = H >= 16 ? 4 : (H >= 8 ? 3 : (H >= 4 ? 2 : (H >= 2 ? 1 : 0)));
  static_assert((1 << LH) == H, "N must be a power of two from 2 to 32");
#pragma unroll
  for (int b = 0; b < LH; ++b)
    if ((stages >> b) & 1u)
#pragma unroll
      for (int k = 0; k < H; ++k)
        if ((k & (1 << b)) == 0) {
          const uint64_t lo = p[k], hi = p[k | (1 << b)];
          p[k] = f2_add(lo, hi);
          p[k | (1 << b)] = f2_sub(lo, hi);
        }
  if ((stages >> LH) & 1u)
#pragma unroll
    for (int k = 0; k < H; ++k) {
      float x, y;
      f2_unpack(p[k], x, y);
      p[k] = f2_pack(x + y, x - y);
    }
}

// ----------------------------------------------------------------- TMA bulk copies and mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order earlier generic-proxy accesses of shared memory before later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 1-D bulk copy global → shared (16-byte aligned addresses, size a multiple of 16),
// completion counted on `bar` in bytes.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar` for at most max_cycles SM clocks; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long max_cycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > max_cycles) return false;
  }
  return true;
}

constexpr long long kWaitCycles = 4000000000LL;  // about two seconds at 2 GHz

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Named barrier `id` over `count` threads (a multiple of 32).
__device__ __forceinline__ void named_barrier(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Named barrier that also ORs a predicate over the participating threads.
__device__ __forceinline__ bool named_barrier_any(int id, int count, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred ? 1u : 0u), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

// ----------------------------------------------------------------- element loads
template <typename T>
__device__ __forceinline__ float load_elem(const T* p);
template <>
__device__ __forceinline__ float load_elem<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_elem<uint16_t>(const uint16_t* p) {
  return __uint_as_float(static_cast<uint32_t>(__ldg(p)) << 16);
}

// ----------------------------------------------------------------- host side
struct DeviceInfo {
  int device;
  int sms;
  int max_smem_optin;
};
DeviceInfo device_info();

void set_error(const char* fmt, ...);

// A named range of an entry point on a profiler's timeline (NVTX; a no-op without a tool).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
bool cuda_ok(cudaError_t e, const char* what);
// Raises fn's dynamic shared-memory limit on the current device to at least `bytes` and
// never lowers it, under a lock, so that calls of different shapes from several host
// threads cannot lower the limit another call has set for its own launch.  False (with
// the CUDA error recorded) when the runtime refuses.
bool allow_dynamic_smem(const void* fn, size_t bytes, const char* what);

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

inline int log2_exact(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return (int64_t(1) << l) == v ? l : -1;
}

// Launch geometry and workspace regions, a pure function of (params, n, d, dtype, device).
struct Plan {
  int64_t n;
  int d, q, s, log2s, r1, r2;
  int64_t nblocks;          // ⌈n / s⌉
  int fct_threads;
  int fct_slices, fct_width;  // column slices of Π1X handled per thread block
  int fct_staged;           // 1: tiles of X arrive in shared memory by TMA bulk copies
  int fct_ws;               // 16 or 32: the narrow-X kernel with that column width runs phase 1
  int fct_tile_log2;        // its tile (rows per pipeline step, 2^fct_tile_log2 ≥ s)
  int fct_lean;             // 1: its one-stage, one-copy form (W = 16)
  int fct_sorted;           // 16 or 32: the bucket-sorted kernel with that column width runs phase 1
  int fct_cols;             // > 0: the column-sliced wide-X kernel runs phase 1 over this many 16-column slices
  int fct_ctas;             // thread blocks per slice
  int fct_chunks;           // inputs in host memory: row chunks whose copies overlap phase 1
  size_t fct_smem;
  int lam_ctas, lam_threads;
  int lam_m_in_smem;        // 1: the λ kernel reads M from shared memory instead of the constant bank
  int smp_ctas, smp_threads;
  int64_t smp_chunk;        // rows per sampling block (multiple of 64)
  int pi2_neg_lo, pi2_neg_hi;  // multiple regression: Π2 rows stored negated (columns read as +B)
  int lm_ctas;              // the fused λ-and-mark pass: blocks and rows per block (λ residency)
  int64_t lm_chunk;
  int irls_ctas;
  int fjlt_rows;            // FCT2: rows of G kept per block of s rows
  int64_t fjlt_n;           // FCT2: rows of H̃X, ⌈n/s⌉·fjlt_rows
  // workspace offsets (bytes)
  size_t off_status, off_partials, off_pix, off_qr, off_r, off_m64, off_m32, off_pi2,
      off_lam, off_lamsum, off_mask, off_counts, off_idx_tmp, off_irls, off_x, off_objp,
      off_stage_a, off_stage_b, off_cdf, off_draws, off_fjlt, total;
};

bool make_plan(const l1s_params* p, int64_t n, int d, l1s_dtype dt, bool host_staging, Plan* plan,
               const l1s_schedule* override_sch = nullptr);
// Π2 entry e (row-major q × r2): word e mod 4 of Philox call ⌊e/4⌋ on stream 1.
__device__ __forceinline__ double pi2_entry(Key2 key, uint32_t problem, int e) {
  const uint4 o = philox4x32_10(make_uint4(static_cast<uint32_t>(e >> 2), 0u, problem, kStreamPi2), key);
  const uint32_t w = (e & 3) == 0 ? o.x : (e & 3) == 1 ? o.y : (e & 3) == 2 ? o.z : o.w;
  return cauchy_f64(w >> 8);
}

// Gaussian Π2 entry e (OptimizedFastCauchyRegression): Box–Muller on Philox call ⌊e/2⌋ of
// stream 1 with two open 53-bit uniforms, u1 from words (0, 1) and u2 from (2, 3);
// entry 2t is √(−2 ln u1)·cos(2π u2), entry 2t+1 the sine.
__device__ __forceinline__ double pi2_entry_gaussian(Key2 key, uint32_t problem, int e) {
  const uint4 o = philox4x32_10(make_uint4(static_cast<uint32_t>(e >> 1), 0u, problem, kStreamPi2), key);
  const double u1 = (static_cast<double>(u53_of(o.x, o.y)) + 0.5) * 0x1p-53;
  const double u2 = (static_cast<double>(u53_of(o.z, o.w)) + 0.5) * 0x1p-53;
  const double rho = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return rho * ((e & 1) ? sn : cs);
}

__device__ __forceinline__ double pi2_value(Key2 key, uint32_t problem, int e, int gaussian) {
  return gaussian ? pi2_entry_gaussian(key, problem, e) : pi2_entry(key, problem, e);
}

// Σ of the λ block partials in a fixed order, for a block of 256 threads: strided
// per-thread sums, a fixed shuffle tree, then the eight warp sums in order (every
// thread returns the total).  The finalize kernel and the sampling kernel both use it,
// so they obtain the same bits.
__device__ __forceinline__ double lambda_total_256(const double* __restrict__ sums, int n, double* wsum8) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += sums[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) wsum8[threadIdx.x >> 5] = acc;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < 8; ++w) tot += wsum8[w];
  return tot;
}

// τ = m_s / Σλ (FP64, one division) and its FP32 copy; false when Σλ is zero or not finite.
__device__ __forceinline__ bool tau_of(double tot, double coreset, double* tau, float* tau32) {
  if (!(tot > 0.0) || !isfinite(tot)) {
    *tau = 0.0;
    *tau32 = 0.f;
    return false;
  }
  *tau = coreset / tot;
  *tau32 = *tau > static_cast<double>(FLT_MAX) ? FLT_MAX : static_cast<float>(*tau);
  return true;
}

// Keep mask bits: lane t's even row goes to bit 2t, its odd row to bit 2t+1.
__device__ __forceinline__ uint64_t spread_bits(uint32_t x) {
  uint64_t v = x;
  v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
  v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
  v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  v = (v | (v << 1)) & 0x5555555555555555ull;
  return v;
}

// p̂ = min(1, τ·λ) in FP64 (the exact definition both sides evaluate).
__device__ __forceinline__ double p_hat(double tau, float lam) { return fmin(1.0, tau * static_cast<double>(lam)); }

// Keep decision for one row: exact result of (U·2^-53 < min(1, τ·λ)).
__device__ __forceinline__ bool keep_row(float lam, float tau32, double tau, uint32_t wa, uint32_t wb) {
  const float p32 = lam > 0.f ? fminf(1.f, tau32 * lam) : 0.f;
  const float u_lo = static_cast<float>(wa >> 8) * 0x1p-24f;   // u ∈ [u_lo, u_lo + 2^-24)
  const float u_hi = u_lo + 0x1p-24f;
  if (u_hi < p32 * (1.f - 0x1p-20f)) return true;
  if (u_lo > p32 * (1.f + 0x1p-20f)) return false;
  const double u = static_cast<double>(u53_of(wa, wb)) * 0x1p-53;
  return u < p_hat(tau, lam);
}

// Adds k to the process-wide count of kernels the library has launched.
void count_launch(int k);
// The schedule installed for (d, dt, log2 s); false (and *out zeroed) when none is.
bool schedule_lookup(int d, l1s_dtype dt, int log2s, l1s_schedule* out);

}  // namespace l1s
