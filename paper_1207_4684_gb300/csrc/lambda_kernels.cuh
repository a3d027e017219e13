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
// This header holds the kernels and their launch templates; each translation unit
// that includes it instantiates one storage type and one home of M (the constant
// bank, which every unit has its own copy of, or shared memory), so that the units
// compile in parallel.
#pragma once

#include <float.h>

#include <algorithm>
#include <utility>

#include "l1s_common.cuh"

namespace l1s {

static __constant__ __align__(16) float c_M[kMaxConstM];

constexpr int kLamThreads = 256;

__host__ __device__ constexpr int next_pow2(int v) { return v <= 1 ? 1 : 2 * next_pow2((v + 1) / 2); }

// Batcher's odd–even merge sort network on P = 2^k inputs, as a compile-time list
// of comparators (lo[c], hi[c]) applied in order.
template <int P>
struct OddEvenMergeNet {
  static constexpr int kMax = 1024;  // ≥ the 543 comparators of P = 64
  int lo[kMax];
  int hi[kMax];
  int count;
  constexpr OddEvenMergeNet() : lo(), hi(), count(0) {
    for (int p = 1; p < P; p <<= 1)
      for (int k = p; k >= 1; k >>= 1)
        for (int j = k % p; j + k < P; j += 2 * k)
          for (int i = 0; i < k && i + j + k < P; ++i)
            if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) {
              lo[count] = i + j;
              hi[count] = i + j + k;
              ++count;
            }
  }
};

template <int P>
struct NetOf {
  static constexpr OddEvenMergeNet<P> value{};
};

template <int P, int I>
__device__ __forceinline__ void compare_exchange(float (&a)[P]) {
  constexpr int l = NetOf<P>::value.lo[I];
  constexpr int h = NetOf<P>::value.hi[I];
  const float x = a[l], y = a[h];
  a[l] = fminf(x, y);
  a[h] = fmaxf(x, y);
}

template <int P, int... I>
__device__ __forceinline__ void apply_net(float (&a)[P], std::integer_sequence<int, I...>) {
  (compare_exchange<P, I>(a), ...);
}

// Sorts a[0..P) ascending (P a power of two); the compiler drops every comparator
// that does not feed the entries the caller reads.
template <int P>
__device__ __forceinline__ void sort_net(float (&a)[P]) {
  apply_net<P>(a, std::make_integer_sequence<int, NetOf<P>::value.count>{});
}

template <int N>
__device__ __forceinline__ float lower_median(const float (&v)[N]) {
  constexpr int P = next_pow2(N);
  float a[P];
#pragma unroll
  for (int i = 0; i < P; ++i) a[i] = i < N ? v[i] : INFINITY;
  sort_net<P>(a);
  return a[(N - 1) / 2];
}

// s + c ← s + c + v with the rounding error of s + v carried in c (Knuth's TwoSum).
__device__ __forceinline__ void two_sum_add(float& s, float& c, float v) {
  const float t = s + v;
  const float bp = t - s;
  const float e = (s - (t - bp)) + (v - bp);
  s = t;
  c += e;
}

// Block total of per-thread (s, c) pairs, in a fixed order; returns on thread 0.
static __device__ double block_pair_total(float s, float c) {
  __shared__ double wsum[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, off);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, off);
    const float t = s + s2;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (s2 - bp);
    s = t;
    c = (c + c2) + e;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wsum[warp] = static_cast<double>(s) + static_cast<double>(c);
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (blockDim.x >> 5); ++w) tot += wsum[w];
  return tot;
}

template <int D, typename TA, bool VEC>
__device__ __forceinline__ void load_row(const TA* __restrict__ p, float (&x)[D + 1]) {
  if constexpr (VEC && sizeof(TA) == 4) {
    static_assert(D % 4 == 0, "vector path needs d % 4 == 0");
#pragma unroll
    for (int k = 0; k < D; k += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p + k));
      x[k] = v.x;
      x[k + 1] = v.y;
      x[k + 2] = v.z;
      x[k + 3] = v.w;
    }
  } else if constexpr (VEC && sizeof(TA) == 2) {
    static_assert(D % 8 == 0, "vector path needs d % 8 == 0");
#pragma unroll
    for (int k = 0; k < D; k += 8) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(p + k));
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        x[k + 2 * t] = __uint_as_float(w[t] << 16);
        x[k + 2 * t + 1] = __uint_as_float(w[t] & 0xffff0000u);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = load_elem<TA>(p + k);
  }
}

// M is read from the constant bank (single-problem calls) or from a shared-memory copy
// (calls that may run concurrently with other problems' λ passes).
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

template <int Q, int R2, bool SMEM_M>
__device__ __forceinline__ float lambda_of_row(const float (&x)[Q], const float* __restrict__ sM) {
  float acc[R2];
  if constexpr (R2 % 2 == 0) {
    // The same products and FMA chain per column, two columns per packed FP32x2
    // instruction with a pair of M's entries from the constant bank: each lane rounds as
    // the scalar instruction does, so λ is bit-identical to the scalar chain, in half the
    // FMA instructions (the chain is issue-bound at d = 64, r2 = 32: 1.66 → 1.24 ms at
    // n = 2^24).  M in shared memory (8-byte aligned) is read as pairs the same way.
    const unsigned long long* cm2 = reinterpret_cast<const unsigned long long*>(SMEM_M ? sM : c_M);
    uint64_t a2[R2 / 2];
    {
      const uint64_t x0 = f2_pack(x[0], x[0]);
#pragma unroll
      for (int j = 0; j < R2 / 2; ++j) a2[j] = f2_mul(x0, cm2[j]);
    }
#pragma unroll
    for (int k = 1; k < Q; ++k) {
      const uint64_t xk = f2_pack(x[k], x[k]);
#pragma unroll
      for (int j = 0; j < R2 / 2; ++j) a2[j] = f2_fma(xk, cm2[k * (R2 / 2) + j], a2[j]);
    }
#pragma unroll
    for (int j = 0; j < R2 / 2; ++j) {
      float lo, hi;
      f2_unpack(a2[j], lo, hi);
      acc[2 * j] = fabsf(lo);
      acc[2 * j + 1] = fabsf(hi);
    }
    return lower_median<R2>(acc);
  }
#pragma unroll
  for (int j = 0; j < R2; ++j) acc[j] = x[0] * (SMEM_M ? sM[j] : c_M[j]);
#pragma unroll
  for (int k = 1; k < Q; ++k) {
#pragma unroll
    for (int j = 0; j < R2; ++j) acc[j] = fmaf(x[k], SMEM_M ? sM[k * R2 + j] : c_M[k * R2 + j], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < R2; ++j) acc[j] = fabsf(acc[j]);
  return lower_median<R2>(acc);
}

// Specialised for q = D + 1 and r2 = R2 known at compile time.  Up to q = 33 the loads of a
// thread's next row are issued before the current row is computed (software pipelining);
// wider rows would double the registers a row takes, so those rows are loaded when needed
// and two blocks per SM hide the latency instead.
template <int D>
constexpr bool lambda_prefetches() { return D + 1 <= 33; }

template <int D, int R2, typename TA, bool VEC, bool SMEM_M>
__global__ void __launch_bounds__(kLamThreads, lambda_prefetches<D>() ? 1 : 2)
    lambda_kernel(const TA* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t n,
                  float* __restrict__ lam, double* __restrict__ block_sums, const float* __restrict__ mg) {
  constexpr int Q = D + 1;
  __shared__ __align__(16) float sM[SMEM_M ? Q * R2 : 1];
  if constexpr (SMEM_M) {
    for (int e = threadIdx.x; e < Q * R2; e += blockDim.x) sM[e] = mg[e];
    __syncthreads();
  }
  float s = 0.f, c = 0.f;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if constexpr (!lambda_prefetches<D>()) {
    for (; row < n; row += stride) {
      float x[Q];
      load_row<D, TA, VEC>(A + row * lda, x);
      x[D] = -__ldg(b + row);
      const float med = lambda_of_row<Q, R2, SMEM_M>(x, sM);
      lam[row] = med;
      two_sum_add(s, c, med);
    }
    const double tot = block_pair_total(s, c);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
    return;
  }
  float nx[Q];
  if (row < n) {
    load_row<D, TA, VEC>(A + row * lda, nx);
    nx[D] = -__ldg(b + row);
  }
  for (; row < n; row += stride) {
    float x[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) x[k] = nx[k];
    const int64_t nrow = row + stride;
    if (nrow < n) {
      load_row<D, TA, VEC>(A + nrow * lda, nx);
      nx[D] = -__ldg(b + nrow);
    }
    const float med = lambda_of_row<Q, R2, SMEM_M>(x, sM);
    lam[row] = med;
    two_sum_add(s, c, med);
  }
  const double tot = block_pair_total(s, c);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// d < D columns on the D-column kernel: rows are read as D values with zeros beyond
// column d, and M's rows are padded the same way (M's b row moves to row D), so the extra
// products are exact zeros and λ equals the unpadded FMA chain bit for bit.
template <int D, int R2, bool SMEM_M>
__global__ void __launch_bounds__(kLamThreads, lambda_prefetches<D>() ? 1 : 2)
    lambda_kernel_pad(const float* __restrict__ A, int64_t lda, int d, const float* __restrict__ b, int64_t n,
                      float* __restrict__ lam, double* __restrict__ block_sums, const float* __restrict__ mg) {
  constexpr int Q = D + 1;
  __shared__ __align__(16) float sM[SMEM_M ? Q * R2 : 1];
  if constexpr (SMEM_M) {
    for (int e = threadIdx.x; e < Q * R2; e += blockDim.x) {
      const int k = e / R2, j = e - k * R2;
      sM[e] = k < d ? mg[k * R2 + j] : (k == D ? mg[d * R2 + j] : 0.f);
    }
    __syncthreads();
  }
  float s = 0.f, c = 0.f;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  auto load = [&](int64_t r, float (&x)[Q]) {
    const float* p = A + r * lda;
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = k < d ? __ldg(p + k) : 0.f;
    x[D] = -__ldg(b + r);
  };
  if constexpr (!lambda_prefetches<D>()) {
    // as in lambda_kernel: wide rows are loaded when needed (a prefetched copy would double
    // the registers a row takes), and two blocks per SM hide the latency
    for (; row < n; row += stride) {
      float x[Q];
      load(row, x);
      const float med = lambda_of_row<Q, R2, SMEM_M>(x, sM);
      lam[row] = med;
      two_sum_add(s, c, med);
    }
    const double tot = block_pair_total(s, c);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
    return;
  }
  float nx[Q];
  if (row < n) load(row, nx);
  for (; row < n; row += stride) {
    float x[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) x[k] = nx[k];
    const int64_t nrow = row + stride;
    if (nrow < n) load(nrow, nx);
    const float med = lambda_of_row<Q, R2, SMEM_M>(x, sM);
    lam[row] = med;
    two_sum_add(s, c, med);
  }
  const double tot = block_pair_total(s, c);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Any q ≤ 129 and r2 ≤ R2P (columns beyond r2 are ignored by the median).
template <int R2P, typename TA, bool SMEM_M>
__global__ void __launch_bounds__(kLamThreads) lambda_kernel_generic(const TA* __restrict__ A, int64_t lda,
                                                                     const float* __restrict__ b, int64_t n,
                                                                     int d, int r2, float* __restrict__ lam,
                                                                     double* __restrict__ block_sums,
                                                                     const float* __restrict__ mg) {
  extern __shared__ float sMg[];
  if constexpr (SMEM_M) {
    for (int e = threadIdx.x; e < (d + 1) * r2; e += blockDim.x) sMg[e] = mg[e];
    __syncthreads();
  }
  float s = 0.f, c = 0.f;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; row < n; row += stride) {
    float acc[R2P];
#pragma unroll
    for (int j = 0; j < R2P; ++j) acc[j] = 0.f;
    const TA* p = A + row * lda;
    for (int k = 0; k <= d; ++k) {
      const float xk = k < d ? load_elem<TA>(p + k) : -__ldg(b + row);
#pragma unroll
      for (int j = 0; j < R2P; ++j)
        if (j < r2) {
          const float m = SMEM_M ? sMg[k * r2 + j] : c_M[k * r2 + j];
          acc[j] = (k == 0) ? xk * m : fmaf(xk, m, acc[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < R2P; ++j) acc[j] = j < r2 ? fabsf(acc[j]) : INFINITY;
    float med;
    {
      // lower median of the first r2 entries: the padded +inf entries sort last, so the
      // ((r2−1)/2)-th order statistic of all R2P values is the wanted one.
      constexpr int P = R2P;
      float a[P];
#pragma unroll
      for (int i = 0; i < P; ++i) a[i] = acc[i];
      sort_net<P>(a);
      const int mid = (r2 - 1) / 2;
      med = a[0];
#pragma unroll
      for (int i = 0; i < P; ++i)
        if (i == mid) med = a[i];
    }
    lam[row] = med;
    two_sum_add(s, c, med);
  }
  const double tot = block_pair_total(s, c);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// OptimizedFastCauchyRegression (p̂_i = min{1, s·λ̂_i}, no Σλ): λ̂ and the Bernoulli keep
// decision in one pass, so λ̂ never leaves registers (it is written only when the caller
// asked for it).  Blocks own contiguous chunks of rows (multiples of 64) as in the
// separate sampling pass, and produce the same keep mask and per-block counts for the
// ordered compaction.  A warp handles 64 consecutive rows per step: lane l computes λ̂
// of rows base+l and base+32+l (coalesced row loads, next step's rows in flight), then
// the uniforms move by shuffles from the lane that drew them (one Philox call per row pair).
struct LamMarkArgs {
  const void* A;
  int64_t lda;
  const float* b;
  int64_t n;
  int64_t chunk;           // rows per block, multiple of 64
  const float* mg;         // M (FP32, q × r2) in global memory (SMEM_M)
  float* lam_out;          // optional λ̂ output
  Key2 key;
  uint32_t problem;
  int64_t row_offset;
  double tau;              // s of the figure (sample_scale)
  uint64_t* mask;
  int64_t* counts;
  StatusBlock* status;
};

template <int D, typename TA, bool VEC>
__device__ __forceinline__ void load_x(const LamMarkArgs& a, int64_t row, int64_t stop, float (&x)[D + 1]) {
  if (row < stop) {
    load_row<D, TA, VEC>(static_cast<const TA*>(a.A) + row * a.lda, x);
    x[D] = -__ldg(a.b + row);
  } else {
#pragma unroll
    for (int k = 0; k <= D; ++k) x[k] = 0.f;
  }
}

template <int D, int R2, typename TA, bool VEC, bool SMEM_M>
__global__ void __launch_bounds__(kLamThreads) lambda_mark_kernel(const LamMarkArgs a) {
  constexpr int Q = D + 1;
  __shared__ __align__(16) float sM[SMEM_M ? Q * R2 : 1];
  __shared__ int64_t wcount[kLamThreads / 32];
  if constexpr (SMEM_M) {
    for (int e = threadIdx.x; e < Q * R2; e += blockDim.x) sM[e] = a.mg[e];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t start = static_cast<int64_t>(blockIdx.x) * a.chunk;
  const int64_t stop = min(a.n, start + a.chunk);
  const double tau = a.tau;
  const float tau32 = tau > static_cast<double>(FLT_MAX) ? FLT_MAX : static_cast<float>(tau);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.status->tau = tau;
    a.status->tau32 = tau32;
  }
  const int64_t stride = 64 * static_cast<int64_t>(nwarps);
  int64_t kept = 0;
  int64_t base = start + 64 * warp;
  float nx[Q];
  if (base < stop) load_x<D, TA, VEC>(a, base + lane, stop, nx);
  for (; base < stop; base += stride) {           // uniform across the warp
    // Row base + j (j < 64) takes its uniforms from Philox call ⌊(g + j)/2⌋, g the global
    // id of row base, word pair (g + j) mod 2; lane l draws call ⌊g/2⌋ + l, and call
    // ⌊g/2⌋ + 32 is needed too when g is odd.
    const uint64_t g = static_cast<uint64_t>(a.row_offset + base);
    const int off0 = static_cast<int>(g & 1);
    const uint4 o = draw_row(a.key, (g >> 1) + lane, a.problem, kStreamSample);
    uint4 o32 = make_uint4(0u, 0u, 0u, 0u);
    if (off0) o32 = draw_row(a.key, (g >> 1) + 32, a.problem, kStreamSample);
    uint32_t bal0 = 0, bal1 = 0;
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {
      float x[Q];
#pragma unroll
      for (int k = 0; k < Q; ++k) x[k] = nx[k];
      const int64_t row = base + 32 * t + lane;
      load_x<D, TA, VEC>(a, t == 0 ? row + 32 : base + stride + lane, stop, nx);   // next row in flight
      const float lam = lambda_of_row<Q, R2, SMEM_M>(x, sM);
      if (a.lam_out && row < stop) a.lam_out[row] = lam;
      const int j = 32 * t + lane;
      const int src = ((off0 + j) >> 1) & 31;
      const bool hi = ((off0 + j) & 1) != 0;
      const uint32_t sx = __shfl_sync(0xffffffffu, o.x, src), sy = __shfl_sync(0xffffffffu, o.y, src);
      const uint32_t sz = __shfl_sync(0xffffffffu, o.z, src), sw = __shfl_sync(0xffffffffu, o.w, src);
      uint32_t wa = hi ? sz : sx, wb = hi ? sw : sy;
      if (off0 + j == 64) {
        wa = o32.x;
        wb = o32.y;
      }
      const uint32_t bt = __ballot_sync(0xffffffffu, row < stop && keep_row(lam, tau32, tau, wa, wb));
      if (t == 0) bal0 = bt;
      else bal1 = bt;
    }
    const uint64_t m = static_cast<uint64_t>(bal0) | (static_cast<uint64_t>(bal1) << 32);
    if (lane == 0) a.mask[base >> 6] = m;
    kept += __popcll(m);
  }
  if (lane == 0) wcount[warp] = kept;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < nwarps; ++w) t += wcount[w];
    a.counts[blockIdx.x] = t;
  }
}

// ----------------------------------------------------------------- dispatch
template <int DD, int RR, typename TA, bool SM>
static void launch_lambda_case(dim3 grid, dim3 block, cudaStream_t st, bool aligned, const TA* A, int64_t lda,
                               const float* b, int64_t n, float* lam, double* sums, const float* mg) {
  if constexpr ((DD * sizeof(TA)) % 16 == 0) {
    if (aligned) {
      lambda_kernel<DD, RR, TA, true, SM><<<grid, block, 0, st>>>(A, lda, b, n, lam, sums, mg);
      return;
    }
  }
  lambda_kernel<DD, RR, TA, false, SM><<<grid, block, 0, st>>>(A, lda, b, n, lam, sums, mg);
}

// The padded kernel's D for FP32 rows of d columns with no kernel of their own: the
// smallest D ≥ d among the padded instantiations for this r2 (0: none, use the generic kernel).
static bool lambda_has_case(int d, int r2) {
  static const int cases[][2] = {{4, 8}, {8, 8}, {16, 8}, {32, 8}, {4, 16}, {8, 16}, {16, 16},
                                 {32, 16}, {64, 16}, {8, 32}, {16, 32}, {32, 32}, {64, 32}};
  for (const auto& c : cases)
    if (c[0] == d && c[1] == r2) return true;
  return false;
}

static int lambda_pad_target(int d, int r2) {
  if (lambda_has_case(d, r2)) return 0;
  static const int pads[][2] = {{8, 8}, {16, 8}, {32, 8}, {8, 16}, {16, 16}, {32, 16}, {64, 16},
                                {16, 32}, {32, 32}, {64, 32}};
  for (const auto& c : pads)
    if (c[1] == r2 && c[0] >= d) return c[0];
  return 0;
}

// M (FP32, q × r2) into this translation unit's constant bank: rows 0..d−1, then (for the
// padded kernel of width D) zero rows d..D−1 and M's b row as row D.
static bool load_const_m(const float* m32, int d, int r2, int pad, cudaStream_t st) {
  const size_t row = sizeof(float) * r2;
  if (!pad)
    return cuda_ok(cudaMemcpyToSymbolAsync(c_M, m32, row * (d + 1), 0, cudaMemcpyDeviceToDevice, st),
                   "copy M to constant memory");
  void* cm = nullptr;
  return cuda_ok(cudaGetSymbolAddress(&cm, c_M), "constant M address") &&
         cuda_ok(cudaMemcpyToSymbolAsync(c_M, m32, row * d, 0, cudaMemcpyDeviceToDevice, st),
                 "copy M to constant memory") &&
         cuda_ok(cudaMemsetAsync(static_cast<char*>(cm) + row * d, 0, row * (pad - d), st), "zero padded M rows") &&
         cuda_ok(cudaMemcpyToSymbolAsync(c_M, m32 + static_cast<size_t>(d) * r2, row, row * pad,
                                         cudaMemcpyDeviceToDevice, st),
                 "copy M's b row");
}

template <typename TA, bool SM>
static bool launch_lambda_t(const Plan& pl, const TA* A, int64_t lda, const float* b, float* lam,
                            double* sums, const float* mg, cudaStream_t st) {
  if constexpr (!SM) {
    const int pad = sizeof(TA) == 4 ? lambda_pad_target(pl.d, pl.r2) : 0;
    if (!load_const_m(mg, pl.d, pl.r2, pad, st)) return false;
  }
  const dim3 grid(pl.lam_ctas), block(pl.lam_threads);
  const size_t esz = sizeof(TA);
  const bool aligned = (reinterpret_cast<uintptr_t>(A) % 16 == 0) && ((lda * esz) % 16 == 0);
  const int d = pl.d, r2 = pl.r2;
#define L1S_LAMBDA_CASE(DD, RR)                                                               \
  if (d == DD && r2 == RR) {                                                                  \
    launch_lambda_case<DD, RR, TA, SM>(grid, block, st, aligned, A, lda, b, pl.n, lam, sums, mg); \
    count_launch(1);                                                                          \
    return cuda_ok(cudaGetLastError(), "launch lambda");                                      \
  }
  L1S_LAMBDA_CASE(4, 8)
  L1S_LAMBDA_CASE(8, 8)
  L1S_LAMBDA_CASE(16, 8)
  L1S_LAMBDA_CASE(32, 8)
  L1S_LAMBDA_CASE(4, 16)
  L1S_LAMBDA_CASE(8, 16)
  L1S_LAMBDA_CASE(16, 16)
  L1S_LAMBDA_CASE(32, 16)
  L1S_LAMBDA_CASE(64, 16)
  L1S_LAMBDA_CASE(8, 32)
  L1S_LAMBDA_CASE(16, 32)
  L1S_LAMBDA_CASE(32, 32)
  L1S_LAMBDA_CASE(64, 32)
#undef L1S_LAMBDA_CASE
  if constexpr (sizeof(TA) == 4) {
    const int D = lambda_pad_target(d, r2);
#define L1S_LAMBDA_PAD(DD, RR)                                                                         \
  if (D == DD && r2 == RR) {                                                                           \
    lambda_kernel_pad<DD, RR, SM><<<grid, block, 0, st>>>(reinterpret_cast<const float*>(A), lda, d, b, \
                                                         pl.n, lam, sums, mg);                          \
    count_launch(1);                                                                                   \
    return cuda_ok(cudaGetLastError(), "launch lambda (padded)");                                      \
  }
    L1S_LAMBDA_PAD(8, 8)
    L1S_LAMBDA_PAD(16, 8)
    L1S_LAMBDA_PAD(32, 8)
    L1S_LAMBDA_PAD(8, 16)
    L1S_LAMBDA_PAD(16, 16)
    L1S_LAMBDA_PAD(32, 16)
    L1S_LAMBDA_PAD(64, 16)
    L1S_LAMBDA_PAD(16, 32)
    L1S_LAMBDA_PAD(32, 32)
    L1S_LAMBDA_PAD(64, 32)
#undef L1S_LAMBDA_PAD
  }
  const size_t gsm = SM ? sizeof(float) * (d + 1) * r2 : 0;
  if (r2 <= 16)
    lambda_kernel_generic<16, TA, SM><<<grid, block, gsm, st>>>(A, lda, b, pl.n, d, r2, lam, sums, mg);
  else if (r2 <= 32)
    lambda_kernel_generic<32, TA, SM><<<grid, block, gsm, st>>>(A, lda, b, pl.n, d, r2, lam, sums, mg);
  else
    lambda_kernel_generic<64, TA, SM><<<grid, block, gsm, st>>>(A, lda, b, pl.n, d, r2, lam, sums, mg);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch lambda (generic)");
}

template <int DD, int RR, typename TA, bool SM>
static void launch_lambda_mark_case(int grid, cudaStream_t st, bool aligned, const LamMarkArgs& a) {
  if constexpr ((DD * sizeof(TA)) % 16 == 0) {
    if (aligned) {
      lambda_mark_kernel<DD, RR, TA, true, SM><<<grid, kLamThreads, 0, st>>>(a);
      return;
    }
  }
  lambda_mark_kernel<DD, RR, TA, false, SM><<<grid, kLamThreads, 0, st>>>(a);
}

}  // namespace l1s
