// Phase 3 (Figure 2, steps 6-7; ℓ1 sampling lemma, §2):
//   p̂_i = min(1, τ·λ_i) with τ = m_s/Σλ (FP64),  D_ii = 1/p̂_i if u_i < p̂_i else 0.
//
// mark:    each block owns a contiguous chunk of rows (a multiple of 64).  For
//          row i the 53-bit uniform comes from Philox stream 2 (one call serves
//          two rows).  The comparison u_i < p̂_i is decided exactly in FP64, but
//          FP64 arithmetic is slow on this part, so an FP32 pre-test settles
//          almost every row: p̂ is known to ~2^-22 relative from τ32·λ and u to
//          2^-24 from its top 24 bits, and only rows inside that margin are
//          re-decided in FP64.  Decisions become a 64-bit mask per 64 rows; the
//          block's kept count is written out.
// compact: each block adds the counts of the blocks before it (fixed order),
//          scans its mask words, and writes kept rows in ascending order:
//          index, weight 1/p̂_i, and the FP64 row [A_i, −b_i] of the coreset.
#include <algorithm>

#include "l1s_common.cuh"

namespace l1s {

constexpr int kSmpThreads = 256;
static_assert(kSmpThreads == 256, "lambda_total_256 assumes blocks of 256 threads");

struct MarkArgs {
  const float* lam;      // λ (mode 0) — or nullptr
  const double* p;       // caller's p̂ (mode 1) — or nullptr
  int64_t n;
  int64_t chunk;         // rows per block, multiple of 64
  Key2 key;
  uint32_t problem;
  int64_t row_offset;
  const StatusBlock* status;
  uint64_t* mask;        // ⌈n/64⌉ words
  int64_t* counts;       // per block
  int lam_pairs;         // 1: λ is 8-byte aligned, read two rows per load
  const double* lam_sums;  // λ block partials when this kernel forms Σλ and τ itself (else null)
  int nsums;
  double coreset;        // m_s
  double tau_fixed;      // > 0: p̂ = min(1, tau_fixed·λ) without Σλ (OptimizedFastCauchyRegression)
  StatusBlock* status_rw;
};

constexpr int kMarkUnroll = 4;

__global__ void __launch_bounds__(kSmpThreads) sample_mark_kernel(const MarkArgs a) {
  __shared__ int64_t wcount[kSmpThreads / 32];
  __shared__ double wsum[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t start = static_cast<int64_t>(blockIdx.x) * a.chunk;
  const int64_t stop = min(a.n, start + a.chunk);
  double tau = 0.0;
  float tau32 = 0.f;
  if (a.tau_fixed > 0.0) {
    tau = a.tau_fixed;
    tau32 = tau > static_cast<double>(FLT_MAX) ? FLT_MAX : static_cast<float>(tau);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.status_rw->tau = tau;
      a.status_rw->tau32 = tau32;
    }
  } else if (a.lam_sums) {
    // Σλ over the λ block partials (the same fixed order as the finalize kernel) and
    // τ = m_s/Σλ, formed by every block; block 0 records them in the status block.
    const double tot = lambda_total_256(a.lam_sums, a.nsums, wsum);
    const bool ok = tau_of(tot, a.coreset, &tau, &tau32);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.status_rw->lambda_total = tot;
      a.status_rw->tau = tau;
      a.status_rw->tau32 = tau32;
      if (!ok) raise_flag(&a.status_rw->flags, L1S_ERR_ZERO_MASS);
    }
  } else if (!a.p) {
    tau = a.status->tau;
    tau32 = a.status->tau32;
  }
  const bool odd_offset = (a.row_offset & 1) != 0;
  const int64_t stride = 64 * static_cast<int64_t>(nwarps);
  int64_t kept = 0;
  // Each warp covers 64 consecutive rows per step (two per lane); kMarkUnroll steps are
  // loaded before any is decided so that several loads are in flight per warp.
  for (int64_t base0 = start + 64 * warp; base0 < stop; base0 += stride * kMarkUnroll) {
    float l0[kMarkUnroll], l1[kMarkUnroll];
    double p0[kMarkUnroll], p1[kMarkUnroll];
#pragma unroll
    for (int u = 0; u < kMarkUnroll; ++u) {
      const int64_t r0 = base0 + u * stride + 2 * lane;
      l0[u] = l1[u] = 0.f;
      p0[u] = p1[u] = 0.0;
      if (a.p) {
        if (r0 < stop) p0[u] = a.p[r0];
        if (r0 + 1 < stop) p1[u] = a.p[r0 + 1];
      } else if (a.lam_pairs && r0 + 1 < stop) {
        const float2 v = *reinterpret_cast<const float2*>(a.lam + r0);
        l0[u] = v.x;
        l1[u] = v.y;
      } else {
        if (r0 < stop) l0[u] = a.lam[r0];
        if (r0 + 1 < stop) l1[u] = a.lam[r0 + 1];
      }
    }
    // The kMarkUnroll Philox calls are independent: compute them together (ILP), then decide.
    uint32_t w0a[kMarkUnroll], w0b[kMarkUnroll], w1a[kMarkUnroll], w1b[kMarkUnroll];
#pragma unroll
    for (int u = 0; u < kMarkUnroll; ++u) {
      const int64_t r0 = base0 + u * stride + 2 * lane;
      const uint64_t g0 = static_cast<uint64_t>(a.row_offset + r0);
      if (!odd_offset) {
        const uint4 o = draw_row(a.key, g0 >> 1, a.problem, kStreamSample);
        w0a[u] = o.x; w0b[u] = o.y; w1a[u] = o.z; w1b[u] = o.w;
      } else {
        const uint4 o0 = draw_row(a.key, g0 >> 1, a.problem, kStreamSample);
        const uint4 o1 = draw_row(a.key, (g0 + 1) >> 1, a.problem, kStreamSample);
        w0a[u] = o0.z; w0b[u] = o0.w; w1a[u] = o1.x; w1b[u] = o1.y;
      }
    }
#pragma unroll
    for (int u = 0; u < kMarkUnroll; ++u) {
      const int64_t base = base0 + u * stride;
      if (base >= stop) break;                 // uniform across the warp
      const int64_t r0 = base + 2 * lane;      // this lane's two rows: r0, r0 + 1
      bool k0 = false, k1 = false;
      if (a.p) {
        if (r0 < stop) k0 = static_cast<double>(u53_of(w0a[u], w0b[u])) * 0x1p-53 < p0[u];
        if (r0 + 1 < stop) k1 = static_cast<double>(u53_of(w1a[u], w1b[u])) * 0x1p-53 < p1[u];
      } else {
        if (r0 < stop) k0 = keep_row(l0[u], tau32, tau, w0a[u], w0b[u]);
        if (r0 + 1 < stop) k1 = keep_row(l1[u], tau32, tau, w1a[u], w1b[u]);
      }
      const uint32_t be = __ballot_sync(0xffffffffu, k0);
      const uint32_t bo = __ballot_sync(0xffffffffu, k1);
      const uint64_t m = spread_bits(be) | (spread_bits(bo) << 1);
      if (lane == 0) a.mask[base >> 6] = m;
      kept += __popcll(m);
    }
  }
  if (lane == 0) wcount[warp] = kept;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < nwarps; ++w) t += wcount[w];
    a.counts[blockIdx.x] = t;
  }
}

template <typename TA>
struct CompactArgs {
  const uint64_t* mask;
  const int64_t* counts;
  int nblocks;
  int64_t n, chunk, capacity;
  const float* lam;           // λ for the weights; null: recomputed from the kept row and M
  const float* m32;           // M (FP32, q × r2) when lam is null
  int r2;
  const StatusBlock* status;
  const TA* A;
  int64_t lda;
  const float* b;
  int d;
  int neg_lo, neg_hi;         // coreset columns written negated (multiple regression: X = [A, −B])
  int64_t* idx;
  double* w;                  // may be null
  double* coreset;            // may be null
  int64_t* count_out;         // may be null
  StatusBlock* status_rw;
  // Several coresets from one λ (blockIdx.y = coreset j): mask words, block counts and
  // outputs of coreset j start j·mask_stride words, j·counts_stride counts, j·capacity
  // rows and j counts further on.
  int64_t mask_stride = 0;
  int64_t counts_stride = 0;
};

// λ of one row with the operation order of the λ kernels (x_0·M_0j, then FMAs over k in
// order, |·|, the ((r2−1)/2)-th order statistic), so the value is bit-identical to the one
// the keep decision used.  R2C = r2 (8 or 16) at compile time, M in shared memory.
template <typename TA, int R2C>
__device__ __forceinline__ float lambda_recompute(const CompactArgs<TA>& a, const float* __restrict__ sM,
                                                  int64_t row) {
  float acc[R2C];
  const TA* src = a.A + row * a.lda;
  const int q = a.d + 1;
  {
    const float x0 = load_elem<TA>(src);
#pragma unroll
    for (int j = 0; j < R2C; ++j) acc[j] = x0 * sM[j];
  }
  for (int k = 1; k < q; ++k) {
    const float xk = k < a.d ? load_elem<TA>(src + k) : -a.b[row];
#pragma unroll
    for (int j = 0; j < R2C; ++j) acc[j] = fmaf(xk, sM[k * R2C + j], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < R2C; ++j) acc[j] = fabsf(acc[j]);
  constexpr int mid = (R2C - 1) / 2;
  float med = acc[0];
#pragma unroll
  for (int i = 0; i < R2C; ++i) {
    int lt = 0, le = 0;
#pragma unroll
    for (int j = 0; j < R2C; ++j) {
      lt += acc[j] < acc[i];
      le += acc[j] <= acc[i];
    }
    if (lt <= mid && mid < le) med = acc[i];
  }
  return med;
}

// Maximum q of the λ recomputation (the fused λ-and-mark pass serves d ≤ 32).
constexpr int kRecomputeMaxQ = 33;

template <typename TA, int R2C>
__global__ void __launch_bounds__(kSmpThreads) sample_compact_kernel(const CompactArgs<TA> a) {
  constexpr int kWarps = kSmpThreads / 32;
  __shared__ int64_t s_warp[kWarps];
  __shared__ int64_t s_base;
  __shared__ float sM[R2C > 0 ? kRecomputeMaxQ * R2C : 1];
  if constexpr (R2C > 0)
    for (int e = threadIdx.x; e < (a.d + 1) * R2C; e += blockDim.x) sM[e] = a.m32[e];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t cj = blockIdx.y;
  const int q = a.d + 1;
  const uint64_t* mask = a.mask + cj * a.mask_stride;
  const int64_t* counts = a.counts + cj * a.counts_stride;
  int64_t* idx = a.idx ? a.idx + cj * a.capacity : nullptr;
  double* wout = a.w ? a.w + cj * a.capacity : nullptr;
  double* cset = a.coreset ? a.coreset + cj * a.capacity * q : nullptr;
  // Offset of this block: Σ counts of the blocks before it (per-thread sums, then warp
  // shuffles and the warp totals in a fixed order).
  int64_t pre = 0;
  for (int i = tid; i < static_cast<int>(blockIdx.x); i += blockDim.x) pre += counts[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
  if (lane == 0) s_warp[warp] = pre;
  __syncthreads();
  if (tid == 0) {
    int64_t t = 0;
    for (int w = 0; w < kWarps; ++w) t += s_warp[w];
    s_base = t;
    if (blockIdx.x == gridDim.x - 1) {
      const int64_t total = t + counts[blockIdx.x];
      if (a.count_out) a.count_out[cj] = total;
      if (cj == 0) a.status_rw->count = total;
      if (total > a.capacity) raise_flag(&a.status_rw->flags, L1S_ERR_CAPACITY);
    }
  }
  __syncthreads();
  int64_t base = s_base;
  const int64_t start = static_cast<int64_t>(blockIdx.x) * a.chunk;
  const int64_t stop = min(a.n, start + a.chunk);
  const int64_t w0 = start >> 6, w1 = (stop + 63) >> 6;
  const double tau = a.status->tau;
  for (int64_t tile = w0; tile < w1; tile += blockDim.x) {
    const int64_t wi = tile + tid;
    const uint64_t m = wi < w1 ? mask[wi] : 0ull;
    const int64_t c = __popcll(m);
    // inclusive scan of c over the block: within warps by shuffles, then over warp totals
    int64_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    __syncthreads();                                  // s_warp free from the previous tile
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int64_t woff = 0, tile_total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const int64_t v = s_warp[w];
      woff += w < warp ? v : 0;
      tile_total += v;
    }
    int64_t pos = base + woff + incl - c;
    uint64_t bits = m;
    while (bits) {
      const int bit = __ffsll(static_cast<long long>(bits)) - 1;
      bits &= bits - 1;
      const int64_t row = (wi << 6) + bit;
      if (pos < a.capacity) {
        idx[pos] = row;
        if (wout) {
          float lam;
          if constexpr (R2C > 0) lam = lambda_recompute<TA, R2C>(a, sM, row);
          else lam = a.lam[row];
          wout[pos] = 1.0 / p_hat(tau, lam);
        }
        if (cset) {
          double* out = cset + pos * q;
          const TA* src = a.A + row * a.lda;
          for (int k = 0; k < a.d; ++k) {
            const double v = static_cast<double>(load_elem<TA>(src + k));
            out[k] = (k >= a.neg_lo && k < a.neg_hi) ? -v : v;
          }
          out[a.d] = -static_cast<double>(a.b[row]);
        }
      }
      ++pos;
    }
    base += tile_total;
  }
}

int sample_threads() { return kSmpThreads; }

bool launch_compact(const Plan& pl, const float* lam, const float* m32, const void* A, int64_t lda, l1s_dtype dt,
                    const float* b, int64_t capacity, int64_t* idx, double* w, double* coreset, int64_t* count_out,
                    unsigned char* ws, cudaStream_t st);

bool launch_sample(const Plan& pl, const float* lam, const double* p, const l1s_params* prm,
                   const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t capacity,
                   int64_t* idx, double* w, double* coreset, int64_t* count_out, unsigned char* ws,
                   cudaStream_t st, int lam_nsums) {
  MarkArgs m;
  m.lam = lam;
  m.p = p;
  m.n = pl.n;
  m.chunk = pl.smp_chunk;
  m.key = make_key(prm->seed);
  m.problem = prm->problem_id;
  m.row_offset = prm->global_row_offset;
  m.status = reinterpret_cast<const StatusBlock*>(ws + pl.off_status);
  m.mask = reinterpret_cast<uint64_t*>(ws + pl.off_mask);
  m.counts = reinterpret_cast<int64_t*>(ws + pl.off_counts);
  m.lam_pairs = (reinterpret_cast<uintptr_t>(lam) % 8 == 0) ? 1 : 0;
  m.lam_sums = lam_nsums > 0 ? reinterpret_cast<const double*>(ws + pl.off_lamsum) : nullptr;
  m.nsums = lam_nsums;
  m.coreset = prm->coreset_size;
  m.tau_fixed = (lam && prm->variant == 1) ? prm->sample_scale : 0.0;
  m.status_rw = reinterpret_cast<StatusBlock*>(ws + pl.off_status);
  sample_mark_kernel<<<pl.smp_ctas, pl.smp_threads, 0, st>>>(m);
  count_launch(1);
  if (!cuda_ok(cudaGetLastError(), "launch sample_mark")) return false;
  return launch_compact(pl, lam, nullptr, A, lda, dt, b, capacity, idx, w, coreset, count_out, ws, st);
}

// Ordered compaction of k keep masks (weights from λ, or from λ recomputed with M).
static bool launch_compact_many(const Plan& pl, const float* lam, const float* m32, const void* A, int64_t lda,
                                l1s_dtype dt, const float* b, int64_t capacity, int64_t* idx, double* w,
                                double* coreset, int64_t* count_out, unsigned char* ws, int k, const uint64_t* mask,
                                int64_t mask_stride, const int64_t* counts, int64_t counts_stride,
                                cudaStream_t st) {
  StatusBlock* sb = reinterpret_cast<StatusBlock*>(ws + pl.off_status);
  const dim3 grid(pl.smp_ctas, k);
  // Weights without λ: λ recomputed from M (r2 ∈ {8, 16} and q ≤ kRecomputeMaxQ only).
  const int r2c = (lam || !w) ? 0 : pl.r2;
  if (r2c && (!m32 || (r2c != 8 && r2c != 16) || pl.q > kRecomputeMaxQ))
    return set_error("compaction: no λ and no recomputation for r2 = %d, q = %d", pl.r2, pl.q), false;
  if (dt == L1S_BF16) {
    CompactArgs<uint16_t> c{mask, counts, pl.smp_ctas, pl.n, pl.smp_chunk, capacity, lam, m32, pl.r2, sb,
                            static_cast<const uint16_t*>(A), lda, b, pl.d, pl.pi2_neg_lo, pl.pi2_neg_hi, idx, w,
                            coreset, count_out, sb, mask_stride, counts_stride};
    if (r2c == 8) sample_compact_kernel<uint16_t, 8><<<grid, pl.smp_threads, 0, st>>>(c);
    else if (r2c == 16) sample_compact_kernel<uint16_t, 16><<<grid, pl.smp_threads, 0, st>>>(c);
    else sample_compact_kernel<uint16_t, 0><<<grid, pl.smp_threads, 0, st>>>(c);
  } else {
    CompactArgs<float> c{mask, counts, pl.smp_ctas, pl.n, pl.smp_chunk, capacity, lam, m32, pl.r2, sb,
                         static_cast<const float*>(A), lda, b, pl.d, pl.pi2_neg_lo, pl.pi2_neg_hi, idx, w, coreset,
                         count_out, sb, mask_stride, counts_stride};
    if (r2c == 8) sample_compact_kernel<float, 8><<<grid, pl.smp_threads, 0, st>>>(c);
    else if (r2c == 16) sample_compact_kernel<float, 16><<<grid, pl.smp_threads, 0, st>>>(c);
    else sample_compact_kernel<float, 0><<<grid, pl.smp_threads, 0, st>>>(c);
  }
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch sample_compact");
}

bool launch_compact(const Plan& pl, const float* lam, const float* m32, const void* A, int64_t lda, l1s_dtype dt,
                    const float* b, int64_t capacity, int64_t* idx, double* w, double* coreset, int64_t* count_out,
                    unsigned char* ws, cudaStream_t st) {
  return launch_compact_many(pl, lam, m32, A, lda, dt, b, capacity, idx, w, coreset, count_out, ws, 1,
                             reinterpret_cast<const uint64_t*>(ws + pl.off_mask), 0,
                             reinterpret_cast<const int64_t*>(ws + pl.off_counts), 0, st);
}

// ----------------------------------------------------------------- k coresets from one λ
// Figure 2, steps 6-7 from a caller-given λ and Σλ, k times over: coreset j keeps row i
// iff u_i^(j) < p̂_i with p̂_i = min(1, τ·λ_i), τ = m_s/Σλ, and u^(j) the sampling uniforms
// of problem id problem_id + j.  Σλ is read from device memory, so it may be a sum over
// row shards (the one scalar a sharded problem exchanges before sampling); coreset j is
// then the j-th call of l1_sample's sampling step with that Σλ.  Each warp reads the λ of
// 64 rows once and decides them for all k coresets (four coresets' Philox calls at a
// time), writing mask word j·words + ⌊i/64⌋ and adding to the block's count of coreset j.
struct MarkManyArgs {
  const float* lam;
  int64_t n, chunk;
  Key2 key;
  uint32_t problem;
  int64_t row_offset;
  int k;
  const double* lam_total;   // Σλ (device); null: τ = tau_fixed
  double coreset;            // m_s
  double tau_fixed;          // OptimizedFastCauchyRegression: p̂ = min(1, s·λ̂)
  uint64_t* mask;            // [k][mask_stride]
  int64_t mask_stride;
  int64_t* counts;           // [k][gridDim.x]
  StatusBlock* status;
  int lam_pairs;
};

constexpr int kManyUnroll = 4;

__global__ void __launch_bounds__(kSmpThreads) sample_mark_many_kernel(const MarkManyArgs a) {
  __shared__ unsigned int s_cnt[kMaxCoresets];
  for (int j = threadIdx.x; j < a.k; j += blockDim.x) s_cnt[j] = 0u;
  double tau;
  float tau32;
  bool ok = true;
  double tot = 0.0;
  if (a.lam_total) {
    tot = *a.lam_total;
    ok = tau_of(tot, a.coreset, &tau, &tau32);
  } else {
    tau = a.tau_fixed;
    tau32 = tau > static_cast<double>(FLT_MAX) ? FLT_MAX : static_cast<float>(tau);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.status->lambda_total = tot;
    a.status->tau = tau;
    a.status->tau32 = tau32;
    if (!ok) raise_flag(&a.status->flags, L1S_ERR_ZERO_MASS);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t start = static_cast<int64_t>(blockIdx.x) * a.chunk;
  const int64_t stop = min(a.n, start + a.chunk);
  const bool odd_offset = (a.row_offset & 1) != 0;
  for (int64_t base = start + 64 * warp; base < stop; base += 64 * static_cast<int64_t>(nwarps)) {
    const int64_t r0 = base + 2 * lane;
    float l0 = 0.f, l1 = 0.f;
    if (a.lam_pairs && r0 + 1 < stop) {
      const float2 v = *reinterpret_cast<const float2*>(a.lam + r0);
      l0 = v.x;
      l1 = v.y;
    } else {
      if (r0 < stop) l0 = a.lam[r0];
      if (r0 + 1 < stop) l1 = a.lam[r0 + 1];
    }
    const uint64_t g0 = static_cast<uint64_t>(a.row_offset + r0);
    for (int j0 = 0; j0 < a.k; j0 += kManyUnroll) {
      uint32_t w0a[kManyUnroll], w0b[kManyUnroll], w1a[kManyUnroll], w1b[kManyUnroll];
#pragma unroll
      for (int u = 0; u < kManyUnroll; ++u) {
        const uint32_t prob = a.problem + static_cast<uint32_t>(j0 + u);
        if (!odd_offset) {
          const uint4 o = draw_row(a.key, g0 >> 1, prob, kStreamSample);
          w0a[u] = o.x; w0b[u] = o.y; w1a[u] = o.z; w1b[u] = o.w;
        } else {
          const uint4 o0 = draw_row(a.key, g0 >> 1, prob, kStreamSample);
          const uint4 o1 = draw_row(a.key, (g0 + 1) >> 1, prob, kStreamSample);
          w0a[u] = o0.z; w0b[u] = o0.w; w1a[u] = o1.x; w1b[u] = o1.y;
        }
      }
#pragma unroll
      for (int u = 0; u < kManyUnroll; ++u) {
        const int j = j0 + u;
        if (j >= a.k) break;                   // uniform across the block
        const bool k0 = r0 < stop && keep_row(l0, tau32, tau, w0a[u], w0b[u]);
        const bool k1 = r0 + 1 < stop && keep_row(l1, tau32, tau, w1a[u], w1b[u]);
        const uint32_t be = __ballot_sync(0xffffffffu, k0);
        const uint32_t bo = __ballot_sync(0xffffffffu, k1);
        if (lane == 0) {
          const uint64_t m = spread_bits(be) | (spread_bits(bo) << 1);
          a.mask[j * a.mask_stride + (base >> 6)] = m;
          if (m) atomicAdd(&s_cnt[j], static_cast<unsigned int>(__popcll(m)));
        }
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < a.k; j += blockDim.x)
    a.counts[static_cast<int64_t>(j) * gridDim.x + blockIdx.x] = static_cast<int64_t>(s_cnt[j]);
}

// Bytes past the plan's workspace that k > 1 coresets need (masks and block counts).
size_t sample_many_extra_bytes(const Plan& pl, int k) {
  if (k <= 1) return 0;
  const size_t words = static_cast<size_t>((pl.n + 63) / 64);
  return align_up(sizeof(uint64_t) * words * k) + align_up(sizeof(int64_t) * static_cast<size_t>(pl.smp_ctas) * k);
}

bool launch_sample_many(const Plan& pl, const float* lam, const double* lam_total, const l1s_params* prm, int k,
                        const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t capacity, int64_t* idx,
                        double* w, double* coreset, int64_t* count_out, unsigned char* ws, cudaStream_t st) {
  MarkManyArgs m;
  m.lam = lam;
  m.n = pl.n;
  m.chunk = pl.smp_chunk;
  m.key = make_key(prm->seed);
  m.problem = prm->problem_id;
  m.row_offset = prm->global_row_offset;
  m.k = k;
  m.lam_total = prm->variant == 1 ? nullptr : lam_total;
  m.coreset = prm->coreset_size;
  m.tau_fixed = prm->variant == 1 ? prm->sample_scale : 0.0;
  m.status = reinterpret_cast<StatusBlock*>(ws + pl.off_status);
  m.lam_pairs = (reinterpret_cast<uintptr_t>(lam) % 8 == 0) ? 1 : 0;
  const size_t words = static_cast<size_t>((pl.n + 63) / 64);
  if (k == 1) {
    m.mask = reinterpret_cast<uint64_t*>(ws + pl.off_mask);
    m.counts = reinterpret_cast<int64_t*>(ws + pl.off_counts);
  } else {
    m.mask = reinterpret_cast<uint64_t*>(ws + pl.total);
    m.counts = reinterpret_cast<int64_t*>(ws + pl.total + align_up(sizeof(uint64_t) * words * k));
  }
  m.mask_stride = static_cast<int64_t>(words);
  sample_mark_many_kernel<<<pl.smp_ctas, pl.smp_threads, 0, st>>>(m);
  count_launch(1);
  if (!cuda_ok(cudaGetLastError(), "launch sample_mark_many")) return false;
  return launch_compact_many(pl, lam, nullptr, A, lda, dt, b, capacity, idx, w, coreset, count_out, ws, k, m.mask,
                             m.mask_stride, m.counts, pl.smp_ctas, st);
}

// ----------------------------------------------------------------- with replacement
// params.variant = 2 (the alternative the caption of Figure 2 allows): exactly m draws
// t = 0 … m−1, draw t takes the row i with C_{i−1} ≤ u_t·Σλ < C_i, C the running FP64 sum
// of λ, and weight 1/(m·p̂_i) = Σλ/(m·λ_i).  C is formed over contiguous chunks of
// pl.smp_chunk rows: one launch sums every chunk, a second adds each chunk's offset (the
// sums of the chunks before it, in order) to its running sum and writes C; both run the
// same per-chunk arithmetic (16 consecutive rows per thread, a warp-shuffle scan, a scan
// of the warp totals by one warp).  C is non-decreasing up to FP64 rounding at thread boundaries.
constexpr int kScanPer = 16;

// s_warp holds 2·(warps) + 1 doubles: the warp totals, their exclusive scan, the tile total.
template <bool WRITE>
__device__ double chunk_scan(const float* __restrict__ lam, int64_t start, int64_t stop, double offset,
                             double* __restrict__ cdf, double* s_warp) {
  constexpr int kWarps = kSmpThreads / 32;
  static_assert(kWarps <= 32, "one warp scans the warp totals");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double carry = 0.0;                                   // the same in every thread
  for (int64_t base = start; base < stop; base += static_cast<int64_t>(kSmpThreads) * kScanPer) {
    const int64_t r0 = base + static_cast<int64_t>(tid) * kScanPer;
    double loc[kScanPer];
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      acc += (r0 + k < stop) ? static_cast<double>(lam[r0 + k]) : 0.0;
      loc[k] = acc;
    }
    double incl = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    __syncthreads();                                    // s_warp free from the previous tile
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {                                    // exclusive scan of the warp totals
      double v = lane < kWarps ? s_warp[lane] : 0.0;
#pragma unroll
      for (int o = 1; o < kWarps; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      const double e = __shfl_up_sync(0xffffffffu, v, 1);
      if (lane < kWarps) s_warp[kWarps + lane] = lane == 0 ? 0.0 : e;
      if (lane == kWarps - 1) s_warp[2 * kWarps] = v;
    }
    __syncthreads();
    const double woff = s_warp[kWarps + warp], tile_total = s_warp[2 * kWarps];
    if constexpr (WRITE) {
      const double t0 = offset + (carry + (woff + excl));
#pragma unroll
      for (int k = 0; k < kScanPer; ++k)
        if (r0 + k < stop) cdf[r0 + k] = t0 + loc[k];
    }
    carry += tile_total;
  }
  return carry;
}

__global__ void __launch_bounds__(kSmpThreads) cdf_total_kernel(const float* __restrict__ lam, int64_t n,
                                                                int64_t chunk, double* __restrict__ totals) {
  __shared__ double s_warp[2 * (kSmpThreads / 32) + 1];
  const int64_t start = static_cast<int64_t>(blockIdx.x) * chunk;
  const double t = chunk_scan<false>(lam, start, min(n, start + chunk), 0.0, nullptr, s_warp);
  if (threadIdx.x == 0) totals[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kSmpThreads) cdf_write_kernel(const float* __restrict__ lam, int64_t n,
                                                                int64_t chunk, const double* __restrict__ totals,
                                                                double* __restrict__ cdf) {
  __shared__ double s_warp[2 * (kSmpThreads / 32) + 1];
  __shared__ double s_off;
  // This chunk's offset: every block runs the same exclusive scan of the chunk sums
  // (a run of consecutive sums per thread, then a warp-shuffle scan and the warp totals
  // in order) and keeps its own entry, so all blocks agree on every offset.
  {
    const int nb = static_cast<int>(gridDim.x);
    const int per = (nb + kSmpThreads - 1) / kSmpThreads;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k0 = tid * per;
    double acc = 0.0;
    for (int k = k0; k < min(nb, k0 + per); ++k) acc += totals[k];
    double incl = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    double woff = 0.0;
    for (int w = 0; w < warp; ++w) woff += s_warp[w];
    const int kb = static_cast<int>(blockIdx.x);
    if (kb >= k0 && kb < k0 + per) {
      double off = woff + excl;
      for (int k = k0; k < kb; ++k) off += totals[k];
      s_off = off;
    }
    __syncthreads();
  }
  const int64_t start = static_cast<int64_t>(blockIdx.x) * chunk;
  chunk_scan<true>(lam, start, min(n, start + chunk), s_off, cdf, s_warp);
}

template <typename TA>
struct DrawArgs {
  const float* lam;
  const double* cdf;
  int64_t n;
  int64_t m;             // draws
  Key2 key;
  uint32_t problem;
  const TA* A;
  int64_t lda;
  const float* b;
  int d;
  int64_t capacity;
  int64_t* idx;
  double* w;             // may be null
  double* coreset;       // may be null
  int64_t* count_out;    // may be null
  StatusBlock* status;
};

template <typename TA>
__global__ void __launch_bounds__(kSmpThreads) replacement_draw_kernel(const DrawArgs<TA> a) {
  const double total = a.cdf[a.n - 1];
  const bool ok = total > 0.0 && isfinite(total);
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t == 0) {
    a.status->lambda_total = total;
    a.status->count = a.m;
    if (a.count_out) *a.count_out = a.m;
    if (!ok) raise_flag(&a.status->flags, L1S_ERR_ZERO_MASS);
    if (a.m > a.capacity) raise_flag(&a.status->flags, L1S_ERR_CAPACITY);
  }
  if (!ok || t >= a.m || t >= a.capacity) return;
  const uint4 o = draw_row(a.key, static_cast<uint64_t>(t) >> 1, a.problem, kStreamReplace);
  const bool odd = (t & 1) != 0;
  const double u = static_cast<double>(u53_of(odd ? o.z : o.x, odd ? o.w : o.y)) * 0x1p-53;
  const double target = u * total;
  int64_t lo = 0, hi = a.n;                             // first i with C_i > target
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (a.cdf[mid] > target) hi = mid;
    else lo = mid + 1;
  }
  int64_t i = lo < a.n ? lo : a.n - 1;
  // A zero-mass row can only be met when u·Σλ rounds up to Σλ (no row then has C_i above
  // the target; a zero λ_i leaves C_i = C_{i−1} exactly): take the row at which C first
  // reaches C_i, the last row with mass (a binary search, no walk over the zero rows).
  if (!(a.lam[i] > 0.f)) {
    const double ci = a.cdf[i];
    int64_t l2 = 0, h2 = i;
    while (l2 < h2) {
      const int64_t mid = l2 + ((h2 - l2) >> 1);
      if (a.cdf[mid] >= ci) h2 = mid;
      else l2 = mid + 1;
    }
    i = l2;
  }
  a.idx[t] = i;
  const float li = a.lam[i];
  if (a.w) a.w[t] = li > 0.f ? total / (static_cast<double>(a.m) * static_cast<double>(li)) : 0.0;
  if (a.coreset) {
    double* out = a.coreset + t * (a.d + 1);
    const TA* src = a.A + i * a.lda;
    for (int k = 0; k < a.d; ++k) out[k] = static_cast<double>(load_elem<TA>(src + k));
    out[a.d] = -static_cast<double>(a.b[i]);
  }
}

bool launch_replacement(const Plan& pl, const float* lam, const l1s_params* prm, const void* A, int64_t lda,
                        l1s_dtype dt, const float* b, int64_t capacity, int64_t* idx, double* w, double* coreset,
                        int64_t* count_out, unsigned char* ws, cudaStream_t st) {
  double* totals = reinterpret_cast<double*>(ws + pl.off_counts);
  double* cdf = reinterpret_cast<double*>(ws + pl.off_cdf);
  cdf_total_kernel<<<pl.smp_ctas, kSmpThreads, 0, st>>>(lam, pl.n, pl.smp_chunk, totals);
  cdf_write_kernel<<<pl.smp_ctas, kSmpThreads, 0, st>>>(lam, pl.n, pl.smp_chunk, totals, cdf);
  count_launch(2);
  if (!cuda_ok(cudaGetLastError(), "launch cdf")) return false;
  const int64_t m = static_cast<int64_t>(prm->coreset_size);
  const int64_t draws = std::min(m, capacity);
  const int blocks = static_cast<int>(std::max<int64_t>(1, (draws + kSmpThreads - 1) / kSmpThreads));
  StatusBlock* sb = reinterpret_cast<StatusBlock*>(ws + pl.off_status);
  if (dt == L1S_BF16) {
    DrawArgs<uint16_t> a{lam, cdf, pl.n, m, make_key(prm->seed), prm->problem_id, static_cast<const uint16_t*>(A),
                         lda, b, pl.d, capacity, idx, w, coreset, count_out, sb};
    replacement_draw_kernel<uint16_t><<<blocks, kSmpThreads, 0, st>>>(a);
  } else {
    DrawArgs<float> a{lam, cdf, pl.n, m, make_key(prm->seed), prm->problem_id, static_cast<const float*>(A),
                      lda, b, pl.d, capacity, idx, w, coreset, count_out, sb};
    replacement_draw_kernel<float><<<blocks, kSmpThreads, 0, st>>>(a);
  }
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch replacement draws");
}

// ----------------------------------------------------------------- bounded-wait check
// One thread waits on an mbarrier that nothing arrives at, with the given cycle limit,
// the same bounded wait the pipelined kernels use; when it gives up it raises the
// TIMEOUT status bit and the kernel returns normally.
__global__ void debug_wait_kernel(uint32_t* flags, long long max_cycles) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, max_cycles)) raise_flag(flags, L1S_ERR_TIMEOUT);
}

bool launch_debug_wait(uint32_t* flags, long long max_cycles, cudaStream_t st) {
  debug_wait_kernel<<<1, 32, 0, st>>>(flags, max_cycles);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch debug_wait");
}

// ----------------------------------------------------------------- debug draws
__global__ void debug_variates_kernel(Key2 key, uint32_t problem, uint32_t r1, int64_t row_start,
                                      int64_t count, int32_t* bh, int32_t* bi, int32_t* kh, int32_t* ki,
                                      float* ch, float* ci, int8_t* sg, uint64_t* ub) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const uint64_t g = static_cast<uint64_t>(row_start + t);
  const uint4 o = draw_row(key, g, problem, kStreamFct);
  if (bh) bh[t] = bucket_of(o.x, r1);
  if (bi) bi[t] = bucket_of(o.z, r1);
  if (kh) kh[t] = static_cast<int32_t>(o.y >> 8);
  if (ki) ki[t] = static_cast<int32_t>(o.w >> 8);
  if (ch) ch[t] = cauchy_f32(o.y >> 8);
  if (ci) ci[t] = cauchy_f32(o.w >> 8);
  if (sg) sg[t] = (o.w & 1u) ? -1 : 1;
  if (ub) {
    const uint4 s = draw_row(key, g >> 1, problem, kStreamSample);
    ub[t] = (g & 1) ? u53_of(s.z, s.w) : u53_of(s.x, s.y);
  }
}

bool launch_debug_variates(const l1s_params* p, int64_t row_start, int64_t count, int32_t* bh,
                           int32_t* bi, int32_t* kh, int32_t* ki, float* ch, float* ci, int8_t* sg,
                           uint64_t* ub, cudaStream_t st) {
  const int64_t blocks = (count + 255) / 256;
  debug_variates_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
      make_key(p->seed), p->problem_id, static_cast<uint32_t>(p->r1), row_start, count, bh, bi, kh, ki,
      ch, ci, sg, ub);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch debug_variates");
}

}  // namespace l1s
