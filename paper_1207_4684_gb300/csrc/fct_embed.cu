// Phase 1: the FCT1 embedding Π1·X = 4·B·C·H̃·D·X (§3.1, FCT1 construction;
// Figure 2, steps 1-2), X = [A, −b].
//
// Persistent thread blocks walk over s-row blocks β of X (grid stride); each
// thread block owns a slice of w columns of Π1X.  Per block β:
//   1. one Philox call per row gives the row's sign σ, the buckets of its two
//      virtual rows and their Cauchy scales (shared memory);
//   2. the s rows of A and b arrive in a shared-memory stage by TMA bulk copies
//      (cp.async.bulk, completion on an mbarrier) issued two blocks ahead, so
//      HBM traffic overlaps the arithmetic; a ragged last block, a padded lda
//      or an unaligned base are read with ordinary loads instead;
//   3. pass 1 reads the raw tile, applies σ, scatters the identity half of
//      G_s = [H_s; I_s] (P[h_I(i), c] += 4·c_I(i)·σ_i·x_ic), runs the first
//      ⌊log2 s / 2⌋ radix-2 butterfly stages in registers and stores the tile;
//   4. pass 2 runs the remaining stages and scatters the Hadamard half
//      (P[h_H(i), c] += 4·c_H(i)/√s·(H_s z)_ic) straight from registers.
// P, the block's r1 × w partial of Π1X, lives in shared memory (B's hashed sum
// is a shared-memory reduction, no global atomics).  A second kernel adds the
// per-block partials in a fixed order.
#include "l1s_common.cuh"

namespace l1s {

constexpr int kFctStages = 2;
constexpr int kFctMaxThreads = 512;

struct FctArgs {
  const void* A;
  int64_t lda;
  const float* b;
  int64_t n;
  int d, q, r1, width;
  int64_t nblocks;
  int64_t full_blocks;    // blocks with s valid rows
  int tma;                // 1: full blocks arrive by bulk copy
  uint32_t stage_a_bytes; // bytes of A in a stage (s·d·elem, multiple of 16 when tma)
  uint32_t stage_bytes;   // A part rounded up to 16 + s·4 for b
  Key2 key;
  uint32_t problem;
  int64_t row_offset;
  int sign_flip;
  int log2s;              // log2 s (the narrow-X kernel's tile may hold several H_s blocks)
  float inv_sqrt_s;
  float* partials;        // [slices][gridDim.x][r1][width]
  int accumulate;         // 1: add to the partials of an earlier launch over other rows
  int sd;                 // narrow-X kernel: row stride of a stage (d, or lda when padded rows are staged)
  uint32_t* flags;
};

struct RowMeta {          // draws of one input row
  int hI;
  float wI;               // 4·c_I
  int hH;
  float wH;               // 4·c_H/√s
};

template <typename TA>
__device__ __forceinline__ float widen(TA v) {
  if constexpr (sizeof(TA) == 4) return v;
  else return __uint_as_float(static_cast<uint32_t>(v) << 16);
}

// x_{row0+row, col} of X = [A, −b]: from the shared-memory stage (STAGED) or from global memory.
template <typename TA, bool STAGED>
__device__ __forceinline__ float x_value(const FctArgs& a, const unsigned char* stage, int64_t row0, int row,
                                         int col) {
  if constexpr (STAGED) {
    if (col < a.d) return widen<TA>(reinterpret_cast<const TA*>(stage)[row * a.d + col]);
    return -reinterpret_cast<const float*>(stage + ((a.stage_a_bytes + 15) & ~15u))[row];
  } else {
    const int64_t r = row0 + row;
    if (r >= a.n) return 0.f;
    if (col < a.d) return widen<TA>(__ldg(static_cast<const TA*>(a.A) + r * a.lda + col));
    return -__ldg(a.b + r);
  }
}

// Pass 1: bits [0, K) of the row index.  Reads the raw stage, signs, scatters the identity half.
template <int LOG2S, int K, bool LAST, typename TA, bool STAGED>
__device__ __forceinline__ void fwht_first(const FctArgs& a, const unsigned char* __restrict__ stage, int64_t row0,
                                           int c0, float* __restrict__ tile, float* __restrict__ part,
                                           const RowMeta* __restrict__ meta, const float* __restrict__ sg,
                                           int W, int wcols) {
  constexpr int G = 1 << K;
  const int ngroups = ((1 << LOG2S) >> K) * W;
  const int step = blockDim.x;
  int rest = threadIdx.x / W;
  int c = threadIdx.x - rest * W;
  const int drest = step / W, dc = step - drest * W;
  for (int g = threadIdx.x; g < ngroups; g += step) {
    const int base = rest << K;
    const bool live = c < wcols;
    float v[G];
#pragma unroll
    for (int j = 0; j < G; ++j) v[j] = live ? x_value<TA, STAGED>(a, stage, row0, base + j, c0 + c) : 0.f;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const int row = base + j;
      v[j] *= sg[row];
      if (live) atomicAdd(&part[meta[row].hI * W + c], meta[row].wI * v[j]);
    }
#pragma unroll
    for (int t = 0; t < K; ++t) {
#pragma unroll
      for (int j = 0; j < G; ++j) {
        if ((j & (1 << t)) == 0) {
          const float lo = v[j], hi = v[j | (1 << t)];
          v[j] = lo + hi;
          v[j | (1 << t)] = lo - hi;
        }
      }
    }
    if constexpr (LAST) {
      if (live) {
#pragma unroll
        for (int j = 0; j < G; ++j) atomicAdd(&part[meta[base + j].hH * W + c], meta[base + j].wH * v[j]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < G; ++j) tile[(base + j) * W + c] = v[j];
    }
    c += dc;
    rest += drest;
    if (c >= W) {
      c -= W;
      ++rest;
    }
  }
}

// Pass 2: bits [LO, LO+K) of the row index from the tile, then the Hadamard-half scatter.
template <int LOG2S, int K, int LO>
__device__ __forceinline__ void fwht_second(const float* __restrict__ tile, float* __restrict__ part,
                                            const RowMeta* __restrict__ meta, int W, int wcols) {
  constexpr int G = 1 << K;
  const int ngroups = ((1 << LOG2S) >> K) * W;
  const int step = blockDim.x;
  int rest = threadIdx.x / W;
  int c = threadIdx.x - rest * W;
  const int drest = step / W, dc = step - drest * W;
  for (int g = threadIdx.x; g < ngroups; g += step) {
    const int base = ((rest >> LO) << (LO + K)) | (rest & ((1 << LO) - 1));
    float v[G];
#pragma unroll
    for (int j = 0; j < G; ++j) v[j] = tile[(base + (j << LO)) * W + c];
#pragma unroll
    for (int t = 0; t < K; ++t) {
#pragma unroll
      for (int j = 0; j < G; ++j) {
        if ((j & (1 << t)) == 0) {
          const float lo = v[j], hi = v[j | (1 << t)];
          v[j] = lo + hi;
          v[j | (1 << t)] = lo - hi;
        }
      }
    }
    if (c < wcols) {
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const RowMeta m = meta[base + (j << LO)];
        atomicAdd(&part[m.hH * W + c], m.wH * v[j]);
      }
    }
    c += dc;
    rest += drest;
    if (c >= W) {
      c -= W;
      ++rest;
    }
  }
}

template <typename TA>
__device__ __forceinline__ void load_stage_plain(const FctArgs& a, int64_t row0, int S, unsigned char* stage) {
  TA* ra = reinterpret_cast<TA*>(stage);
  float* rb = reinterpret_cast<float*>(stage + ((a.stage_a_bytes + 15) & ~15u));
  const TA* A = static_cast<const TA*>(a.A);
  const int d = a.d;
  for (int e = threadIdx.x; e < S * d; e += blockDim.x) {
    const int i = e / d, c = e - i * d;
    const int64_t row = row0 + i;
    TA v = TA(0);
    if (row < a.n) v = A[row * a.lda + c];
    ra[e] = v;
  }
  for (int i = threadIdx.x; i < S; i += blockDim.x) {
    const int64_t row = row0 + i;
    rb[i] = row < a.n ? a.b[row] : 0.f;
  }
}

template <typename TA>
__device__ __forceinline__ void issue_stage_tma(const FctArgs& a, int64_t blk, int S, unsigned char* stage,
                                                uint64_t* bar) {
  const unsigned char* srcA = static_cast<const unsigned char*>(a.A) + static_cast<size_t>(blk) * a.stage_a_bytes;
  const float* srcB = a.b + static_cast<size_t>(blk) * S;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, a.stage_a_bytes + static_cast<uint32_t>(S) * 4u);
  bulk_copy_g2s(stage, srcA, a.stage_a_bytes, bar);
  bulk_copy_g2s(stage + ((a.stage_a_bytes + 15) & ~15u), srcB, static_cast<uint32_t>(S) * 4u, bar);
}

template <int LOG2S, typename TA, bool STAGED>
__global__ void __launch_bounds__(kFctMaxThreads) fct_embed_kernel(const FctArgs a) {
  constexpr int S = 1 << LOG2S;
  constexpr int K1 = LOG2S / 2;          // pass 1: bits [0, K1)
  constexpr int K2 = LOG2S - K1;         // pass 2: bits [K1, LOG2S)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t bars[kFctStages];
  __shared__ int s_timeout;
  const int W = a.width;
  const int c0 = blockIdx.y * W;
  const int wcols = min(W, a.q - c0);
  // layout: stages (STAGED only) | part | tile | meta | sg
  unsigned char* stages = smem_raw;
  float* part = reinterpret_cast<float*>(stages + (STAGED ? static_cast<size_t>(kFctStages) * a.stage_bytes : 0));
  float* tile = part + a.r1 * W;
  RowMeta* meta = reinterpret_cast<RowMeta*>(tile + S * W);
  float* sg = reinterpret_cast<float*>(meta + S);

  for (int i = threadIdx.x; i < a.r1 * W; i += blockDim.x) part[i] = 0.f;
  if (threadIdx.x == 0) {
    s_timeout = 0;
    for (int k = 0; k < kFctStages; ++k) mbar_init(&bars[k], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool tma = STAGED;
  if (threadIdx.x == 0 && tma) {
    for (int k = 0; k < kFctStages; ++k) {
      const int64_t blk = blockIdx.x + static_cast<int64_t>(k) * gridDim.x;
      if (blk < a.full_blocks) issue_stage_tma<TA>(a, blk, S, stages + static_cast<size_t>(k) * a.stage_bytes, &bars[k]);
    }
  }
  int64_t it = 0;
  for (int64_t blk = blockIdx.x; blk < a.nblocks; blk += gridDim.x, ++it) {
    const int64_t row0 = blk * S;
    const int st = static_cast<int>(it % kFctStages);
    unsigned char* stage = stages + static_cast<size_t>(st) * a.stage_bytes;
    for (int i = threadIdx.x; i < S; i += blockDim.x) {
      const uint64_t grow = static_cast<uint64_t>(a.row_offset + row0 + i);
      const uint4 o = draw_row(a.key, grow, a.problem, kStreamFct);
      RowMeta m;
      m.hH = bucket_of(o.x, a.r1);
      m.hI = bucket_of(o.z, a.r1);
      m.wH = 4.f * cauchy_f32(o.y >> 8) * a.inv_sqrt_s;
      m.wI = 4.f * cauchy_f32(o.w >> 8);
      meta[i] = m;
      sg[i] = (a.sign_flip && (o.w & 1u)) ? -1.f : 1.f;
    }
    if constexpr (STAGED) {
      if (blk < a.full_blocks) {
        const bool ok = mbar_wait_bounded(&bars[st], static_cast<uint32_t>((it / kFctStages) & 1), kWaitCycles);
        if (!ok) s_timeout = 1;
      } else {
        load_stage_plain<TA>(a, row0, S, stage);
      }
    }
    __syncthreads();
    if (s_timeout) break;
    if constexpr (LOG2S <= 1) {
      fwht_first<LOG2S, LOG2S, true, TA, STAGED>(a, stage, row0, c0, tile, part, meta, sg, W, wcols);
      __syncthreads();
      if (threadIdx.x == 0 && tma) {
        const int64_t nxt = blk + static_cast<int64_t>(kFctStages) * gridDim.x;
        if (nxt < a.full_blocks) issue_stage_tma<TA>(a, nxt, S, stage, &bars[st]);
      }
    } else {
      fwht_first<LOG2S, K1, false, TA, STAGED>(a, stage, row0, c0, tile, part, meta, sg, W, wcols);
      __syncthreads();
      if (threadIdx.x == 0 && tma) {
        const int64_t nxt = blk + static_cast<int64_t>(kFctStages) * gridDim.x;
        if (nxt < a.full_blocks) issue_stage_tma<TA>(a, nxt, S, stage, &bars[st]);
      }
      fwht_second<LOG2S, K2, K1>(tile, part, meta, W, wcols);
    }
    __syncthreads();
  }
  if (s_timeout) {
    // Drain the copies still in flight (bounded) before the block's shared memory is released.
    if (threadIdx.x == 0) {
      raise_flag(a.flags, L1S_ERR_TIMEOUT);
      for (int64_t k = 0; k < kFctStages; ++k) {
        const int64_t j = it + k;
        const int64_t blk = blockIdx.x + j * gridDim.x;
        if (tma && blk < a.full_blocks)
          mbar_wait_bounded(&bars[j % kFctStages], static_cast<uint32_t>((j / kFctStages) & 1), kWaitCycles);
      }
    }
    __syncthreads();
    return;
  }
  // Non-finite input shows up as a non-finite partial (checked in the reduction).
  float* out = a.partials + (static_cast<size_t>(blockIdx.y) * gridDim.x + blockIdx.x) * a.r1 * W;
  for (int i = threadIdx.x; i < a.r1 * W; i += blockDim.x) out[i] = (a.accumulate ? out[i] : 0.f) + part[i];
}

// ----------------------------------------------------------------- d ≤ 32, 32 ≤ s ≤ 512
// A dedicated kernel for narrow X, where the generic kernel is bound by shared-memory
// bank conflicts and per-element draw loads.  It is warp-specialised and software
// pipelined over the s-row blocks of a thread block.  W = 16 (d ≤ 16) is described
// below; W = 32 (16 < d ≤ 32) has 16 A warps whose lanes are the 32 columns of one row
// (pass 1 over row bits 0-3, pass 2 over bits 4 and up) and a single copy of P.
//  * 4 producer warps compute the draws of block i into one of two draw buffers while
//    the consumers work on block i−1, and one producer thread issues the TMA copy of
//    block i into one of two stages;
//  * 8 A warps: a half-warp owns one 16-column tile of one row group, and the two
//    half-warps of a warp always hold rows of opposite parity, so each shared-memory
//    access of a warp covers both bank halves once.  Pass 1 runs the butterflies over
//    row bits 1-4 (and scatters the identity half), pass 2 over bit 0 and bits 5 and up
//    (the stages of H_s commute).  In pass 2 the odd half-warp reads its rows in the
//    order j ^ 1, which negates its outputs at odd positions (H_s applied to a permuted
//    vector); the sign is undone in the scatter.  P is kept as two copies, one per
//    half-warp, at bank offsets 0 and 16, so a warp's hashed scatter never conflicts;
//    the copies are added when the partial is written out;
//  * 1 b warp: 32 rows per register slot; stages over row bits ≥ 5 in registers, over
//    bits 0-4 by shuffles; its own scatter array.
// Hand-offs use mbarriers (bounded waits; a timeout raises the TIMEOUT status bit and
// every role stops).  Draws of a row are packed as {PST·h_I with σ in bit 31, 4·c_I} and
// {PST·h_H, 4·c_H/√s} (8 bytes each); the butterflies run on packed FP32 pairs.
constexpr int kWsB = 1, kWsP = 4;
template <int W>
struct WsCfg {
  static constexpr int kA = W / 2;                              // A warps
  static constexpr int kThreads = 32 * (kA + kWsB + kWsP);      // 416 or 672
};

struct __align__(8) T16Meta {
  uint32_t offs;      // PST·h_I (first word of row h_I of P), | 2^31 when σ = −1
  float wI;           // 4·c_I (the identity term of row i is wI·z_i, z_i = σ_i·x_i)
};
struct __align__(8) T16MetaH {
  int offH;           // 32·h_H
  float wH;           // 4·c_H/√s
};

// LOG2S here is the tile: 2^LOG2S rows per pipeline step, which may hold several
// H_s blocks (s = 2^a.log2s ≤ tile): butterfly stages over row bits ≥ log2 s are skipped.
// LEAN (W = 16 only): one stage buffer (the next tile's copy overlaps pass 2, which no
// longer reads the stage) and one copy of P with rows padded to 17 words instead of two
// copies, so that three thread blocks fit an SM.
template <int LOG2S, typename TA, int W, bool EXACT, bool LEAN>
__global__ void __launch_bounds__(WsCfg<W>::kThreads, LEAN ? 3 : (W == 16 ? 2 : 1)) fct_embed_ws_kernel(const FctArgs a) {
  constexpr int kWsA = WsCfg<W>::kA;
  constexpr int PST = LEAN ? 17 : 32;         // words per bucket row of P
  constexpr int NSTAGE = LEAN ? 1 : 2;
  constexpr int S = 1 << LOG2S;
  const int lg = EXACT ? LOG2S : a.log2s;   // H_s acts on row bits [0, lg); EXACT: s is the tile
  constexpr int K2 = LOG2S - 4;          // pass 2: row bit 0 and bits [5, LOG2S)
  constexpr int G2 = 1 << K2;
  constexpr int KB = S / 32;             // b column: values per lane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // mbarriers: stage_full (TMA or producer), stage_free (A + b warps done with pass 1),
  // meta_full (producers), meta_free (A + b warps done with the block)
  __shared__ uint64_t stage_full[2], stage_free[2], meta_full[2], meta_free[2];
  __shared__ volatile int s_abort;
  const int r1 = a.r1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = a.d;
  const int sd = a.sd;                   // stage row stride
  unsigned char* stages = smem_raw;
  float* P = reinterpret_cast<float*>(stages + NSTAGE * static_cast<size_t>(a.stage_bytes));   // [r1][PST]
  float* Pb = P + ((r1 * PST + 3) & ~3);                                                           // [r1]
  float* tile = Pb + ((r1 + 3) & ~3);                                                              // [S][16]
  T16Meta* mI = reinterpret_cast<T16Meta*>(tile + S * W);                                          // [2][S]
  T16MetaH* mH = reinterpret_cast<T16MetaH*>(mI + 2 * S);                                          // [2][S]

  for (int i = tid; i < ((r1 * PST + 3) & ~3) + r1; i += blockDim.x) P[i] = 0.f;   // P and Pb
  if (tid == 0) {
    s_abort = 0;
    for (int k = 0; k < 2; ++k) {
      mbar_init(&stage_full[k], 1);
      mbar_init(&stage_free[k], kWsA + kWsB);
      mbar_init(&meta_full[k], 1);
      mbar_init(&meta_free[k], kWsA + kWsB);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const bool tma = a.tma != 0;
  const uint32_t b_off = (a.stage_a_bytes + 15) & ~15u;

  if (warp >= kWsA + kWsB) {
    // ---------------- producers: draws of block i and its stage
    const int pt = tid - 32 * (kWsA + kWsB);       // 0..127
    int64_t i = 0;
    for (int64_t blk = blockIdx.x; blk < a.nblocks; blk += gridDim.x, ++i) {
      const int buf = static_cast<int>(i & 1);
      const uint32_t use = static_cast<uint32_t>((i >> 1) & 1);
      const int sbuf = LEAN ? 0 : buf;                         // stage buffer and its phase parity
      const uint32_t suse = LEAN ? static_cast<uint32_t>(i & 1) : use;
      unsigned char* stage = stages + static_cast<size_t>(sbuf) * a.stage_bytes;
      const int64_t row0 = blk * S;
      const bool by_tma = tma && blk < a.full_blocks;
      // the stage is free once its previous tile finished pass 1, the draw buffer once
      // block i−2 is done with it
      if (pt == 0) {
        const bool ok = mbar_wait_bounded(&stage_free[sbuf], suse ^ 1u, kWaitCycles) &&
                        mbar_wait_bounded(&meta_free[buf], use ^ 1u, kWaitCycles);
        if (!ok) s_abort = 1;
        else if (by_tma) issue_stage_tma<TA>(a, blk, S, stage, &stage_full[sbuf]);
      }
      // one decision for all producers (a consumer may set s_abort at any moment)
      if (named_barrier_any(1, 32 * kWsP, s_abort != 0)) break;
      if (!by_tma) {
        // plain loads into the stage (ragged last block, or rows that are not contiguous):
        // producer warp w copies rows w, w + 4, …, its lanes the columns of a row
        TA* ra = reinterpret_cast<TA*>(stage);
        float* rb = reinterpret_cast<float*>(stage + b_off);
        const TA* A = static_cast<const TA*>(a.A);
        // (d ≤ 32; two rows per warp instruction when d ≤ 16), 16 loads in flight per
        // lane before any is stored
        const int pw = pt >> 5, pl = pt & 31;
        const int cw = d <= 16 ? 16 : 32;                 // lanes per row
        const int rpw = 32 / cw;                          // rows per warp instruction
        const int c = pl & (cw - 1), rr = pl / cw;
        constexpr int kBatch = 16;
        for (int t0 = 0; (pw + kWsP * t0) * rpw < S; t0 += kBatch) {
          TA v[kBatch];
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int r = (pw + kWsP * (t0 + u)) * rpw + rr;
            v[u] = (r < S && c < d && row0 + r < a.n) ? A[(row0 + r) * a.lda + c] : TA(0);
          }
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int r = (pw + kWsP * (t0 + u)) * rpw + rr;
            if (r < S && c < d) ra[r * sd + c] = v[u];
          }
        }
        for (int r = pt; r < S; r += 32 * kWsP) rb[r] = (row0 + r < a.n) ? a.b[row0 + r] : 0.f;
      }
      T16Meta* mi = mI + buf * S;
      T16MetaH* mh = mH + buf * S;
      for (int r = pt; r < S; r += 32 * kWsP) {
        const uint64_t grow = static_cast<uint64_t>(a.row_offset + row0 + r);
        const uint4 o = draw_row(a.key, grow, a.problem, kStreamFct);
        const bool neg = a.sign_flip && (o.w & 1u);
        T16Meta m;
        m.offs = static_cast<uint32_t>(PST * bucket_of(o.z, r1)) | (neg ? 0x80000000u : 0u);
        m.wI = 4.f * cauchy_f32(o.w >> 8);
        mi[r] = m;
        T16MetaH h;
        h.offH = PST * bucket_of(o.x, r1);
        h.wH = 4.f * cauchy_f32(o.y >> 8) * a.inv_sqrt_s;
        mh[r] = h;
      }
      named_barrier(1, 32 * kWsP);                  // all draws (and a plain stage) written
      if (pt == 0) {
        if (!by_tma) mbar_arrive(&stage_full[sbuf]);
        mbar_arrive(&meta_full[buf]);
      }
    }
  } else {
    // ---------------- consumers: 8 A warps and the b warp
    const bool is_b = warp == kWsA;
    int64_t i = 0;
    for (int64_t blk = blockIdx.x; blk < a.nblocks; blk += gridDim.x, ++i) {
      const int buf = static_cast<int>(i & 1);
      const uint32_t use = static_cast<uint32_t>((i >> 1) & 1);
      const int sbuf = LEAN ? 0 : buf;
      const uint32_t suse = LEAN ? static_cast<uint32_t>(i & 1) : use;
      bool ok = true;
      if (lane == 0)
        ok = mbar_wait_bounded(&meta_full[buf], use, kWaitCycles) &&
             mbar_wait_bounded(&stage_full[sbuf], suse, kWaitCycles);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      // all consumer warps take the same decision, so none is left waiting at a barrier
      if (named_barrier_any(3, 32 * (kWsA + kWsB), !ok || s_abort)) {
        s_abort = 1;
        break;
      }
      const unsigned char* stage = stages + static_cast<size_t>(sbuf) * a.stage_bytes;
      const TA* rawA = reinterpret_cast<const TA*>(stage);
      const float* rawB = reinterpret_cast<const float*>(stage + b_off);
      const T16Meta* mi = mI + buf * S;
      const T16MetaH* mh = mH + buf * S;
      if (!is_b) {
        // ---- pass 1 on A: 4 row bits in registers, identity scatter on the way in
        if constexpr (W == 32) {
          for (int task = tid; task < 2 * S; task += 32 * kWsA) {
            const int c = task & 31, g = task >> 5;
            const int base = g << 4;                            // row bits 0-3 vary
            const bool live = c < d;
            float* Pl = P + c;
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = live ? widen<TA>(rawA[(base | j) * sd + c]) : 0.f;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const T16Meta m = mi[base | j];
              const uint32_t sg = m.offs & 0x80000000u;
              v[j] = __uint_as_float(__float_as_uint(v[j]) ^ sg);   // z = σ·x
              if (live) atomicAdd(Pl + (m.offs ^ sg), m.wI * v[j]);
            }
            uint64_t p[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) p[k] = f2_pack(v[k], v[k + 8]);
            f2_butterflies<16>(p, f2_stage_mask(0, lg));         // row bits 0-3
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              float x, y;
              f2_unpack(p[k], x, y);
              tile[(base | k) * 32 + c] = x;
              tile[(base | (k + 8)) * 32 + c] = y;
            }
          }
        } else
        for (int task = tid; task < S; task += 32 * kWsA) {
          const int c = task & 15;
          const int g = task >> 4;
          const int hb = g & 1;
          const int base = (g & 1) | ((g >> 1) << 5);
          const bool live = c < d;
          float* Pl = P + (LEAN ? 0 : hb * 16) + c;
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = live ? widen<TA>(rawA[(base | (j << 1)) * sd + c]) : 0.f;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const T16Meta m = mi[base | (j << 1)];
            const uint32_t sg = m.offs & 0x80000000u;
            v[j] = __uint_as_float(__float_as_uint(v[j]) ^ sg);     // z = σ·x
            if (live) atomicAdd(Pl + (m.offs ^ sg), m.wI * v[j]);
          }
          uint64_t p[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) p[k] = f2_pack(v[k], v[k + 8]);
          f2_butterflies<16>(p, f2_stage_mask(1, lg));           // row bits 1-4
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            float x, y;
            f2_unpack(p[k], x, y);
            tile[(base | (k << 1)) * 16 + c] = x;
            tile[(base | ((k + 8) << 1)) * 16 + c] = y;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&stage_free[sbuf]);
        named_barrier(2, 32 * kWsA);                   // tile complete
        // ---- pass 2 on A: the remaining row bits, then the Hadamard scatter
        if constexpr (W == 32) {
          constexpr int K2 = LOG2S - 4;
          constexpr int G2 = 1 << K2;
          const int c = tid & 31, g2 = tid >> 5;               // g2 = row bits 0-3
          float v[G2];
#pragma unroll
          for (int j = 0; j < G2; ++j) v[j] = tile[(g2 | (j << 4)) * 32 + c];
          {
            uint64_t p[G2 / 2];
#pragma unroll
            for (int k = 0; k < G2 / 2; ++k) p[k] = f2_pack(v[k], v[k + G2 / 2]);
            f2_butterflies<G2>(p, f2_stage_mask(4, lg));         // row bits 4 and up
#pragma unroll
            for (int k = 0; k < G2 / 2; ++k) f2_unpack(p[k], v[k], v[k + G2 / 2]);
          }
          if (c < d) {
            float* Pl = P + c;
#pragma unroll
            for (int k = 0; k < G2; ++k) {
              const int2 h = *reinterpret_cast<const int2*>(&mh[g2 | (k << 4)]);
              atomicAdd(Pl + h.x, __int_as_float(h.y) * v[k]);
            }
          }
        } else {
          const int c = tid & 15;
          const int g2 = tid >> 4;
          const int hb = g2 & 1;
          float v[G2];
#pragma unroll
          for (int j = 0; j < G2; ++j) {
            const int jj = j ^ hb;
            v[j] = tile[((g2 << 1) | (jj & 1) | ((jj >> 1) << 5)) * 16 + c];
          }
          {
            uint64_t p[G2 / 2];
#pragma unroll
            for (int k = 0; k < G2 / 2; ++k) p[k] = f2_pack(v[k], v[k + G2 / 2]);
            f2_butterflies<G2>(p, f2_stage_mask(4, lg) | 1u);    // row bit 0, then bits 5 and up
#pragma unroll
            for (int k = 0; k < G2 / 2; ++k) f2_unpack(p[k], v[k], v[k + G2 / 2]);
          }
          if (c < d) {
            float* Pl = P + (LEAN ? 0 : hb * 16) + c;
            const float odd_sign = hb ? -1.f : 1.f;
#pragma unroll
            for (int k = 0; k < G2; ++k) {
              const int2 h = *reinterpret_cast<const int2*>(&mh[(g2 << 1) | (k & 1) | ((k >> 1) << 5)]);
              const float val = (k & 1) ? odd_sign * v[k] : v[k];
              atomicAdd(Pl + h.x, __int_as_float(h.y) * val);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&meta_free[buf]);
        named_barrier(2, 32 * kWsA);                   // tile free for the next block
      } else {
        // ---- the b column: one warp, all stages, both scatters
        float v[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const int row = lane + 32 * k;
          const T16Meta m = mi[row];
          const uint32_t sg = m.offs & 0x80000000u;
          v[k] = __uint_as_float(__float_as_uint(-rawB[row]) ^ sg);   // z = σ·x
          atomicAdd(&Pb[(m.offs ^ sg) / PST], m.wI * v[k]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&stage_free[sbuf]);
#pragma unroll
        for (int t = 0; (1 << t) < KB; ++t) {
          if (5 + t < lg) {                                     // row bit 5 + t
#pragma unroll
            for (int k = 0; k < KB; ++k) {
              if ((k & (1 << t)) == 0) {
                const float lo = v[k], hi = v[k | (1 << t)];
                v[k] = lo + hi;
                v[k | (1 << t)] = lo - hi;
              }
            }
          }
        }
#pragma unroll
        for (int t = 0; t < 5; ++t) {
          if (t < lg) {                                         // row bit t (uniform over the warp)
            const bool upper = (lane >> t) & 1;
#pragma unroll
            for (int k = 0; k < KB; ++k) {
              const float o = __shfl_xor_sync(0xffffffffu, v[k], 1 << t);
              v[k] = upper ? (o - v[k]) : (v[k] + o);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const int2 h = *reinterpret_cast<const int2*>(&mh[lane + 32 * k]);
          atomicAdd(&Pb[h.x / PST], __int_as_float(h.y) * v[k]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&meta_free[buf]);
      }
    }
  }
  __syncthreads();
  if (s_abort) {
    // Let copies still in flight land (a bounded pause) before shared memory is released.
    if (tid == 0) {
      raise_flag(a.flags, L1S_ERR_TIMEOUT);
      const long long t0 = clock64();
      while (clock64() - t0 < 20000000LL) {
      }
    }
    __syncthreads();
    return;
  }
  const int q = d + 1;
  float* out = a.partials + static_cast<size_t>(blockIdx.x) * r1 * q;
  for (int i = tid; i < r1 * q; i += blockDim.x) {
    const int h = i / q, c = i - h * q;
    const float v = c < d ? (LEAN ? P[h * PST + c] : (W == 16 ? P[h * 32 + c] + P[h * 32 + 16 + c] : P[h * 32 + c]))
                          : Pb[h];
    out[i] = (a.accumulate ? out[i] : 0.f) + v;
  }
}

// ----------------------------------------------------------------- bucket-sorted scatter
// d ≤ 32, 32 ≤ s ≤ 512.  Shared-memory float atomics run at a small fraction of the
// rate of plain loads and stores, so this kernel avoids them on A: the producers sort
// the 2s virtual rows of a block by bucket (a counting sort: one integer atomic per
// virtual row gives its rank, a scan gives the bucket offsets), and each consumer warp
// owns a contiguous range of buckets — split at bucket boundaries, so no two warps,
// and no two half-warps, ever touch the same row of P.  A warp walks its sorted
// entries, sums the scaled rows of one bucket in registers (lane = column) and adds
// the sum to P once per bucket with a plain read-modify-write.  Roles:
//  * 4 producer warps: the TMA copy (or plain loads) of block i into one of two stages,
//    the row draws, the sign mask (one ballot per 32 rows), the sort;
//  * W/2 A warps (8 for W = 16 columns per entry, 16 for W = 32): pass 1 (σ and the
//    butterflies over 4 row bits, in registers) and pass 2 (the remaining bits), both
//    through the tile, then the sorted scatter; the identity half reads the raw stage,
//    with σ folded into its weight;
//  * 1 b warp: the b column as in the narrow-X kernel (its own atomics on a 1-column P).
// W = 16: the two half-warps of a warp hold rows of opposite parity in both passes, as
// in the narrow-X kernel (its second pass reads in the order j ^ 1 and undoes the sign
// on the way back to the tile); in the scatter each half-warp takes one half of the
// warp's bucket range.
constexpr int kSrtP = 4;

template <int W>
struct SrtCfg {
  static constexpr int kA = W / 2;
  static constexpr int kThreads = 32 * (kA + 1 + kSrtP);
};

struct __align__(16) SrtBMeta {   // draws of one row for the b warp
  int hI;
  float wI;                       // 4·c_I·σ
  int hH;
  float wH;                       // 4·c_H/√s
};

__host__ __device__ constexpr int srt_cnt_len(int r1) { return (r1 + 4) & ~3; }   // r1 + 1 offsets, padded

template <int LOG2S, typename TA, int W>
__global__ void __launch_bounds__(SrtCfg<W>::kThreads) fct_embed_sorted_kernel(const FctArgs a) {
  constexpr int S = 1 << LOG2S;
  constexpr int NA = SrtCfg<W>::kA;
  constexpr int E = 2 * S;                 // entries (virtual rows) per block
  constexpr int KB = S / 32;               // b column: values per lane
  constexpr int SW = S / 32;               // sign-mask words per block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t stage_full[2], stage_free[2], meta_full[2], meta_free[2];
  __shared__ volatile int s_abort;
  __shared__ int s_wsum[kSrtP];
  const int r1 = a.r1, d = a.d;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rc = srt_cnt_len(r1);
  unsigned char* stages = smem_raw;
  float* P = reinterpret_cast<float*>(stages + 2 * static_cast<size_t>(a.stage_bytes));   // [r1][W]
  float* Pb = P + r1 * W;                                                                    // [r1]
  float* tile = Pb + ((r1 + 3) & ~3);                                                        // [S][W]
  uint2* ent = reinterpret_cast<uint2*>(tile + S * W);                                       // [2][E]
  int* cnt = reinterpret_cast<int*>(ent + 2 * E);                                            // [2][rc]
  SrtBMeta* bm = reinterpret_cast<SrtBMeta*>(cnt + 2 * rc);                                  // [2][S]
  uint32_t* smask = reinterpret_cast<uint32_t*>(bm + 2 * S);                                 // [2][SW]

  for (int i = tid; i < r1 * W + ((r1 + 3) & ~3); i += blockDim.x) P[i] = 0.f;   // P and Pb
  if (tid == 0) {
    s_abort = 0;
    for (int k = 0; k < 2; ++k) {
      mbar_init(&stage_full[k], 1);
      mbar_init(&stage_free[k], NA + 1);
      mbar_init(&meta_full[k], 1);
      mbar_init(&meta_free[k], NA + 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const bool tma = a.tma != 0;
  const uint32_t b_off = (a.stage_a_bytes + 15) & ~15u;

  if (warp > NA) {
    // ---------------- producers
    const int pt = tid - 32 * (NA + 1);            // 0..127
    constexpr int RP = (S + 32 * kSrtP - 1) / (32 * kSrtP);
    int64_t i = 0;
    for (int64_t blk = blockIdx.x; blk < a.nblocks; blk += gridDim.x, ++i) {
      const int buf = static_cast<int>(i & 1);
      const uint32_t use = static_cast<uint32_t>((i >> 1) & 1);
      unsigned char* stage = stages + static_cast<size_t>(buf) * a.stage_bytes;
      const int64_t row0 = blk * S;
      const bool by_tma = tma && blk < a.full_blocks;
      if (pt == 0) {
        const bool ok = mbar_wait_bounded(&stage_free[buf], use ^ 1u, kWaitCycles) &&
                        mbar_wait_bounded(&meta_free[buf], use ^ 1u, kWaitCycles);
        if (!ok) s_abort = 1;
        else if (by_tma) issue_stage_tma<TA>(a, blk, S, stage, &stage_full[buf]);
      }
      // one decision for all producers (a consumer may set s_abort at any moment)
      if (named_barrier_any(1, 32 * kSrtP, s_abort != 0)) break;
      if (!by_tma) {
        TA* ra = reinterpret_cast<TA*>(stage);
        float* rb = reinterpret_cast<float*>(stage + b_off);
        const TA* A = static_cast<const TA*>(a.A);
        for (int e = pt; e < S * d; e += 32 * kSrtP) {
          const int r = e / d, c = e - r * d;
          ra[e] = (row0 + r < a.n) ? A[(row0 + r) * a.lda + c] : TA(0);
        }
        for (int r = pt; r < S; r += 32 * kSrtP) rb[r] = (row0 + r < a.n) ? a.b[row0 + r] : 0.f;
      }
      int* cb = cnt + buf * rc;
      for (int h = pt; h < rc; h += 32 * kSrtP) cb[h] = 0;
      named_barrier(1, 32 * kSrtP);
      int hH[RP], hI[RP], rkH[RP], rkI[RP];
      float wH[RP], wI[RP];
#pragma unroll
      for (int k = 0; k < RP; ++k) {
        const int r = pt + 32 * kSrtP * k;
        bool neg = false;
        if (r < S) {
          const uint64_t grow = static_cast<uint64_t>(a.row_offset + row0 + r);
          const uint4 o = draw_row(a.key, grow, a.problem, kStreamFct);
          neg = a.sign_flip && (o.w & 1u);
          hI[k] = bucket_of(o.z, r1);
          const float ci = 4.f * cauchy_f32(o.w >> 8);
          wI[k] = neg ? -ci : ci;
          hH[k] = bucket_of(o.x, r1);
          wH[k] = 4.f * cauchy_f32(o.y >> 8) * a.inv_sqrt_s;
          rkH[k] = atomicAdd(&cb[hH[k]], 1);
          rkI[k] = atomicAdd(&cb[hI[k]], 1);
          bm[buf * S + r] = SrtBMeta{hI[k], wI[k], hH[k], wH[k]};
        }
        // rows r of a warp are 32 consecutive rows, all below S or all at or above it
        const unsigned m = __ballot_sync(0xffffffffu, neg);
        if (r < S && lane == 0) smask[buf * SW + (r >> 5)] = m;
      }
      named_barrier(1, 32 * kSrtP);
      // Exclusive scan of the counts over buckets 0..r1 (cb[r1] stays 0, so its offset is E).
      {
        const int per = (r1 + 1 + 32 * kSrtP - 1) / (32 * kSrtP);
        const int h0 = pt * per;
        int loc = 0;
        for (int j = 0; j < per; ++j)
          if (h0 + j <= r1) loc += cb[h0 + j];
        int incl = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        if (lane == 31) s_wsum[pt >> 5] = incl;
        named_barrier(1, 32 * kSrtP);
        int run = incl - loc;
        for (int w = 0; w < (pt >> 5); ++w) run += s_wsum[w];
        for (int j = 0; j < per; ++j) {
          const int h = h0 + j;
          if (h <= r1) {
            const int c = cb[h];
            cb[h] = run;
            run += c;
          }
        }
      }
      named_barrier(1, 32 * kSrtP);
      uint2* eb = ent + buf * E;
#pragma unroll
      for (int k = 0; k < RP; ++k) {
        const int r = pt + 32 * kSrtP * k;
        if (r < S) {
          eb[cb[hH[k]] + rkH[k]] = make_uint2((static_cast<uint32_t>(hH[k]) << 16) | 0x8000u | r,
                                              __float_as_uint(wH[k]));
          eb[cb[hI[k]] + rkI[k]] = make_uint2((static_cast<uint32_t>(hI[k]) << 16) | r, __float_as_uint(wI[k]));
        }
      }
      named_barrier(1, 32 * kSrtP);                  // entries, offsets, masks and a plain stage written
      if (pt == 0) {
        if (!by_tma) mbar_arrive(&stage_full[buf]);
        mbar_arrive(&meta_full[buf]);
      }
    }
  } else {
    // ---------------- consumers: NA A warps and the b warp
    const bool is_b = warp == NA;
    int64_t i = 0;
    for (int64_t blk = blockIdx.x; blk < a.nblocks; blk += gridDim.x, ++i) {
      const int buf = static_cast<int>(i & 1);
      const uint32_t use = static_cast<uint32_t>((i >> 1) & 1);
      bool ok = true;
      if (lane == 0)
        ok = mbar_wait_bounded(&meta_full[buf], use, kWaitCycles) && mbar_wait_bounded(&stage_full[buf], use, kWaitCycles);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (named_barrier_any(3, 32 * (NA + 1), !ok || s_abort)) {
        s_abort = 1;
        break;
      }
      const unsigned char* stage = stages + static_cast<size_t>(buf) * a.stage_bytes;
      const TA* rawA = reinterpret_cast<const TA*>(stage);
      const float* rawB = reinterpret_cast<const float*>(stage + b_off);
      const uint32_t* sm = smask + buf * SW;
      if (!is_b) {
        // ---- pass 1: σ, butterflies over 4 row bits
        if constexpr (W == 16) {
          for (int task = tid; task < S; task += 32 * NA) {
            const int c = task & 15, g = task >> 4;
            const int base = (g & 1) | ((g >> 1) << 5);       // row bits 1-4 vary in registers
            const bool live = c < d;
            const uint32_t mw = sm[base >> 5];
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int row = base | (j << 1);
              const float x = live ? widen<TA>(rawA[row * d + c]) : 0.f;
              v[j] = __uint_as_float(__float_as_uint(x) ^ (((mw >> (row & 31)) & 1u) << 31));
            }
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if ((j & (1 << t)) == 0) {
                  const float lo = v[j], hi = v[j | (1 << t)];
                  v[j] = lo + hi;
                  v[j | (1 << t)] = lo - hi;
                }
#pragma unroll
            for (int j = 0; j < 16; ++j) tile[(base | (j << 1)) * 16 + c] = v[j];
          }
        } else {
          for (int task = tid; task < 2 * S; task += 32 * NA) {
            const int c = task & 31, g = task >> 5;
            const int base = g << 4;                            // row bits 0-3 vary in registers
            const bool live = c < d;
            const uint32_t mw = sm[base >> 5];
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int row = base | j;
              const float x = live ? widen<TA>(rawA[row * d + c]) : 0.f;
              v[j] = __uint_as_float(__float_as_uint(x) ^ (((mw >> (row & 31)) & 1u) << 31));
            }
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if ((j & (1 << t)) == 0) {
                  const float lo = v[j], hi = v[j | (1 << t)];
                  v[j] = lo + hi;
                  v[j | (1 << t)] = lo - hi;
                }
#pragma unroll
            for (int j = 0; j < 16; ++j) tile[(base | j) * 32 + c] = v[j];
          }
        }
        named_barrier(2, 32 * NA);                    // tile holds pass 1
        // ---- pass 2: the remaining row bits
        {
          constexpr int K2 = LOG2S - 4;
          constexpr int G2 = 1 << K2;
          float v[G2];
          if constexpr (W == 16) {
            const int c = tid & 15, g2 = tid >> 4, hb = g2 & 1;   // g2 = row bits 1-4
            auto row2 = [&](int k) { return (g2 << 1) | (k & 1) | ((k >> 1) << 5); };
#pragma unroll
            for (int j = 0; j < G2; ++j) v[j] = tile[row2(j ^ hb) * 16 + c];
#pragma unroll
            for (int t = 0; t < K2; ++t)
#pragma unroll
              for (int j = 0; j < G2; ++j)
                if ((j & (1 << t)) == 0) {
                  const float lo = v[j], hi = v[j | (1 << t)];
                  v[j] = lo + hi;
                  v[j | (1 << t)] = lo - hi;
                }
            // The odd half-warp transformed its rows in the order j ^ 1, which negates its
            // outputs at odd positions; it writes output k = j ^ 1 at step j with the sign undone.
#pragma unroll
            for (int j = 0; j < G2; ++j) {
              const float val = hb ? ((j & 1) ? v[j ^ 1] : -v[j ^ 1]) : v[j];
              tile[row2(j ^ hb) * 16 + c] = val;
            }
          } else {
            const int c = tid & 31, g2 = tid >> 5;               // g2 = row bits 0-3
#pragma unroll
            for (int j = 0; j < G2; ++j) v[j] = tile[(g2 | (j << 4)) * 32 + c];
#pragma unroll
            for (int t = 0; t < K2; ++t)
#pragma unroll
              for (int j = 0; j < G2; ++j)
                if ((j & (1 << t)) == 0) {
                  const float lo = v[j], hi = v[j | (1 << t)];
                  v[j] = lo + hi;
                  v[j | (1 << t)] = lo - hi;
                }
#pragma unroll
            for (int j = 0; j < G2; ++j) tile[(g2 | (j << 4)) * 32 + c] = v[j];
          }
        }
        named_barrier(2, 32 * NA);                    // tile holds H_s·z
        // ---- sorted scatter over this warp's bucket range
        {
          const uint2* eb = ent + buf * E;
          const int* off = cnt + buf * rc;
          auto snap = [&](int e) { return e >= E ? E : off[eb[e].x >> 16]; };
          const int start = warp == 0 ? 0 : snap((warp * E) / NA);
          const int end = warp == NA - 1 ? E : snap(((warp + 1) * E) / NA);
          int lo = start, hi = end;
          if constexpr (W == 16) {
            const int mid = (start + end) >> 1;
            int M = end;
            if (mid < end) {
              const int h = eb[mid].x >> 16;
              M = off[h];
              if (M <= start) M = off[h + 1];
            }
            if (lane >> 4) lo = M;
            else hi = M;
          }
          const int c = lane & (W - 1);
          const bool live = c < d;
          const int cnt_mine = hi - lo;
          const int steps = W == 16 ? max(cnt_mine, __shfl_xor_sync(0xffffffffu, cnt_mine, 16)) : cnt_mine;
          float acc = 0.f;
          int cur = -1;
          for (int t = 0; t < steps; ++t) {
            if (t < cnt_mine) {
              const uint2 en = eb[lo + t];
              const int h = static_cast<int>(en.x >> 16);
              const int row = static_cast<int>(en.x & 0x7FFFu);
              float val = 0.f;
              if (live) val = (en.x & 0x8000u) ? tile[row * W + c] : widen<TA>(rawA[row * d + c]);
              if (h != cur) {
                if (cur >= 0 && live) P[cur * W + c] += acc;
                acc = 0.f;
                cur = h;
              }
              acc = fmaf(__uint_as_float(en.y), val, acc);
            }
          }
          if (cur >= 0 && live) P[cur * W + c] += acc;
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&stage_free[buf]);
          mbar_arrive(&meta_free[buf]);
        }
        named_barrier(2, 32 * NA);                    // tile free for the next block
      } else {
        // ---- the b column: one warp, all stages, both scatters (atomics on Pb)
        const SrtBMeta* mb = bm + buf * S;
        float v[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const int row = lane + 32 * k;
          const float x = -rawB[row];
          const SrtBMeta m = mb[row];
          atomicAdd(&Pb[m.hI], m.wI * x);
          v[k] = __uint_as_float(__float_as_uint(x) ^ (((sm[k] >> lane) & 1u) << 31));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&stage_free[buf]);
#pragma unroll
        for (int t = 0; (1 << t) < KB; ++t)
#pragma unroll
          for (int k = 0; k < KB; ++k)
            if ((k & (1 << t)) == 0) {
              const float lo = v[k], hi = v[k | (1 << t)];
              v[k] = lo + hi;
              v[k | (1 << t)] = lo - hi;
            }
#pragma unroll
        for (int t = 0; t < 5; ++t) {
          const bool upper = (lane >> t) & 1;
#pragma unroll
          for (int k = 0; k < KB; ++k) {
            const float o = __shfl_xor_sync(0xffffffffu, v[k], 1 << t);
            v[k] = upper ? (o - v[k]) : (v[k] + o);
          }
        }
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const SrtBMeta m = mb[lane + 32 * k];
          atomicAdd(&Pb[m.hH], m.wH * v[k]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&meta_free[buf]);
      }
    }
  }
  __syncthreads();
  if (s_abort) {
    if (tid == 0) {
      raise_flag(a.flags, L1S_ERR_TIMEOUT);
      const long long t0 = clock64();
      while (clock64() - t0 < 20000000LL) {
      }
    }
    __syncthreads();
    return;
  }
  const int q = d + 1;
  float* out = a.partials + static_cast<size_t>(blockIdx.x) * r1 * q;
  for (int i = tid; i < r1 * q; i += blockDim.x) {
    const int h = i / q, c = i - h * q;
    out[i] = (a.accumulate ? out[i] : 0.f) + (c < d ? P[h * W + c] : Pb[h]);
  }
}

// Fixed-order sum of the per-block partials: PiX[r][c0+c] = Σ_blocks partial[r][c].
// Block = 32 warps; warp w adds partials w, w+32, …; warp 0 then adds the 32
// warp sums in order, so the result does not depend on scheduling.
// It also draws Π2 (q × r2 FP64, when pi2 is non-null), which depends on no data, so
// that the FP64 Cauchy transforms stay off the conditioning's serial path.
__global__ void __launch_bounds__(1024) fct_reduce_kernel(const float* __restrict__ partials, int ctas,
                                                          int r1, int W, int q, float* __restrict__ pix,
                                                          uint32_t* flags, Key2 key, uint32_t problem,
                                                          int npi2, int r2, int pi2_gauss, int neg_lo, int neg_hi,
                                                          double* __restrict__ pi2) {
  // Π2 rows [neg_lo, neg_hi) are stored negated: they pair with columns of X that the
  // passes read with the opposite sign (multiple regression), so that X·M is unchanged.
  if (pi2 && blockIdx.y == 0)
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < npi2; e += gridDim.x * blockDim.x) {
      const double v = pi2_value(key, problem, e, pi2_gauss);
      const int row = e / r2;
      pi2[e] = (row >= neg_lo && row < neg_hi) ? -v : v;
    }
  __shared__ float red[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int per = r1 * W;
  const int e = blockIdx.x * 32 + lane;
  float acc = 0.f;
  if (e < per) {
    const float* base = partials + static_cast<size_t>(blockIdx.y) * ctas * per + e;
    int c = warp;
    for (; c + 96 < ctas; c += 128) {
      const float v0 = base[static_cast<size_t>(c) * per];
      const float v1 = base[static_cast<size_t>(c + 32) * per];
      const float v2 = base[static_cast<size_t>(c + 64) * per];
      const float v3 = base[static_cast<size_t>(c + 96) * per];
      acc += v0;
      acc += v1;
      acc += v2;
      acc += v3;
    }
    for (; c < ctas; c += 32) acc += base[static_cast<size_t>(c) * per];
  }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && e < per) {
    float s = 0.f;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) s += red[k][lane];
    const int r = e / W, c = e - r * W;
    const int col = blockIdx.y * W + c;
    if (col < q) {
      pix[static_cast<size_t>(r) * q + col] = s;
      if (!isfinite(s)) raise_flag(flags, L1S_ERR_NONFINITE);
    }
  }
}

// ----------------------------------------------------------------- dispatch
template <typename TA, bool STAGED>
static const void* fct_kernel_for(int log2s) {
  switch (log2s) {
    case 0: return reinterpret_cast<const void*>(&fct_embed_kernel<0, TA, STAGED>);
    case 1: return reinterpret_cast<const void*>(&fct_embed_kernel<1, TA, STAGED>);
    case 2: return reinterpret_cast<const void*>(&fct_embed_kernel<2, TA, STAGED>);
    case 3: return reinterpret_cast<const void*>(&fct_embed_kernel<3, TA, STAGED>);
    case 4: return reinterpret_cast<const void*>(&fct_embed_kernel<4, TA, STAGED>);
    case 5: return reinterpret_cast<const void*>(&fct_embed_kernel<5, TA, STAGED>);
    case 6: return reinterpret_cast<const void*>(&fct_embed_kernel<6, TA, STAGED>);
    case 7: return reinterpret_cast<const void*>(&fct_embed_kernel<7, TA, STAGED>);
    case 8: return reinterpret_cast<const void*>(&fct_embed_kernel<8, TA, STAGED>);
    case 9: return reinterpret_cast<const void*>(&fct_embed_kernel<9, TA, STAGED>);
    case 10: return reinterpret_cast<const void*>(&fct_embed_kernel<10, TA, STAGED>);
    case 11: return reinterpret_cast<const void*>(&fct_embed_kernel<11, TA, STAGED>);
    case 12: return reinterpret_cast<const void*>(&fct_embed_kernel<12, TA, STAGED>);
    default: return nullptr;
  }
}

const void* fct_kernel(int log2s, l1s_dtype dt, bool staged) {
  if (dt == L1S_BF16) return staged ? fct_kernel_for<uint16_t, true>(log2s) : fct_kernel_for<uint16_t, false>(log2s);
  return staged ? fct_kernel_for<float, true>(log2s) : fct_kernel_for<float, false>(log2s);
}

template <typename TA, int W, bool LEAN>
static const void* ws_kernel_for(int log2t, bool exact) {
  switch (log2t) {
    case 8: return exact ? reinterpret_cast<const void*>(&fct_embed_ws_kernel<8, TA, W, true, LEAN>)
                         : reinterpret_cast<const void*>(&fct_embed_ws_kernel<8, TA, W, false, LEAN>);
    case 9: return exact ? reinterpret_cast<const void*>(&fct_embed_ws_kernel<9, TA, W, true, LEAN>)
                         : reinterpret_cast<const void*>(&fct_embed_ws_kernel<9, TA, W, false, LEAN>);
    default: return nullptr;
  }
}

// Column width of the narrow-X kernel for d (16 or 32; 2 ≤ s ≤ 512), 0 when it does not apply.
int fct_ws_width(int log2s, int d) {
  if (log2s < 1 || log2s > 9) return 0;
  return d <= 16 ? 16 : (d <= 32 ? 32 : 0);
}

// Its tile: at least 256 rows, so that blocks of small s share the per-tile pipeline costs.
int fct_ws_tile_log2(int log2s) { return log2s < 8 ? 8 : log2s; }

// The kernel for a tile of 2^log2t rows and blocks of 2^log2s rows (log2s ≤ log2t); lean
// (W = 16 only) selects the one-stage, one-copy form.
const void* fct_ws_kernel(int log2t, int log2s, l1s_dtype dt, int w, bool lean) {
  const bool exact = log2s == log2t;
  if (w == 16 && lean)
    return dt == L1S_BF16 ? ws_kernel_for<uint16_t, 16, true>(log2t, exact)
                          : ws_kernel_for<float, 16, true>(log2t, exact);
  if (w == 16)
    return dt == L1S_BF16 ? ws_kernel_for<uint16_t, 16, false>(log2t, exact)
                          : ws_kernel_for<float, 16, false>(log2t, exact);
  if (w == 32)
    return dt == L1S_BF16 ? ws_kernel_for<uint16_t, 32, false>(log2t, exact)
                          : ws_kernel_for<float, 32, false>(log2t, exact);
  return nullptr;
}

int fct_ws_threads(int w) { return w == 16 ? WsCfg<16>::kThreads : WsCfg<32>::kThreads; }

uint32_t fct_stage_bytes(int s, int d, l1s_dtype dt) {
  const uint32_t esz = dt == L1S_BF16 ? 2u : 4u;
  const uint32_t a_bytes = static_cast<uint32_t>(s) * d * esz;
  return ((a_bytes + 15u) & ~15u) + static_cast<uint32_t>(s) * 4u;
}

template <typename TA, int W>
static const void* sorted_kernel_for(int log2s) {
  switch (log2s) {
    case 5: return reinterpret_cast<const void*>(&fct_embed_sorted_kernel<5, TA, W>);
    case 6: return reinterpret_cast<const void*>(&fct_embed_sorted_kernel<6, TA, W>);
    case 7: return reinterpret_cast<const void*>(&fct_embed_sorted_kernel<7, TA, W>);
    case 8: return reinterpret_cast<const void*>(&fct_embed_sorted_kernel<8, TA, W>);
    case 9: return reinterpret_cast<const void*>(&fct_embed_sorted_kernel<9, TA, W>);
    default: return nullptr;
  }
}

// Column width of the bucket-sorted kernel for d (16 or 32), 0 when it does not apply.
int fct_sorted_width(int log2s, int d) {
  if (log2s < 5 || log2s > 9) return 0;
  return d <= 16 ? 16 : (d <= 32 ? 32 : 0);
}

const void* fct_sorted_kernel(int log2s, l1s_dtype dt, int w) {
  if (w == 16) return dt == L1S_BF16 ? sorted_kernel_for<uint16_t, 16>(log2s) : sorted_kernel_for<float, 16>(log2s);
  if (w == 32) return dt == L1S_BF16 ? sorted_kernel_for<uint16_t, 32>(log2s) : sorted_kernel_for<float, 32>(log2s);
  return nullptr;
}

int fct_sorted_threads(int w) { return w == 16 ? SrtCfg<16>::kThreads : SrtCfg<32>::kThreads; }

size_t fct_sorted_smem_bytes(int s, int d, l1s_dtype dt, int r1, int w) {
  return 2 * static_cast<size_t>(fct_stage_bytes(s, d, dt)) + static_cast<size_t>(r1) * w * 4 +
         static_cast<size_t>((r1 + 3) & ~3) * 4 + static_cast<size_t>(s) * w * 4 +
         2 * static_cast<size_t>(2 * s) * sizeof(uint2) + 2 * static_cast<size_t>(srt_cnt_len(r1)) * 4 +
         2 * static_cast<size_t>(s) * sizeof(SrtBMeta) + 2 * static_cast<size_t>(s / 32) * 4;
}


size_t fct_smem_bytes(int s, int d, l1s_dtype dt, int r1, int width, bool staged) {
  return (staged ? static_cast<size_t>(kFctStages) * fct_stage_bytes(s, d, dt) : 0) +
         static_cast<size_t>(r1) * width * 4 + static_cast<size_t>(s) * width * 4 +
         static_cast<size_t>(s) * (sizeof(RowMeta) + 4);
}

size_t fct_ws_smem_bytes(int s, int d, l1s_dtype dt, int r1, int w, bool lean) {
  const int pst = lean ? 17 : 32;
  return (lean ? 1 : 2) * static_cast<size_t>(fct_stage_bytes(s, d, dt)) +
         static_cast<size_t>((r1 * pst + 3) & ~3) * 4 +
         static_cast<size_t>((r1 + 3) & ~3) * 4 + static_cast<size_t>(s) * w * 4 +
         2 * static_cast<size_t>(s) * (sizeof(T16Meta) + sizeof(T16MetaH));
}

// TMA staging needs A's rows back to back (lda = d), 16-byte aligned bases and stage parts.
bool fct_can_stage(int s, int d, l1s_dtype dt, int64_t lda, const void* A, const float* b) {
  const uint32_t esz = dt == L1S_BF16 ? 2u : 4u;
  return lda == d && (reinterpret_cast<uintptr_t>(A) % 16 == 0) && (reinterpret_cast<uintptr_t>(b) % 16 == 0) &&
         ((static_cast<uint64_t>(s) * d * esz) % 16 == 0) && ((s * 4) % 16 == 0);
}

// Threads: enough for one butterfly group per (column, row group) of the larger pass.
int fct_threads_for(int log2s, int width) {
  const int k = log2s / 2;
  const int groups = std::max(((1 << log2s) >> k) * width, ((1 << log2s) >> (log2s - k)) * width);
  int t = (groups + 31) / 32 * 32;
  t = t < 256 ? 256 : t;
  return t > kFctMaxThreads ? kFctMaxThreads : t;
}

bool launch_fct_cols(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n,
                     int64_t row_offset, const l1s_params* p, bool accumulate, unsigned char* ws, cudaStream_t st);
bool launch_fct_cols_reduce(const Plan& pl, const l1s_params* p, float* pix, unsigned char* ws, cudaStream_t st,
                            double* pi2_out);
int fct_cols_tile();
bool launch_sct(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n,
                int64_t row_offset, const l1s_params* p, bool accumulate, unsigned char* ws, cudaStream_t st,
                float scale);
bool launch_fct2(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n,
                 int64_t row_offset, const l1s_params* p, bool accumulate, unsigned char* ws, cudaStream_t st);

// One phase-1 launch over rows [0, n) of A and b (device) whose global ids start at
// row_offset, writing the per-block partials at `partials`.
static bool launch_fct_part(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n,
                            int64_t row_offset, const l1s_params* p, bool accumulate, unsigned char* ws,
                            cudaStream_t st) {
  if (p->transform == 1)
    return launch_sct(pl, A, lda, dt, b, n, row_offset, p, accumulate, ws, st, static_cast<float>(4.0 / pl.r1));
  if (p->transform == 2) return launch_fct2(pl, A, lda, dt, b, n, row_offset, p, accumulate, ws, st);
  if (pl.fct_cols) return launch_fct_cols(pl, A, lda, dt, b, n, row_offset, p, accumulate, ws, st);
  FctArgs a;
  a.A = A;
  a.lda = lda;
  a.b = b;
  a.n = n;
  a.d = pl.d;
  a.q = pl.q;
  a.r1 = pl.r1;
  a.width = pl.fct_width;
  // The narrow-X kernel steps over tiles of 2^fct_tile_log2 ≥ s rows, the others over s-row blocks.
  const int tile = pl.fct_ws ? (1 << pl.fct_tile_log2) : pl.s;
  a.nblocks = (n + tile - 1) / tile;
  a.full_blocks = n / tile;
  a.log2s = pl.log2s;
  const uint32_t esz = dt == L1S_BF16 ? 2u : 4u;
  a.stage_a_bytes = static_cast<uint32_t>(tile) * pl.d * esz;
  a.stage_bytes = fct_stage_bytes(tile, pl.d, dt);
  const bool staged = pl.fct_staged && fct_can_stage(pl.s, pl.d, dt, lda, A, b);
  a.tma = staged ? 1 : 0;
  a.key = make_key(p->seed);
  a.problem = p->problem_id;
  a.row_offset = row_offset;
  a.sign_flip = p->sign_flip;
  a.inv_sqrt_s = static_cast<float>(1.0 / sqrt(static_cast<double>(pl.s)));
  a.partials = reinterpret_cast<float*>(ws + pl.off_partials);
  a.accumulate = accumulate ? 1 : 0;
  a.sd = pl.d;
  a.flags = reinterpret_cast<uint32_t*>(ws + pl.off_status);
  // A layout that cannot be staged falls back to direct loads with the same grid; the
  // direct variant needs less shared memory than the staged one it was planned for.
  // The narrow-X kernel stages every block (by TMA when it can, else with plain loads).
  // So does the bucket-sorted kernel.
  const int wsw = pl.fct_ws;
  const int srt = pl.fct_sorted;
  if (srt) a.tma = fct_can_stage(tile, pl.d, dt, lda, A, b) ? 1 : 0;
  if (wsw) {
    // Rows with padding (lda > d) are staged whole by the same bulk copies (S consecutive
    // rows are one contiguous range) when the wider stage keeps the planned residency.
    if (lda != pl.d && lda <= 2 * pl.d && fct_can_stage(tile, static_cast<int>(lda), dt, lda, A, b)) {
      const void* fw = fct_ws_kernel(pl.fct_tile_log2, pl.log2s, dt, wsw, pl.fct_lean != 0);
      const size_t s0 = fct_ws_smem_bytes(tile, pl.d, dt, pl.r1, wsw, pl.fct_lean != 0);
      const size_t s1 = fct_ws_smem_bytes(tile, static_cast<int>(lda), dt, pl.r1, wsw, pl.fct_lean != 0);
      int o0 = 0, o1 = 0;
      if (s1 <= device_info().max_smem_optin &&
          allow_dynamic_smem(reinterpret_cast<const void*>(fw), s1, "cudaFuncSetAttribute(fct_embed)") &&
          cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o0, fw, pl.fct_threads, s0), "occupancy") &&
          cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, fw, pl.fct_threads, s1), "occupancy") &&
          o1 >= o0 && o1 > 0)
        a.sd = static_cast<int>(lda);
    }
    a.stage_a_bytes = static_cast<uint32_t>(tile) * a.sd * esz;
    a.stage_bytes = fct_stage_bytes(tile, a.sd, dt);
    a.tma = fct_can_stage(tile, a.sd, dt, a.sd == pl.d ? lda : a.sd, A, b) ? 1 : 0;
  }
  const void* fn = srt ? fct_sorted_kernel(pl.log2s, dt, srt)
                       : (wsw ? fct_ws_kernel(pl.fct_tile_log2, pl.log2s, dt, wsw, pl.fct_lean != 0)
                              : fct_kernel(pl.log2s, dt, staged));
  const size_t smem = srt ? fct_sorted_smem_bytes(pl.s, pl.d, dt, pl.r1, srt)
                          : (wsw ? fct_ws_smem_bytes(tile, a.sd, dt, pl.r1, wsw, pl.fct_lean != 0)
                                 : fct_smem_bytes(pl.s, pl.d, dt, pl.r1, pl.fct_width, staged));
  if (!allow_dynamic_smem(reinterpret_cast<const void*>(fn), smem, "cudaFuncSetAttribute(fct_embed)"))
    return false;
  void* args[] = {&a};
  dim3 grid(pl.fct_ctas, pl.fct_slices);
  if (!cuda_ok(cudaLaunchKernel(fn, grid, dim3(pl.fct_threads), args, smem, st), "launch fct_embed")) return false;
  count_launch(1);
  return true;
}

static bool launch_fct_reduce(const Plan& pl, const l1s_params* p, float* pix, unsigned char* ws, cudaStream_t st,
                              double* pi2_out) {
  if (pl.fct_cols) return launch_fct_cols_reduce(pl, p, pix, ws, st, pi2_out);
  const int per = pl.r1 * pl.fct_width;
  dim3 rgrid((per + 31) / 32, pl.fct_slices);
  fct_reduce_kernel<<<rgrid, 1024, 0, st>>>(reinterpret_cast<float*>(ws + pl.off_partials), pl.fct_ctas, pl.r1,
                                            pl.fct_width, pl.q, pix, reinterpret_cast<uint32_t*>(ws + pl.off_status),
                                            make_key(p->seed), p->problem_id, pl.q * pl.r2, pl.r2,
                                            p->variant == 1 ? 1 : 0, pl.pi2_neg_lo, pl.pi2_neg_hi, pi2_out);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch fct_reduce");
}

bool launch_fct(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b,
                const l1s_params* p, float* pix, unsigned char* ws, cudaStream_t st, double* pi2_out) {
  if (!launch_fct_part(pl, A, lda, dt, b, pl.n, p->global_row_offset, p, false, ws, st)) return false;
  return launch_fct_reduce(pl, p, pix, ws, st, pi2_out);
}

// Phase 1 on inputs that are still in host memory: the rows arrive in pl.fct_chunks
// chunks (multiples of the kernel's tile) by copies on `cp`, and the phase-1 launch of
// chunk k on `st` waits only for its own copy (event evs[k]), so the transfer of chunk
// k+1 overlaps the transform of chunk k.  Launches after the first add their block
// partials to the earlier ones (the launches are ordered on `st`), and one reduction
// forms Π1X.  A_dev and b_dev receive the rows (lda = d) for the later phases.  The
// caller has made `cp` wait for earlier work on `st` that reads A_dev or b_dev.
bool launch_fct_streamed(const Plan& pl, const void* A_host, int64_t lda_host, l1s_dtype dt, const float* b_host,
                         void* A_dev, float* b_dev, const l1s_params* p, float* pix, unsigned char* ws,
                         cudaStream_t st, cudaStream_t cp, const cudaEvent_t* evs, double* pi2_out) {
  const int K = std::max(pl.fct_chunks, 1);
  const int64_t tile = pl.fct_cols ? fct_cols_tile() : (pl.fct_ws ? (int64_t{1} << pl.fct_tile_log2) : pl.s);
  const int64_t per_chunk = ((pl.n + K - 1) / K + tile - 1) / tile * tile;
  const size_t esz = dt == L1S_BF16 ? 2 : 4;
  for (int k = 0; k < K; ++k) {
    const int64_t r0 = k * per_chunk;
    if (r0 >= pl.n) break;
    const int64_t rows = std::min(per_chunk, pl.n - r0);
    unsigned char* a_dst = static_cast<unsigned char*>(A_dev) + static_cast<size_t>(r0) * pl.d * esz;
    const unsigned char* a_src = static_cast<const unsigned char*>(A_host) + static_cast<size_t>(r0) * lda_host * esz;
    if (!cuda_ok(cudaMemcpy2DAsync(a_dst, esz * pl.d, a_src, esz * lda_host, esz * pl.d, rows,
                                   cudaMemcpyHostToDevice, cp),
                 "copy A chunk") ||
        !cuda_ok(cudaMemcpyAsync(b_dev + r0, b_host + r0, sizeof(float) * rows, cudaMemcpyHostToDevice, cp),
                 "copy b chunk") ||
        !cuda_ok(cudaEventRecord(evs[k], cp), "record chunk event") ||
        !cuda_ok(cudaStreamWaitEvent(st, evs[k], 0), "wait for chunk"))
      return false;
    if (!launch_fct_part(pl, a_dst, pl.d, dt, b_dev + r0, rows, p->global_row_offset + r0, p, k > 0, ws, st))
      return false;
  }
  return launch_fct_reduce(pl, p, pix, ws, st, pi2_out);
}

}  // namespace l1s
