// Phase 1 for wide X: the FCT1 embedding Π1·X = 4·B·C·H̃·D·X (§3.1, FCT1 construction;
// Figure 2, steps 1-2) when the r1 × q partial of Π1X does not fit one thread block's
// shared memory (16 < d ≤ 128, s ≤ 1024, r1 ≤ 2280).
//
// The columns of A are cut into slices of 16; a thread block owns one slice and keeps
// that slice's r1 × 16 FP32 partial of Π1X in shared memory (B's hashed sum is a
// shared-memory reduction, no global atomics).  Blocks of one slice walk the tiles of
// 1024 rows (each tile holds 1024/s blocks of H_s) in a grid stride; there is one block
// per SM, and a slice's blocks read only its 16 columns of every row, so X crosses HBM
// once.  Per tile, in a block of 16 warps:
//   * the rows' values arrive straight in registers (coalesced loads issued one tile
//     ahead, so the transfer of tile t+1 overlaps the arithmetic of tile t; no staging
//     buffer, which leaves the shared memory to the partial);
//   * pass 1: a half-warp holds one 16-column row group (rows g, g+32, …, g+992 of the
//     tile; lanes are the columns); it scatters the identity half of G_s = [H_s; I_s]
//     (P[h_I(i)][c] += 4·c_I(i)·σ_i·x_ic), applies σ, runs the butterflies over row bits
//     5-9 in registers and stores the tile;
//   * pass 2: a half-warp reads 32 consecutive rows of the tile (row bits 0-4 in
//     registers), runs those butterflies and scatters the Hadamard half
//     (P[h_H(i)][c] += 4·c_H(i)/√s·(H_s z)_ic);
//   * the threads draw the next tile's signs, buckets and Cauchy scales (one Philox call
//     per row, counter = global row id) while the atomics of the current passes drain.
// Every slice redraws the row variates: the bound of this kernel is the shared-memory
// FP32 atomic rate (two atomics per element), and the draws run on the ALUs beside it.
// The tile and the draws are padded by 16 words / one entry after every 32 rows, so that
// both passes read and write them without bank conflicts.  The draws hold the byte offset
// of their row of the partial and σ as a sign mask, and the scatter is a shared-memory
// reduction issued without a compiler memory barrier, so that a warp can keep loading the
// draws of later rows while its earlier additions are in flight.
//
// The b column (−b, the last column of X) is transformed by a second, light kernel: one
// warp per tile of 1024 rows, lane l holding rows l + 32k; it draws its own rows, runs the
// butterflies over k in registers and over l by shuffles, and scatters both halves into
// its block's r1-entry partial.
#include <cuda.h>

#include <algorithm>

#include "l1s_common.cuh"

namespace l1s {

constexpr int kColW = 16;                                   // columns of A per slice
constexpr int kColT = 1024;                                 // rows per tile
constexpr int kColAWarps = 16;
constexpr int kColThreads = 32 * kColAWarps;
constexpr int kBcolThreads = 256;                           // b-column kernel: 8 warps, one tile each
constexpr int kColJ = 32;                                   // rows per thread in each pass
constexpr int kColTileWords = kColT * kColW + (kColT / 32) * kColW;
constexpr int kColMeta = kColT + kColT / 32;

// P[off] += v in shared memory (off in bytes from the shared window), with no result and
// no compiler memory barrier: nothing in the passes reads P, so later loads of other
// arrays may be scheduled ahead of it (the block barriers order it before P is read).
__device__ __forceinline__ void red_add_shared(uint32_t addr, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v));
}

static_assert(kColT == 2 * kColAWarps * kColJ, "a pass covers the tile once");

struct ColsArgs {
  const void* A;
  int64_t lda;
  const float* b;
  int64_t n;
  int d, r1, nslices;
  int log2s;
  float inv_sqrt_s;
  int64_t ntiles;
  Key2 key;
  uint32_t problem;
  int64_t row_offset;
  int sign_flip;
  float* partials;      // [nslices][gridDim.x][r1][16]
  float* partials_b;    // b-column kernel: [its blocks][r1]
  int accumulate;       // 1: add to the partials of an earlier launch over other rows
  uint32_t* flags;      // status word (TIMEOUT)
  // Per-row draws of this launch's tiles (fct_draws_kernel), read by the TMA form and the
  // b-column kernel: {4·c_I, byte offset of h_I's partial row | σ·2^31, 4·c_H/√s, byte
  // offset of h_H's partial row}, row r of the launch at index r.
  uint4* draws;
};

__device__ __forceinline__ int col_tile_off(int row, int c) { return row * kColW + c + ((row >> 5) << 4); }
__device__ __forceinline__ int col_meta(int row) { return row + (row >> 5); }

// Raw bits of one element (widened where it is used, so that a prefetch does not wait).
template <typename TA>
__device__ __forceinline__ uint32_t col_ld(const TA* p) {
  if constexpr (sizeof(TA) == 4) return __float_as_uint(__ldcs(p));
  else return static_cast<uint32_t>(__ldcs(reinterpret_cast<const unsigned short*>(p)));
}

template <typename TA>
__device__ __forceinline__ uint32_t col_widen(uint32_t raw) {
  if constexpr (sizeof(TA) == 4) return raw;
  else return raw << 16;
}

// One pass-1/pass-2 step over tile t of this block's slice; x holds t's values (raw bits),
// xn receives tile t + stride's (loads issued here, consumed by the next step).  FULL: the
// tile is one H_s block (s = 1024), every butterfly stage runs.
template <typename TA, bool FULL>
struct ColsBlock {
  const ColsArgs& a;
  uint32_t pc;          // shared address of P[0][c]
  float* tile;
  uint4* mI;            // {4·c_I·σ, byte offset of row h_I of P, σ sign mask, 0}
  uint2* mH;            // {4·c_H/√s, byte offset of row h_H of P}
  int slice, c, hw;
  bool live;

  __device__ __forceinline__ void load(int64_t t, uint32_t (&x)[kColJ]) const {
    if (t >= a.ntiles) return;
    const int64_t r0 = t * kColT + hw;
    const TA* A = static_cast<const TA*>(a.A) + r0 * a.lda + slice * kColW + c;
    const int64_t stride = 32 * a.lda;
    if (live && t * kColT + kColT <= a.n) {
#pragma unroll
      for (int j = 0; j < kColJ; ++j) x[j] = col_ld<TA>(A + j * stride);
    } else {
#pragma unroll
      for (int j = 0; j < kColJ; ++j) x[j] = (live && r0 + 32 * j < a.n) ? col_ld<TA>(A + j * stride) : 0u;
    }
  }

  // Draws of tile-row r of tile t: the identity and Hadamard entries of both halves.
  __device__ __forceinline__ void draw(int64_t t, int r, uint4& mi, uint2& mh) const {
    const uint64_t grow = static_cast<uint64_t>(a.row_offset + t * kColT + r);
    const uint4 o = draw_row(a.key, grow, a.problem, kStreamFct);
    const bool neg = a.sign_flip && (o.w & 1u);
    const float wI = 4.f * cauchy_f32(o.w >> 8);
    mi = make_uint4(__float_as_uint(neg ? -wI : wI), static_cast<uint32_t>(bucket_of(o.z, a.r1)) * (kColW * 4),
                    neg ? 0x80000000u : 0u, 0u);
    mh = make_uint2(__float_as_uint(4.f * cauchy_f32(o.y >> 8) * a.inv_sqrt_s),
                    static_cast<uint32_t>(bucket_of(o.x, a.r1)) * (kColW * 4));
  }

  __device__ __forceinline__ void butterflies(float (&v)[kColJ], int lo_bit) const {
#pragma unroll
    for (int b = 0; b < 5; ++b)
      if (FULL || lo_bit + b < a.log2s)
#pragma unroll
        for (int j = 0; j < kColJ; ++j)
          if ((j & (1 << b)) == 0) {
            const float lo = v[j], hi = v[j | (1 << b)];
            v[j] = lo + hi;
            v[j | (1 << b)] = lo - hi;
          }
  }

  __device__ __forceinline__ void step(int64_t t, uint32_t (&x)[kColJ], uint32_t (&xn)[kColJ]) const {
    const int64_t tn = t + gridDim.x;
    const int tid = threadIdx.x;
    __syncthreads();                                     // draws of t visible; the tile is free
    load(tn, xn);
    uint4 mi0 = make_uint4(0u, 0u, 0u, 0u), mi1 = mi0;
    uint2 mh0 = make_uint2(0u, 0u), mh1 = mh0;
    {
      // ---- pass 1: identity scatter, σ, butterflies over row bits 5-9, tile store
      float v[kColJ];
#pragma unroll
      for (int j = 0; j < kColJ; ++j) {
        const uint4 m = mI[col_meta(hw + 32 * j)];
        const uint32_t xb = col_widen<TA>(x[j]);
        if (live) red_add_shared(pc + m.y, __uint_as_float(m.x) * __uint_as_float(xb));
        v[j] = __uint_as_float(xb ^ m.z);                // z = σ·x
      }
      butterflies(v, 5);
#pragma unroll
      for (int j = 0; j < kColJ; ++j) tile[col_tile_off(hw + 32 * j, c)] = v[j];
      if (tn < a.ntiles) draw(tn, tid, mi0, mh0);      // the next tile's draws, first row
    }
    __syncthreads();                                     // the tile holds pass 1; mI of t is free
    if (tn < a.ntiles) mI[col_meta(tid)] = mi0;
    {
      // ---- pass 2: butterflies over row bits 0-4, Hadamard scatter
      float v[kColJ];
#pragma unroll
      for (int i = 0; i < kColJ; ++i) v[i] = tile[col_tile_off(32 * hw + i, c)];
      butterflies(v, 0);
      if (live) {
#pragma unroll
        for (int i = 0; i < kColJ; ++i) {
          const uint2 m = mH[col_meta(32 * hw + i)];
          red_add_shared(pc + m.y, __uint_as_float(m.x) * v[i]);
        }
      }
      if (tn < a.ntiles) draw(tn, tid + kColT / 2, mi1, mh1);   // second row
    }
    __syncthreads();                                     // pass 2 done: mH of t and the tile are free
    if (tn < a.ntiles) {
      mH[col_meta(tid)] = mh0;
      mI[col_meta(tid + kColT / 2)] = mi1;
      mH[col_meta(tid + kColT / 2)] = mh1;
    }
  }
};

template <typename TA, bool FULL>
__global__ void __launch_bounds__(kColThreads, 1) fct_embed_cols_kernel(const ColsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r1 = a.r1;
  float* P = reinterpret_cast<float*>(smem_raw);                 // [r1][16]
  float* tile = P + r1 * kColW;                                  // padded [1024][16]
  uint4* mI = reinterpret_cast<uint4*>(tile + kColTileWords);    // padded [1024]
  uint2* mH = reinterpret_cast<uint2*>(mI + kColMeta);           // padded [1024]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int slice = blockIdx.y;
  const int wcols = min(kColW, a.d - slice * kColW);
  const int c = lane & 15;
  ColsBlock<TA, FULL> blk{a, smem_u32(P + c), tile, mI, mH, slice, c, 2 * warp + (lane >> 4), c < wcols};
  for (int i = tid; i < r1 * kColW; i += blockDim.x) P[i] = 0.f;
  const int64_t t0 = blockIdx.x;
  if (t0 < a.ntiles)
    for (int r = tid; r < kColT; r += kColThreads) {
      uint4 mi;
      uint2 mh;
      blk.draw(t0, r, mi, mh);
      mI[col_meta(r)] = mi;
      mH[col_meta(r)] = mh;
    }
  uint32_t xa[kColJ], xb[kColJ];
  blk.load(t0, xa);
#pragma unroll 1
  for (int64_t t = t0; t < a.ntiles; t += 2 * static_cast<int64_t>(gridDim.x)) {
    blk.step(t, xa, xb);
    if (t + gridDim.x >= a.ntiles) break;
    blk.step(t + gridDim.x, xb, xa);
  }
  __syncthreads();
  // Non-finite input shows up as a non-finite partial (checked in the reduction).
  const size_t cta = static_cast<size_t>(slice) * gridDim.x + blockIdx.x;
  float* out = a.partials + cta * r1 * kColW;
  for (int i = tid; i < r1 * kColW; i += blockDim.x) out[i] = (a.accumulate ? out[i] : 0.f) + P[i];
}


// ----------------------------------------------------------------- TMA-staged form
// The same slices with twice the warps: shared-memory FP32 reductions are latency bound
// per warp (about one in flight per warp), so their rate grows with the warps that issue
// them; 32 warps of 64 registers hold 16 values each per pass.  The tile arrives by TMA
// (2-D boxes of 16 columns × 256 rows; rows past n and columns past d read as zeros) in
// the tile buffer itself, pass 1 transforms it in place, and the next tile's copy is
// issued as soon as pass 2 has read the tile, so the transfer overlaps the scatter.
//   pass 1: half h of warp w holds rows h + 2w + 64j (j < 16): butterflies over row bits
//           6-9 in registers and bit 0 by a shuffle between the two half-warps;
//   pass 2: rows (w & 1) + 2i + 32h + 64(w >> 1) (i < 16): bits 1-4 in registers and
//           bit 5 by a shuffle.
// BF16 tiles land in the upper half of the buffer and are widened to FP32 in pass 1.
// Pass 1 stores row r of its output at row r ^ (bit 5 of r): a warp instruction touches
// two rows, which differ in bit 0 in pass 1 and in bit 5 in pass 2, and this placement
// puts them in opposite halves of the 32 banks in both passes.  The identity half's draws
// are 8 bytes a row ({4·c_I, offset of its partial row with σ in bit 31}), which a warp
// reads in half the shared-memory wavefronts of a 16-byte record.
constexpr int kTmaThreads = 1024;

// Every row's draws, once per launch: the Philox call of the row's global id (stream 0),
// its two Cauchy scales and buckets and σ, in the 16-byte record the phase-1 kernels read.
// Each of the column slices and the b column would otherwise redraw every row.
__global__ void __launch_bounds__(256) fct_draws_kernel(const ColsArgs a) {
  const int64_t rows = a.ntiles * kColT;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < rows;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint4 o = draw_row(a.key, static_cast<uint64_t>(a.row_offset + r), a.problem, kStreamFct);
    const bool neg = a.sign_flip && (o.w & 1u);
    a.draws[r] = make_uint4(__float_as_uint(4.f * cauchy_f32(o.w >> 8)),
                            (static_cast<uint32_t>(bucket_of(o.z, a.r1)) * (kColW * 4)) | (neg ? 0x80000000u : 0u),
                            __float_as_uint(4.f * cauchy_f32(o.y >> 8) * a.inv_sqrt_s),
                            static_cast<uint32_t>(bucket_of(o.x, a.r1)) * (kColW * 4));
  }
}

// The butterfly across the two half-warps (lane bit 4) on pairs: the lower half keeps
// v + o, the upper o − v, as one packed fma with ±1.
__device__ __forceinline__ void f2_cross_halves(uint64_t (&p)[8], uint64_t sgn) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float x, y;
    f2_unpack(p[k], x, y);
    const float ox = __shfl_xor_sync(0xffffffffu, x, 16), oy = __shfl_xor_sync(0xffffffffu, y, 16);
    p[k] = f2_fma(sgn, p[k], f2_pack(ox, oy));
  }
}
constexpr int kTmaJ = 16;
constexpr int kTmaBoxRows = 256;

__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ int tma_hpad(int row) { return row + (row >> 5); }

template <typename TA, bool FULL>
__global__ void __launch_bounds__(kTmaThreads, 1)
    fct_embed_cols_tma_kernel(const __grid_constant__ CUtensorMap mapA, const ColsArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full_bar;
  const int r1 = a.r1;
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float* tile = reinterpret_cast<float*>(base);                   // [1024][16] FP32
  float* P = tile + kColT * kColW;                                // [r1][16]
  uint2* mI = reinterpret_cast<uint2*>(P + r1 * kColW);           // [1024] {4·c_I, offset | σ·2^31}
  uint2* mH = reinterpret_cast<uint2*>(mI + kColT);               // padded [1024]
  unsigned char* stage = reinterpret_cast<unsigned char*>(tile) + (sizeof(TA) == 4 ? 0 : kColT * kColW * 2);
  constexpr uint32_t kTileBytes = kColT * kColW * sizeof(TA);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, h = lane >> 4, c = lane & 15;
  const int sw = (warp >> 4) & 1;                                  // bit 5 of this thread's pass-1 rows
  const uint64_t sgn = h ? f2_pack(-1.f, -1.f) : f2_pack(1.f, 1.f);  // cross-half butterfly sign
  const int slice = blockIdx.y;
  const bool live = c < min(kColW, a.d - slice * kColW);
  const uint32_t pc = smem_u32(P + c);
  const int lg = FULL ? 10 : a.log2s;
  const int64_t G = gridDim.x;

  // Row r of tile t's draws from the per-launch table (loaded one tile ahead, like the tile).
  auto draw = [&](int64_t t, int r, uint2& mi, uint2& mh) {
    const uint4 e = __ldg(a.draws + (t * kColT + r));
    mi = make_uint2(e.x, e.y);
    mh = make_uint2(e.z, e.w);
  };
  auto issue = [&](int64_t t) {
    mbar_arrive_expect_tx(&full_bar, kTileBytes);
#pragma unroll
    for (int k = 0; k < kColT / kTmaBoxRows; ++k)
      tma_load_box(stage + k * kTmaBoxRows * kColW * sizeof(TA), &mapA, slice * kColW,
                   static_cast<int>(t * kColT + k * kTmaBoxRows), &full_bar);
  };

  for (int i = tid; i < r1 * kColW; i += blockDim.x) P[i] = 0.f;
  if (tid == 0) {
    mbar_init(&full_bar, 1);
    fence_mbar_init();
  }
  const int64_t t0 = blockIdx.x;
  uint2 mh_next = make_uint2(0u, 0u);
  if (t0 < a.ntiles) {
    uint2 mi;
    draw(t0, tid, mi, mh_next);
    mI[tid] = mi;
  }
  __syncthreads();
  if (tid == 0 && t0 < a.ntiles) issue(t0);
  uint32_t phase = 0;
  bool aborted = false;
#pragma unroll 1
  for (int64_t t = t0; t < a.ntiles; t += G, phase ^= 1u) {
    const bool ok = mbar_wait_bounded(&full_bar, phase, kWaitCycles);
    if (__syncthreads_or(!ok)) {                         // the tile of t has landed; mI of t is visible
      aborted = true;
      break;
    }
    mH[tma_hpad(tid)] = mh_next;                         // pass 2 of the previous tile is done with mH
    const int64_t tn = t + G;
    uint2 mi_next = make_uint2(0u, 0u);
    float v[kTmaJ];
    // ---- pass 1: identity scatter, σ, butterflies over row bits 0 and 6-9, in place
    {
      const int rb = h + 2 * warp;
#pragma unroll
      for (int j = 0; j < kTmaJ; ++j) {
        const int row = rb + 64 * j;
        uint32_t xb;
        if constexpr (sizeof(TA) == 4) xb = __float_as_uint(tile[row * kColW + c]);
        else xb = static_cast<uint32_t>(reinterpret_cast<const uint16_t*>(stage)[row * kColW + c]) << 16;
        const uint2 m = mI[row];
        const uint32_t sg = m.y & 0x80000000u;
        v[j] = __uint_as_float(xb ^ sg);                 // z = σ·x
        if (live) red_add_shared(pc + (m.y ^ sg), __uint_as_float(m.x) * v[j]);
      }
      if constexpr (sizeof(TA) == 2) __syncthreads();    // every BF16 value read before FP32 rows are written
      uint64_t p[kTmaJ / 2];
#pragma unroll
      for (int q = 0; q < kTmaJ / 2; ++q) p[q] = f2_pack(v[q], v[q + 8]);
      if (FULL || lg > 0) f2_cross_halves(p, sgn);     // row bit 0
      f2_butterflies<kTmaJ>(p, FULL ? 0xFu : f2_stage_mask(6, lg));   // row bits 6-9
#pragma unroll
      for (int q = 0; q < kTmaJ / 2; ++q) {
        float x, y;
        f2_unpack(p[q], x, y);
        tile[((rb + 64 * q) ^ sw) * kColW + c] = x;
        tile[((rb + 64 * (q + 8)) ^ sw) * kColW + c] = y;
      }
      if (tn < a.ntiles) draw(tn, tid, mi_next, mh_next);
    }
    __syncthreads();                                     // the tile holds pass 1; mI of t is free
    if (tn < a.ntiles) mI[tid] = mi_next;
    // ---- pass 2: butterflies over row bits 1-5, Hadamard scatter
    const int qb = (warp & 1) + 32 * h + 64 * (warp >> 1);
#pragma unroll
    for (int i = 0; i < kTmaJ; ++i) v[i] = tile[((qb + 2 * i) ^ h) * kColW + c];
    __syncthreads();                                     // the tile is free: the next copy may land
    if (tid == 0 && tn < a.ntiles) {
      fence_proxy_async_smem();
      issue(tn);
    }
    {
      uint64_t p[kTmaJ / 2];
#pragma unroll
      for (int q = 0; q < kTmaJ / 2; ++q) p[q] = f2_pack(v[q], v[q + 8]);
      f2_butterflies<kTmaJ>(p, FULL ? 0xFu : f2_stage_mask(1, lg));   // row bits 1-4
      if (FULL || 5 < lg) f2_cross_halves(p, sgn);     // row bit 5
#pragma unroll
      for (int q = 0; q < kTmaJ / 2; ++q) f2_unpack(p[q], v[q], v[q + 8]);
    }
    if (live) {
#pragma unroll
      for (int i = 0; i < kTmaJ; ++i) {
        const uint2 m = mH[tma_hpad(qb + 2 * i)];
        red_add_shared(pc + m.y, __uint_as_float(m.x) * v[i]);
      }
    }
  }
  __syncthreads();
  if (aborted) {
    // Let the copy in flight land (a bounded wait) before the shared memory is released.
    if (tid == 0) {
      raise_flag(a.flags, L1S_ERR_TIMEOUT);
      mbar_wait_bounded(&full_bar, phase, 20000000LL);
    }
    __syncthreads();
    return;
  }
  const size_t cta = static_cast<size_t>(slice) * gridDim.x + blockIdx.x;
  float* out = a.partials + cta * r1 * kColW;
  for (int i = tid; i < r1 * kColW; i += blockDim.x) out[i] = (a.accumulate ? out[i] : 0.f) + P[i];
}

// The b column of X (−b): warp w of the grid transforms tiles w, w + warps, … of 1024 rows.
// Lane l holds rows l + 32k (k < 32) and draws them itself; the Hadamard entries wait in
// a per-warp shared-memory table until the transform is done.
__global__ void __launch_bounds__(kBcolThreads) fct_embed_bcol_kernel(const ColsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r1 = a.r1;
  float* Pb = reinterpret_cast<float*>(smem_raw);                           // [r1]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* mH = reinterpret_cast<float2*>(Pb + ((r1 + 3) & ~3)) + warp * kColT;   // [32 k][32 lanes]
  for (int i = tid; i < r1; i += blockDim.x) Pb[i] = 0.f;
  __syncthreads();
  const int lg = a.log2s;
  const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (kBcolThreads / 32);
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * (kBcolThreads / 32) + warp; t < a.ntiles; t += nwarps) {
    const int64_t r0 = t * kColT;
    float v[kColJ];
#pragma unroll
    for (int k = 0; k < kColJ; ++k) {
      const int64_t row = r0 + lane + 32 * k;
      v[k] = row < a.n ? -__ldcs(a.b + row) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kColJ; ++k) {
      const uint4 e = __ldg(a.draws + (r0 + lane + 32 * k));
      if (e.y & 0x80000000u) v[k] = -v[k];                                  // z = σ·x
      red_add_shared(smem_u32(Pb + ((e.y & 0x7FFFFFFFu) >> 6)), __uint_as_float(e.x) * v[k]);   // identity half
      mH[k * 32 + lane] = make_float2(__uint_as_float(e.z), __uint_as_float(e.w >> 6));
    }
#pragma unroll
    for (int b = 0; b < 5; ++b)
      if (5 + b < lg)
#pragma unroll
        for (int k = 0; k < kColJ; ++k)
          if ((k & (1 << b)) == 0) {
            const float lo = v[k], hi = v[k | (1 << b)];
            v[k] = lo + hi;
            v[k | (1 << b)] = lo - hi;
          }
#pragma unroll
    for (int b = 0; b < 5; ++b)
      if (b < lg) {
        const bool upper = (lane >> b) & 1;
#pragma unroll
        for (int k = 0; k < kColJ; ++k) {
          const float o = __shfl_xor_sync(0xffffffffu, v[k], 1 << b);
          v[k] = upper ? (o - v[k]) : (v[k] + o);
        }
      }
#pragma unroll
    for (int k = 0; k < kColJ; ++k) {
      const float2 m = mH[k * 32 + lane];
      red_add_shared(smem_u32(Pb + __float_as_uint(m.y)), m.x * v[k]);     // Hadamard half
    }
  }
  __syncthreads();
  float* out = a.partials_b + static_cast<size_t>(blockIdx.x) * r1;
  for (int i = tid; i < r1; i += blockDim.x) out[i] = (a.accumulate ? out[i] : 0.f) + Pb[i];
}

// Fixed-order sum of the per-block partials: Π1X[r][16·k + c] = Σ_g partial[k][g][r][c]
// (y-block k < slices) and Π1X[r][d] = Σ_g partial_b[g][r] over the b-column kernel's
// blocks (y-block k = slices).
// Warp w adds partials w, w + 32, …; warp 0 then adds the 32 warp sums in order.  Π2
// (q × r2 FP64) is drawn here too, as in the other phase-1 reduction.
__global__ void __launch_bounds__(1024) fct_reduce_cols_kernel(const float* __restrict__ partials,
                                                               const float* __restrict__ partials_b, int ctas,
                                                               int ctas_b, int slices, int r1, int d,
                                                               float* __restrict__ pix,
                                                               uint32_t* flags, Key2 key, uint32_t problem, int npi2,
                                                               int r2, int pi2_gauss, int neg_lo, int neg_hi,
                                                               double* __restrict__ pi2) {
  if (pi2 && blockIdx.y == 0)
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < npi2; e += gridDim.x * blockDim.x) {
      const double v = pi2_value(key, problem, e, pi2_gauss);
      const int row = e / r2;
      pi2[e] = (row >= neg_lo && row < neg_hi) ? -v : v;
    }
  __shared__ float red[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool bcol = static_cast<int>(blockIdx.y) == slices;
  const int per = bcol ? r1 : r1 * kColW;
  const int nparts = bcol ? ctas_b : ctas;
  const float* base0 = bcol ? partials_b : partials + static_cast<size_t>(blockIdx.y) * ctas * per;
  const int e = blockIdx.x * 32 + lane;
  float acc = 0.f;
  if (e < per) {
    const float* base = base0 + e;
    int c = warp;
    for (; c + 96 < nparts; c += 128) {
      const float v0 = base[static_cast<size_t>(c) * per];
      const float v1 = base[static_cast<size_t>(c + 32) * per];
      const float v2 = base[static_cast<size_t>(c + 64) * per];
      const float v3 = base[static_cast<size_t>(c + 96) * per];
      acc += v0;
      acc += v1;
      acc += v2;
      acc += v3;
    }
    for (; c < nparts; c += 32) acc += base[static_cast<size_t>(c) * per];
  }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && e < per) {
    float s = 0.f;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) s += red[k][lane];
    const int q = d + 1;
    int r, col;
    if (bcol) {
      r = e;
      col = d;
    } else {
      r = e / kColW;
      col = blockIdx.y * kColW + (e - r * kColW);
    }
    if (col < q && (bcol || col < d)) {
      pix[static_cast<size_t>(r) * q + col] = s;
      if (!isfinite(s)) raise_flag(flags, L1S_ERR_NONFINITE);
    }
  }
}

// ----------------------------------------------------------------- host side
size_t fct_cols_smem_bytes(int r1) {
  return static_cast<size_t>(r1) * kColW * 4 + static_cast<size_t>(kColTileWords) * 4 +
         static_cast<size_t>(kColMeta) * (sizeof(uint4) + sizeof(uint2));
}

static size_t bcol_smem_bytes(int r1) {
  return static_cast<size_t>((r1 + 3) & ~3) * 4 + static_cast<size_t>(kBcolThreads / 32) * kColT * sizeof(float2);
}

static size_t cols_tma_smem_bytes(int r1) {
  return 128 + static_cast<size_t>(kColT) * kColW * 4 + static_cast<size_t>(r1) * kColW * 4 +
         static_cast<size_t>(kColT) * sizeof(uint2) + static_cast<size_t>(kColMeta) * sizeof(uint2);
}

int fct_cols_slices(int log2s, int d, int r1, int max_smem) {
  if (log2s > 10 || d <= 0) return 0;
  if (fct_cols_smem_bytes(r1) > static_cast<size_t>(max_smem) || bcol_smem_bytes(r1) > static_cast<size_t>(max_smem) ||
      cols_tma_smem_bytes(r1) > static_cast<size_t>(max_smem))
    return 0;
  return (d + kColW - 1) / kColW;
}

int fct_cols_threads() { return kColThreads; }
int fct_cols_tile() { return kColT; }

bool encode_tiled_2d(CUtensorMap* map, CUtensorMapDataType dtype, const void* base, uint64_t rows, uint64_t cols,
                     uint64_t row_bytes, uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swizzle);

const void* fct_cols_kernel(l1s_dtype dt, bool full) {
  if (full)
    return dt == L1S_BF16 ? reinterpret_cast<const void*>(&fct_embed_cols_kernel<uint16_t, true>)
                          : reinterpret_cast<const void*>(&fct_embed_cols_kernel<float, true>);
  return dt == L1S_BF16 ? reinterpret_cast<const void*>(&fct_embed_cols_kernel<uint16_t, false>)
                        : reinterpret_cast<const void*>(&fct_embed_cols_kernel<float, false>);
}

// Blocks of the b-column kernel: two per SM, no more than one warp per tile.
static int bcol_ctas(int64_t n) {
  const int64_t tiles = (n + kColT - 1) / kColT;
  const int64_t want = 2 * static_cast<int64_t>(device_info().sms);
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, (tiles + 7) / 8)));
}

// Partial floats of a launch with `ctas` blocks per slice over n rows.
size_t fct_cols_partial_floats(int slices, int ctas, int r1, int64_t n) {
  return static_cast<size_t>(slices) * ctas * r1 * kColW + static_cast<size_t>(bcol_ctas(n)) * r1;
}

bool launch_fct_cols(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n,
                     int64_t row_offset, const l1s_params* p, bool accumulate, unsigned char* ws, cudaStream_t st) {
  ColsArgs a;
  a.A = A;
  a.lda = lda;
  a.b = b;
  a.n = n;
  a.d = pl.d;
  a.r1 = pl.r1;
  a.nslices = pl.fct_cols;
  a.log2s = pl.log2s;
  a.inv_sqrt_s = static_cast<float>(1.0 / sqrt(static_cast<double>(pl.s)));
  a.ntiles = (n + kColT - 1) / kColT;
  a.key = make_key(p->seed);
  a.problem = p->problem_id;
  a.row_offset = row_offset;
  a.sign_flip = p->sign_flip;
  float* parts = reinterpret_cast<float*>(ws + pl.off_partials);
  a.partials = parts;
  a.partials_b = parts + static_cast<size_t>(pl.fct_cols) * pl.fct_ctas * pl.r1 * kColW;
  a.accumulate = accumulate ? 1 : 0;
  a.flags = reinterpret_cast<uint32_t*>(ws + pl.off_status);
  a.draws = reinterpret_cast<uint4*>(ws + pl.off_draws);
  void* args[] = {&a};
  {
    const int64_t rows = a.ntiles * kColT;
    const int64_t blocks = std::min<int64_t>((rows + 255) / 256, 8 * static_cast<int64_t>(device_info().sms));
    fct_draws_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(a);
    if (!cuda_ok(cudaGetLastError(), "launch fct_draws")) return false;
  }
  // TMA staging needs a 16-byte aligned base and a row pitch that is a multiple of 16 bytes.
  const size_t esz = dt == L1S_BF16 ? 2 : 4;
  CUtensorMap mapA;
  const bool tma = reinterpret_cast<uintptr_t>(A) % 16 == 0 && (static_cast<uint64_t>(lda) * esz) % 16 == 0 &&
                   encode_tiled_2d(&mapA, dt == L1S_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                   A, static_cast<uint64_t>(n), static_cast<uint64_t>(pl.d), static_cast<uint64_t>(lda) * esz,
                                   kColW, kTmaBoxRows, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (tma) {
    const bool full = pl.log2s == 10;
    const void* fn = dt == L1S_BF16 ? (full ? reinterpret_cast<const void*>(&fct_embed_cols_tma_kernel<uint16_t, true>)
                                            : reinterpret_cast<const void*>(&fct_embed_cols_tma_kernel<uint16_t, false>))
                                    : (full ? reinterpret_cast<const void*>(&fct_embed_cols_tma_kernel<float, true>)
                                            : reinterpret_cast<const void*>(&fct_embed_cols_tma_kernel<float, false>));
    const size_t smem = cols_tma_smem_bytes(pl.r1);
    void* targs[] = {&mapA, &a};
    if (!allow_dynamic_smem(reinterpret_cast<const void*>(fn), smem, "cudaFuncSetAttribute(fct_embed_cols_tma)") ||
        !cuda_ok(cudaLaunchKernel(fn, dim3(pl.fct_ctas, pl.fct_cols), dim3(kTmaThreads), targs, smem, st),
                 "launch fct_embed_cols_tma"))
      return false;
  } else {
    set_error("");
    const void* fn = fct_cols_kernel(dt, pl.log2s == 10);
    const size_t smem = fct_cols_smem_bytes(pl.r1);
    if (!allow_dynamic_smem(reinterpret_cast<const void*>(fn), smem, "cudaFuncSetAttribute(fct_embed_cols)") ||
        !cuda_ok(cudaLaunchKernel(fn, dim3(pl.fct_ctas, pl.fct_cols), dim3(kColThreads), args, smem, st),
                 "launch fct_embed_cols"))
      return false;
  }
  // The b column: its blocks are a function of this launch's n (the reduction reads them).
  const size_t bsmem = bcol_smem_bytes(pl.r1);
  const void* fb = reinterpret_cast<const void*>(&fct_embed_bcol_kernel);
  if (!allow_dynamic_smem(reinterpret_cast<const void*>(fb), bsmem, "cudaFuncSetAttribute(fct_embed_bcol)") ||
      !cuda_ok(cudaLaunchKernel(fb, dim3(bcol_ctas(pl.n)), dim3(kBcolThreads), args, bsmem, st),
               "launch fct_embed_bcol"))
    return false;
  count_launch(3);
  return true;
}

bool launch_fct_cols_reduce(const Plan& pl, const l1s_params* p, float* pix, unsigned char* ws, cudaStream_t st,
                            double* pi2_out) {
  const float* parts = reinterpret_cast<const float*>(ws + pl.off_partials);
  const float* parts_b = parts + static_cast<size_t>(pl.fct_cols) * pl.fct_ctas * pl.r1 * kColW;
  dim3 grid((pl.r1 * kColW + 31) / 32, pl.fct_cols + 1);
  fct_reduce_cols_kernel<<<grid, 1024, 0, st>>>(parts, parts_b, pl.fct_ctas, bcol_ctas(pl.n), pl.fct_cols, pl.r1,
                                                pl.d, pix, reinterpret_cast<uint32_t*>(ws + pl.off_status),
                                                make_key(p->seed), p->problem_id, pl.q * pl.r2, pl.r2,
                                                p->variant == 1 ? 1 : 0, pl.pi2_neg_lo, pl.pi2_neg_hi, pi2_out);
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch fct_reduce_cols");
}

}  // namespace l1s
