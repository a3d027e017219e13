// The slow Cauchy transform: Π1·X = (4/r1)·C·X with C an r1 × n matrix of i.i.d.
// standard Cauchy variables (§3, the theorem of Sohler and Woodruff the paper restates:
// ‖y‖₁ ≤ (4/r1)‖C·y‖₁ ≤ κ'‖y‖₁ on a d-dimensional subspace for r1 = O(d log d); §6.3
// conditions with it).  C is never stored: entry (r, i), r = 4g + w, is word w of the
// Philox call with counter (i_lo, (i_hi mod 2^16) + g·2^16, problem, 4) through the same
// 24-bit Cauchy map as the other draws.
//
// The product is a dense contraction whose cost is drawing the r1·n variates (one Philox
// call per four of them); the q FMAs each variate feeds are the smaller part.  A thread
// owns four output rows (one call per input row) and QW columns of X (QW = 5, 9 or 17;
// wider X runs as several column slices): 4·QW FP32 accumulators.  A block is 8 warps;
// warp l takes rows l, l + 8, … of each 64-row tile of X, which the block stages in shared
// memory, and its 32 lanes are 32 groups of output rows, so every lane reads the same row
// of the tile (a broadcast).  Blocks split the rows of X into contiguous chunks and the
// output rows into bands of 128; at the end a block adds its 8 warps' accumulators in a
// fixed order, scales by 4/r1 and writes its band of the per-chunk partial, which the
// phase-1 reduction sums in a fixed order.
#include <algorithm>

#include "l1s_common.cuh"

namespace l1s {

constexpr uint32_t kStreamSct = 4;
constexpr int kSctThreads = 256;
constexpr int kSctLanes = 8;             // warps = row lanes
constexpr int kSctBand = 4 * 32;         // output rows per block
constexpr int kSctTile = 64;             // rows of X per staged tile

struct SctArgs {
  const void* A;
  int64_t lda;
  const float* b;
  int64_t n;
  int d, r1;
  Key2 key;
  uint32_t problem;
  int64_t row_offset;
  float scale;              // 4/r1
  int64_t chunk;            // rows of X per block
  float* partials;          // [slices][gridDim.x][r1][QW]
  int accumulate;           // 1: add to the partials of an earlier launch over other rows
};

template <int QW>
__host__ __device__ constexpr size_t sct_smem_floats() {
  return static_cast<size_t>(kSctLanes) * kSctBand * QW > static_cast<size_t>(kSctTile) * QW
             ? static_cast<size_t>(kSctLanes) * kSctBand * QW
             : static_cast<size_t>(kSctTile) * QW;
}

template <int QW, typename TA>
__global__ void __launch_bounds__(kSctThreads, 2) sct_embed_kernel(const SctArgs a) {
  extern __shared__ __align__(16) float sct_smem[];
  const int tid = threadIdx.x, lane = tid & 31, lrow = tid >> 5;
  const int g = blockIdx.y * 32 + lane;                 // output rows 4g … 4g + 3
  const int c0 = blockIdx.z * QW;
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * a.chunk;
  const int64_t i1 = min(a.n, i0 + a.chunk);
  const TA* A = static_cast<const TA*>(a.A);
  float acc[4][QW];
#pragma unroll
  for (int w = 0; w < 4; ++w)
#pragma unroll
    for (int c = 0; c < QW; ++c) acc[w][c] = 0.f;
  float* tile = sct_smem;
  const uint32_t gbits = static_cast<uint32_t>(g) << 16;
  for (int64_t t0 = i0; t0 < i1; t0 += kSctTile) {
    __syncthreads();
    const int rows = i1 - t0 < kSctTile ? static_cast<int>(i1 - t0) : kSctTile;
    for (int e = tid; e < kSctTile * QW; e += kSctThreads) {
      const int rr = e / QW, cc = e - rr * QW;
      const int col = c0 + cc;
      float v = 0.f;
      if (rr < rows) {
        const int64_t row = t0 + rr;
        if (col < a.d) v = load_elem<TA>(A + row * a.lda + col);
        else if (col == a.d) v = -__ldg(a.b + row);
      }
      tile[e] = v;
    }
    __syncthreads();
    for (int rr = lrow; rr < rows; rr += kSctLanes) {
      const uint64_t grow = static_cast<uint64_t>(a.row_offset + t0 + rr);
      const uint4 o = philox4x32_10(
          make_uint4(static_cast<uint32_t>(grow), (static_cast<uint32_t>(grow >> 32) & 0xFFFFu) | gbits, a.problem,
                     kStreamSct),
          a.key);
      const float cw[4] = {cauchy_f32(o.x >> 8), cauchy_f32(o.y >> 8), cauchy_f32(o.z >> 8), cauchy_f32(o.w >> 8)};
      const float* xr = tile + rr * QW;
#pragma unroll
      for (int c = 0; c < QW; ++c) {
        const float x = xr[c];
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[w][c] = fmaf(cw[w], x, acc[w][c]);
      }
    }
  }
  // The 8 row lanes' accumulators of the block's band, added in a fixed order.
  __syncthreads();
  float* red = sct_smem;                                  // [lane row][band row][QW]
#pragma unroll
  for (int w = 0; w < 4; ++w)
#pragma unroll
    for (int c = 0; c < QW; ++c) red[(lrow * kSctBand + 4 * lane + w) * QW + c] = acc[w][c];
  __syncthreads();
  float* out = a.partials + (static_cast<size_t>(blockIdx.z) * gridDim.x + blockIdx.x) * a.r1 * QW;
  for (int e = tid; e < kSctBand * QW; e += kSctThreads) {
    float s = 0.f;
#pragma unroll
    for (int l = 0; l < kSctLanes; ++l) s += red[l * kSctBand * QW + e];
    const int r = blockIdx.y * kSctBand + e / QW;
    if (r < a.r1) {
      const size_t o = static_cast<size_t>(r) * QW + (e % QW);
      out[o] = (a.accumulate ? out[o] : 0.f) + s * a.scale;
    }
  }
}

// Columns per slice for q columns of X.
int sct_width(int q) { return q <= 5 ? 5 : (q <= 9 ? 9 : 17); }

// Blocks along the rows of X: two waves of two blocks per SM over all bands and slices.
int sct_ctas(int64_t n, int r1, int q, int sms) {
  const int w = sct_width(q);
  const int slices = (q + w - 1) / w;
  const int bands = (r1 + kSctBand - 1) / kSctBand;
  const int64_t want = std::max<int64_t>(1, (4 * static_cast<int64_t>(sms)) / (slices * bands));
  const int64_t tiles = (n + kSctTile - 1) / kSctTile;
  return static_cast<int>(std::max<int64_t>(1, std::min(want, tiles)));
}

template <int QW, typename TA>
static bool launch_sct_t(const SctArgs& a, dim3 grid, cudaStream_t st) {
  const size_t smem = sct_smem_floats<QW>() * sizeof(float);
  const void* fn = reinterpret_cast<const void*>(&sct_embed_kernel<QW, TA>);
  if (!allow_dynamic_smem(reinterpret_cast<const void*>(fn), smem, "cudaFuncSetAttribute(sct_embed)"))
    return false;
  void* args[] = {const_cast<SctArgs*>(&a)};
  return cuda_ok(cudaLaunchKernel(fn, grid, dim3(kSctThreads), args, smem, st), "launch sct_embed");
}

// One slow-transform launch over rows [0, n) of A and b whose global ids start at
// row_offset, writing (or adding to) the per-chunk partials of the plan, the product
// scaled by `scale` (4/r1 for the slow transform itself).
bool launch_sct(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n,
                int64_t row_offset, const l1s_params* p, bool accumulate, unsigned char* ws, cudaStream_t st,
                float scale) {
  SctArgs a;
  a.A = A;
  a.lda = lda;
  a.b = b;
  a.n = n;
  a.d = pl.d;
  a.r1 = pl.r1;
  a.key = make_key(p->seed);
  a.problem = p->problem_id;
  a.row_offset = row_offset;
  a.scale = scale;
  a.chunk = (n + pl.fct_ctas - 1) / pl.fct_ctas;
  a.partials = reinterpret_cast<float*>(ws + pl.off_partials);
  a.accumulate = accumulate ? 1 : 0;
  const dim3 grid(pl.fct_ctas, (pl.r1 + kSctBand - 1) / kSctBand, pl.fct_slices);
  bool ok;
  const bool bf = dt == L1S_BF16;
  switch (pl.fct_width) {
    case 5: ok = bf ? launch_sct_t<5, uint16_t>(a, grid, st) : launch_sct_t<5, float>(a, grid, st); break;
    case 9: ok = bf ? launch_sct_t<9, uint16_t>(a, grid, st) : launch_sct_t<9, float>(a, grid, st); break;
    default: ok = bf ? launch_sct_t<17, uint16_t>(a, grid, st) : launch_sct_t<17, float>(a, grid, st); break;
  }
  if (ok) count_launch(1);
  return ok;
}

}  // namespace l1s
