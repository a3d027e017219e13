// FCT2 (§3.2, FCT2 construction), phase 1: Π1·X = (8/r1)·√(πt/(2s))·C·(H̃·X) with H̃
// block diagonal, one s × t fast Johnson–Lindenstrauss block G per t rows, and C an
// r1 × (ns/t) matrix of i.i.d. standard Cauchys (the slow transform, sct.cu, applied to
// the rows of H̃X).  G is a subsampled randomized Hadamard transform,
// G = √(t/s)·S·H_t·D: D_i = ±1 (stream 5, bit 0 of word 0 of call i), H_t the normalized
// Sylvester matrix, S the rows sel_r = ⌊word1·t/2^32⌋ of call r, so G_{r,i} =
// D_i·(−1)^{popcount(sel_r ∧ i)}/√s and one G serves every block.
//
// fjlt_kernel forms H̃X with a fast Walsh–Hadamard transform per block: a thread block
// stages the block's t rows (a slice of at most W columns, W·t·4 bytes ≤ 160 KB) in shared
// memory with D applied, runs the log2 t radix-2 stages in place (one barrier a stage; the
// threads are (pair, column) lanes, so each stage's accesses are consecutive words), then
// writes the s rows sel_r scaled by 1/√s.  A block costs log2 t butterflies per element
// of X, where a direct sum over the sampled rows would cost s per element.
#include <algorithm>

#include "l1s_common.cuh"

namespace l1s {

constexpr uint32_t kStreamFjlt = 5;
constexpr int kFjltThreads = 256;

struct FjltArgs {
  const void* A;
  int64_t lda;
  const float* b;
  int64_t n;
  int d, q, t, sf;
  int width;    // columns of X per slice (blockIdx.y)
  Key2 key;
  uint32_t problem;
  int64_t nblocks;
  float inv_sqrt_sf;
  float* Y;     // rows of H̃X, columns 0 … d−1 (d a row)
  float* bY;    // G·b per row of H̃X (the slow transform reads −bY as the last column)
};

template <typename TA>
__global__ void __launch_bounds__(kFjltThreads) fjlt_kernel(const FjltArgs a) {
  extern __shared__ __align__(16) float fj_smem[];
  uint32_t* sgn = reinterpret_cast<uint32_t*>(fj_smem);   // [t]: D_i as a sign mask
  int* sel = reinterpret_cast<int*>(sgn + a.t);            // [sf]
  float* xs = reinterpret_cast<float*>(sel + a.sf);        // [t][wc], this slice's columns
  const int tid = threadIdx.x;
  for (int i = tid; i < max(a.t, a.sf); i += blockDim.x) {
    const uint4 o = philox4x32_10(make_uint4(static_cast<uint32_t>(i), 0u, a.problem, kStreamFjlt), a.key);
    if (i < a.t) sgn[i] = (o.x & 1u) ? 0x80000000u : 0u;
    if (i < a.sf) sel[i] = static_cast<int>(__umulhi(o.y, static_cast<uint32_t>(a.t)));
  }
  const int c0 = blockIdx.y * a.width;
  const int wc = min(a.width, a.q - c0);                   // columns of this slice
  const int lanes = kFjltThreads / wc;                     // (row or pair, column) lanes
  const int pl = tid / wc, cc = tid - pl * wc;
  const bool active = pl < lanes;
  const int col = c0 + cc;
  const TA* A = static_cast<const TA*>(a.A);
  for (int64_t blk = blockIdx.x; blk < a.nblocks; blk += gridDim.x) {
    const int64_t r0 = blk * a.t;
    __syncthreads();                                       // the previous block's rows are written out
    if (active)
      for (int rr = pl; rr < a.t; rr += lanes) {
        const int64_t row = r0 + rr;
        float v = 0.f;
        if (row < a.n) v = col < a.d ? load_elem<TA>(A + row * a.lda + col) : -__ldg(a.b + row);
        xs[rr * wc + cc] = __uint_as_float(__float_as_uint(v) ^ sgn[rr]);   // D·x
      }
    for (int h = 1; h < a.t; h <<= 1) {
      __syncthreads();
      if (active)
        for (int p = pl; p < (a.t >> 1); p += lanes) {
          const int i = ((p & ~(h - 1)) << 1) | (p & (h - 1));
          float* lo = xs + i * wc + cc;
          float* hi = lo + h * wc;
          const float x = *lo, y = *hi;
          *lo = x + y;
          *hi = x - y;
        }
    }
    __syncthreads();
    if (active)
      for (int r = pl; r < a.sf; r += lanes) {
        const float y = xs[sel[r] * wc + cc] * a.inv_sqrt_sf;
        const int64_t yrow = blk * a.sf + r;
        if (col < a.d) a.Y[yrow * a.d + col] = y;
        else a.bY[yrow] = -y;
      }
  }
}

// Columns per slice: as many as fit 160 KB of shared memory next to the draws, and no more
// than there are threads.
static int fjlt_width(int t, int q) {
  const int fit = std::max(1, static_cast<int>((160 * 1024) / (4 * static_cast<int64_t>(t))));
  return std::min(std::min(q, fit), kFjltThreads);
}

bool launch_sct(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n,
                int64_t row_offset, const l1s_params* p, bool accumulate, unsigned char* ws, cudaStream_t st,
                float scale);

// One FCT2 launch over rows [0, n) of A and b whose global ids start at row_offset (a
// multiple of t): H̃X into the workspace, then the slow transform on its rows.
bool launch_fct2(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n,
                 int64_t row_offset, const l1s_params* p, bool accumulate, unsigned char* ws, cudaStream_t st) {
  FjltArgs a;
  a.A = A;
  a.lda = lda;
  a.b = b;
  a.n = n;
  a.d = pl.d;
  a.q = pl.q;
  a.t = pl.s;
  a.sf = pl.fjlt_rows;
  a.key = make_key(p->seed);
  a.problem = p->problem_id;
  a.nblocks = (n + pl.s - 1) / pl.s;
  a.inv_sqrt_sf = static_cast<float>(1.0 / sqrt(static_cast<double>(pl.fjlt_rows)));
  a.Y = reinterpret_cast<float*>(ws + pl.off_fjlt);
  a.bY = a.Y + static_cast<size_t>(pl.fjlt_n) * pl.d;
  a.width = fjlt_width(a.t, a.q);
  const int slices = (a.q + a.width - 1) / a.width;
  const size_t smem = sizeof(uint32_t) * a.t + sizeof(int) * a.sf + sizeof(float) * static_cast<size_t>(a.t) * a.width;
  const void* fn = dt == L1S_BF16 ? reinterpret_cast<const void*>(&fjlt_kernel<uint16_t>)
                                  : reinterpret_cast<const void*>(&fjlt_kernel<float>);
  if (!allow_dynamic_smem(reinterpret_cast<const void*>(fn), smem, "cudaFuncSetAttribute(fjlt)"))
    return false;
  const int grid = static_cast<int>(std::min<int64_t>(a.nblocks, 8 * static_cast<int64_t>(device_info().sms)));
  void* args[] = {&a};
  if (!cuda_ok(cudaLaunchKernel(fn, dim3(grid, slices), dim3(kFjltThreads), args, smem, st), "launch fjlt"))
    return false;
  count_launch(1);
  const int64_t ny = a.nblocks * a.sf;
  const float scale = static_cast<float>(8.0 / pl.r1 * sqrt(M_PI * pl.s / (2.0 * pl.fjlt_rows)));
  return launch_sct(pl, a.Y, pl.d, L1S_F32, a.bY, ny, (row_offset / pl.s) * pl.fjlt_rows, p, accumulate, ws, st,
                    scale);
}

}  // namespace l1s
