// FCT2 (§3.2, FCT2 construction), phase 1: Π1·X = (8/r1)·√(πt/(2s))·C·(H̃·X) with H̃
// block diagonal, one s × t fast Johnson–Lindenstrauss block G per t rows, and C an
// r1 × (ns/t) matrix of i.i.d. standard Cauchys (the slow transform, sct.cu, applied to
// the rows of H̃X).  G is a subsampled randomized Hadamard transform,
// G = √(t/s)·S·H_t·D: D_i = ±1 (stream 5, bit 0 of word 0 of call i), H_t the normalized
// Sylvester matrix, S the rows sel_r = ⌊word1·t/2^32⌋ of call r, so G_{r,i} =
// D_i·(−1)^{popcount(sel_r ∧ i)}/√s and one G serves every block.
//
// fjlt_kernel forms H̃X directly: output (block β, row r, column c) is the ±1 sum over the
// block's t rows of X, the sign of row i being D_i times the parity of sel_r ∧ i.  A thread
// block walks the blocks of X in a grid stride; it stages 64 rows of X at a time in shared
// memory and its threads own (r, c) outputs, eight a thread per pass (more passes when
// s·q > 2048).  The direct sum costs s sign-adds per element of X, against log2 t
// butterfly stages for all t rows of a Hadamard transform of which only s are kept;
// s·q ≤ 2048 keeps it one pass over X.
#include "l1s_common.cuh"

namespace l1s {

constexpr uint32_t kStreamFjlt = 5;
constexpr int kFjltThreads = 256;
constexpr int kFjltChunk = 64;   // rows of X staged per step
constexpr int kFjltOut = 8;      // outputs a thread accumulates per pass

struct FjltArgs {
  const void* A;
  int64_t lda;
  const float* b;
  int64_t n;
  int d, q, t, sf;
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
  float* xs = reinterpret_cast<float*>(sel + a.sf);        // [kFjltChunk][q]
  const int tid = threadIdx.x;
  for (int i = tid; i < max(a.t, a.sf); i += blockDim.x) {
    const uint4 o = philox4x32_10(make_uint4(static_cast<uint32_t>(i), 0u, a.problem, kStreamFjlt), a.key);
    if (i < a.t) sgn[i] = (o.x & 1u) ? 0x80000000u : 0u;
    if (i < a.sf) sel[i] = static_cast<int>(__umulhi(o.y, static_cast<uint32_t>(a.t)));
  }
  __syncthreads();
  const int q = a.q, outs = a.sf * q;
  const TA* A = static_cast<const TA*>(a.A);
  for (int64_t blk = blockIdx.x; blk < a.nblocks; blk += gridDim.x) {
    const int64_t r0 = blk * a.t;
    for (int o0 = 0; o0 < outs; o0 += kFjltThreads * kFjltOut) {
      float acc[kFjltOut];
      int orow[kFjltOut], ocol[kFjltOut], osel[kFjltOut];
#pragma unroll
      for (int k = 0; k < kFjltOut; ++k) {
        const int o = o0 + k * kFjltThreads + tid;
        orow[k] = o < outs ? o / q : -1;
        ocol[k] = o < outs ? o - (o / q) * q : 0;
        osel[k] = o < outs ? sel[orow[k]] : 0;
        acc[k] = 0.f;
      }
      for (int c0 = 0; c0 < a.t; c0 += kFjltChunk) {
        const int rows = min(kFjltChunk, a.t - c0);
        __syncthreads();                                   // the previous chunk is consumed
        for (int e = tid; e < rows * q; e += blockDim.x) {
          const int rr = e / q, cc = e - rr * q;
          const int64_t row = r0 + c0 + rr;
          float v = 0.f;
          if (row < a.n) v = cc < a.d ? load_elem<TA>(A + row * a.lda + cc) : -__ldg(a.b + row);
          xs[e] = v;
        }
        __syncthreads();
        float part[kFjltOut];
#pragma unroll
        for (int k = 0; k < kFjltOut; ++k) part[k] = 0.f;
        for (int i = 0; i < rows; ++i) {
          const int ii = c0 + i;
          const uint32_t di = sgn[ii];
#pragma unroll
          for (int k = 0; k < kFjltOut; ++k) {
            const uint32_t par = static_cast<uint32_t>(__popc(osel[k] & ii) & 1) << 31;
            const float x = xs[i * q + ocol[k]];
            part[k] += __uint_as_float(__float_as_uint(x) ^ di ^ par);
          }
        }
#pragma unroll
        for (int k = 0; k < kFjltOut; ++k) acc[k] += part[k];   // a chunk's sum, then the running one
      }
#pragma unroll
      for (int k = 0; k < kFjltOut; ++k) {
        if (orow[k] < 0) continue;
        const float y = acc[k] * a.inv_sqrt_sf;
        const int64_t yrow = blk * a.sf + orow[k];
        if (ocol[k] < a.d) a.Y[yrow * a.d + ocol[k]] = y;
        else a.bY[yrow] = -y;
      }
    }
  }
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
  const size_t smem = sizeof(uint32_t) * a.t + sizeof(int) * a.sf + sizeof(float) * kFjltChunk * a.q;
  const void* fn = dt == L1S_BF16 ? reinterpret_cast<const void*>(&fjlt_kernel<uint16_t>)
                                  : reinterpret_cast<const void*>(&fjlt_kernel<float>);
  if (!cuda_ok(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)),
               "cudaFuncSetAttribute(fjlt)"))
    return false;
  const int grid = static_cast<int>(std::min<int64_t>(a.nblocks, 8 * static_cast<int64_t>(device_info().sms)));
  void* args[] = {&a};
  if (!cuda_ok(cudaLaunchKernel(fn, dim3(grid), dim3(kFjltThreads), args, smem, st), "launch fjlt")) return false;
  count_launch(1);
  const int64_t ny = a.nblocks * a.sf;
  const float scale = static_cast<float>(8.0 / pl.r1 * sqrt(M_PI * pl.s / (2.0 * pl.fjlt_rows)));
  return launch_sct(pl, a.Y, pl.d, L1S_F32, a.bY, ny, (row_offset / pl.s) * pl.fjlt_rows, p, accumulate, ws, st,
                    scale);
}

}  // namespace l1s
