// Phase 1: the FCT1 embedding Π1·X = 4·B·C·H̃·D·X (§3.1, FCT1 construction;
// Figure 2, steps 1-2), X = [A, −b].
//
// One thread block owns a slice of columns of X and walks over s-row blocks
// β (grid-stride).  Per block:
//   1. one Philox call per row gives the row's sign σ, the buckets of its two
//      virtual rows and their Cauchy scales (kept in shared memory);
//   2. the s × w tile of X is read with coalesced loads, the sign is applied
//      on load, and the identity half of G_s = [H_s; I_s] is scattered at once:
//      P[h_I(i), c] += 4·c_I(i)·σ_i·x_ic;
//   3. the Sylvester–Hadamard transform of each column runs in shared memory
//      as two passes of radix-2^k butterflies held in registers (k = ⌈log2 s / 2⌉),
//      and the second pass scatters the Hadamard half straight from registers:
//      P[h_H(i), c] += 4·c_H(i)/√s·(H_s z)_ic.
// P, the block's r1 × w partial of Π1X, lives in shared memory (B's hashed sum
// as a shared-memory reduction, no global atomics).  A second kernel adds the
// per-block partials in a fixed order.
#include "l1s_common.cuh"

namespace l1s {

struct FctArgs {
  const void* A;
  int64_t lda;
  const float* b;
  int64_t n;
  int d, q, r1, width;
  int64_t nblocks;
  Key2 key;
  uint32_t problem;
  int64_t row_offset;
  int sign_flip;
  float inv_sqrt_s;
  float* partials;  // [slices][gridDim.x][r1][width]
  uint32_t* flags;
};

constexpr int kFctThreads = 256;

// One radix-2^K pass over index bits [LO, LO+K) of every column of the tile.
// tile is s × W (row-major, row stride W).  LAST: scatter instead of store.
template <int LOG2S, int K, int LO, bool LAST>
__device__ __forceinline__ void fwht_pass(float* __restrict__ tile, float* __restrict__ part,
                                          const int* __restrict__ hH, const float* __restrict__ wH,
                                          int W, int wcols) {
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
    if constexpr (!LAST) {
#pragma unroll
      for (int j = 0; j < G; ++j) tile[(base + (j << LO)) * W + c] = v[j];
    } else {
      if (c < wcols) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int row = base + (j << LO);
          atomicAdd(&part[hH[row] * W + c], wH[row] * v[j]);
        }
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

template <int LOG2S, typename TA>
__global__ void __launch_bounds__(kFctThreads) fct_embed_kernel(const FctArgs a) {
  constexpr int S = 1 << LOG2S;
  constexpr int K1 = LOG2S / 2;          // first pass: bits [0, K1)
  constexpr int K2 = LOG2S - K1;         // second pass: bits [K1, LOG2S)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int W = a.width;
  const int c0 = blockIdx.y * W;
  const int wcols = min(W, a.q - c0);
  float* part = reinterpret_cast<float*>(smem_raw);
  float* tile = part + a.r1 * W;
  int* hH = reinterpret_cast<int*>(tile + S * W);
  int* hI = hH + S;
  float* wH = reinterpret_cast<float*>(hI + S);
  float* wI = wH + S;
  float* sg = wI + S;
  const TA* A = static_cast<const TA*>(a.A);

  for (int i = threadIdx.x; i < a.r1 * W; i += blockDim.x) part[i] = 0.f;
  bool finite = true;
  const int step = blockDim.x;
  const int di = step / W, dcol = step - di * W;

  for (int64_t blk = blockIdx.x; blk < a.nblocks; blk += gridDim.x) {
    const int64_t row0 = blk * S;
    __syncthreads();  // the previous block is done with tile and draws
    for (int i = threadIdx.x; i < S; i += step) {
      const uint64_t grow = static_cast<uint64_t>(a.row_offset + row0 + i);
      const uint4 o = draw_row(a.key, grow, a.problem, kStreamFct);
      hH[i] = bucket_of(o.x, a.r1);
      hI[i] = bucket_of(o.z, a.r1);
      wH[i] = 4.f * cauchy_f32(o.y >> 8) * a.inv_sqrt_s;
      wI[i] = 4.f * cauchy_f32(o.w >> 8);
      sg[i] = (a.sign_flip && (o.w & 1u)) ? -1.f : 1.f;
    }
    __syncthreads();
    {
      int i = threadIdx.x / W;
      int c = threadIdx.x - i * W;
      for (int e = threadIdx.x; e < S * W; e += step) {
        const int64_t row = row0 + i;
        const int col = c0 + c;
        float x = 0.f;
        if (row < a.n && c < wcols) {
          x = (col < a.d) ? load_elem<TA>(A + row * a.lda + col) : -__ldg(a.b + row);
          finite &= isfinite(x);
        }
        const float z = sg[i] * x;
        tile[e] = z;
        if (c < wcols) atomicAdd(&part[hI[i] * W + c], wI[i] * z);
        c += dcol;
        i += di;
        if (c >= W) {
          c -= W;
          ++i;
        }
      }
    }
    __syncthreads();
    if constexpr (LOG2S <= 1) {
      fwht_pass<LOG2S, LOG2S, 0, true>(tile, part, hH, wH, W, wcols);
    } else {
      fwht_pass<LOG2S, K1, 0, false>(tile, part, hH, wH, W, wcols);
      __syncthreads();
      fwht_pass<LOG2S, K2, K1, true>(tile, part, hH, wH, W, wcols);
    }
  }
  __syncthreads();
  float* out = a.partials + (static_cast<size_t>(blockIdx.y) * gridDim.x + blockIdx.x) * a.r1 * W;
  for (int i = threadIdx.x; i < a.r1 * W; i += blockDim.x) out[i] = part[i];
  if (!finite) raise_flag(a.flags, L1S_ERR_NONFINITE);
}

// Fixed-order sum of the per-block partials: PiX[r][c0+c] = Σ_blocks partial[r][c].
// Block = 32 warps; warp w adds partials w, w+32, …; warp 0 then adds the 32
// warp sums in order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(1024) fct_reduce_kernel(const float* __restrict__ partials, int ctas,
                                                          int r1, int W, int q, float* __restrict__ pix,
                                                          uint32_t* flags) {
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
template <typename TA>
static const void* fct_kernel_for(int log2s) {
  switch (log2s) {
    case 0: return reinterpret_cast<const void*>(&fct_embed_kernel<0, TA>);
    case 1: return reinterpret_cast<const void*>(&fct_embed_kernel<1, TA>);
    case 2: return reinterpret_cast<const void*>(&fct_embed_kernel<2, TA>);
    case 3: return reinterpret_cast<const void*>(&fct_embed_kernel<3, TA>);
    case 4: return reinterpret_cast<const void*>(&fct_embed_kernel<4, TA>);
    case 5: return reinterpret_cast<const void*>(&fct_embed_kernel<5, TA>);
    case 6: return reinterpret_cast<const void*>(&fct_embed_kernel<6, TA>);
    case 7: return reinterpret_cast<const void*>(&fct_embed_kernel<7, TA>);
    case 8: return reinterpret_cast<const void*>(&fct_embed_kernel<8, TA>);
    case 9: return reinterpret_cast<const void*>(&fct_embed_kernel<9, TA>);
    case 10: return reinterpret_cast<const void*>(&fct_embed_kernel<10, TA>);
    case 11: return reinterpret_cast<const void*>(&fct_embed_kernel<11, TA>);
    case 12: return reinterpret_cast<const void*>(&fct_embed_kernel<12, TA>);
    default: return nullptr;
  }
}

const void* fct_kernel(int log2s, l1s_dtype dt) {
  return dt == L1S_BF16 ? fct_kernel_for<uint16_t>(log2s) : fct_kernel_for<float>(log2s);
}

size_t fct_smem_bytes(int s, int r1, int width) {
  return static_cast<size_t>(r1) * width * 4 + static_cast<size_t>(s) * width * 4 +
         static_cast<size_t>(s) * 20;
}

int fct_threads() { return kFctThreads; }

bool launch_fct(const Plan& pl, const void* A, int64_t lda, l1s_dtype dt, const float* b,
                const l1s_params* p, float* pix, unsigned char* ws, cudaStream_t st) {
  FctArgs a;
  a.A = A;
  a.lda = lda;
  a.b = b;
  a.n = pl.n;
  a.d = pl.d;
  a.q = pl.q;
  a.r1 = pl.r1;
  a.width = pl.fct_width;
  a.nblocks = pl.nblocks;
  a.key = make_key(p->seed);
  a.problem = p->problem_id;
  a.row_offset = p->global_row_offset;
  a.sign_flip = p->sign_flip;
  a.inv_sqrt_s = static_cast<float>(1.0 / sqrt(static_cast<double>(pl.s)));
  a.partials = reinterpret_cast<float*>(ws + pl.off_partials);
  a.flags = reinterpret_cast<uint32_t*>(ws + pl.off_status);
  const void* fn = fct_kernel(pl.log2s, dt);
  if (!cuda_ok(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(pl.fct_smem)),
               "cudaFuncSetAttribute(fct_embed)"))
    return false;
  void* args[] = {&a};
  dim3 grid(pl.fct_ctas, pl.fct_slices);
  if (!cuda_ok(cudaLaunchKernel(fn, grid, dim3(pl.fct_threads), args, pl.fct_smem, st),
               "launch fct_embed"))
    return false;
  const int per = pl.r1 * pl.fct_width;
  dim3 rgrid((per + 31) / 32, pl.fct_slices);
  fct_reduce_kernel<<<rgrid, 1024, 0, st>>>(a.partials, pl.fct_ctas, pl.r1, pl.fct_width, pl.q, pix,
                                            a.flags);
  return cuda_ok(cudaGetLastError(), "launch fct_reduce");
}

}  // namespace l1s
