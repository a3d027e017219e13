// Phase 2 for BF16 A on the tensor cores (Figure 2, steps 4-5, mixed-precision form):
//   λ_i = lower median_j |A_i·M_A[:, j] + (−b_i)·M_b[j]|,
// M_A = the first d rows of M = R⁻¹Π2 rounded to FP32 then BF16, M_b = M's last row in
// FP32.  The product A·M_A runs as tcgen05.mma (kind::f16, BF16 × BF16 → FP32 in
// tensor memory, M = 128 rows, N = r2 ∈ {16, 32}, K = 32 or 64 in steps of 16, the
// columns of A beyond d read as zeros by the tensor map, the rows of M_Aᵀ beyond d
// zero); the b column, |·| and the median stay in FP32 registers.
//
// Roles of the six warps of a persistent thread block (three per SM, so that twelve
// epilogue warps share each SM):
//   warp 0  TMA producer: 128-row tiles of A (2-D tensor map, 64-byte swizzle for K = 32,
//           128-byte for K = 64) into a ring of shared-memory stages, and the BF16 M_Aᵀ
//           tile once;
//   warp 1  allocates the tensor memory (two accumulators of N columns) and, from one
//           thread, issues the MMAs of a tile and commits them to mbarriers that free the
//           stage and publish the accumulator;
//   warps 2-5  epilogue: each reads its 32 TMEM lanes (rows) with tcgen05.ld, adds the
//           FP32 b term, takes |·| and the lower median by a sorting network, writes λ
//           and accumulates Σλ.
// Every mbarrier wait is bounded; a timeout raises the TIMEOUT status bit and the
// block stops issuing work, pauses (bounded) so that its copies and MMAs in flight can
// land, releases its tensor memory and returns.
#include <cuda.h>
#include <float.h>

#include <utility>

#include "l1s_common.cuh"

namespace l1s {

constexpr int kTcTile = 128;           // rows per MMA (M)
constexpr int kTcStages = 4;
constexpr int kTcThreads = 192;

template <int K, int N>
struct TcShape {
  static constexpr uint32_t kTileBytes = kTcTile * K * 2;            // one stage of A
  static constexpr uint32_t kBBytes = N * K * 2;                     // M_Aᵀ
  static constexpr uint32_t kTmemCols = 2 * N < 32 ? 32 : 2 * N;     // two accumulators
  static constexpr uint32_t kAtom = 8 * K * 2;                       // 8 swizzled rows
  static constexpr uint64_t kLayout = K == 64 ? 2 : 4;               // 128- or 64-byte swizzle
};

// ----------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand in the swizzled layout that the tensor
// map writes (8-row atoms of 8·K·2 bytes, 64-byte swizzle for K = 32 and 128-byte for
// K = 64), version 1.
template <int K>
__device__ __forceinline__ uint64_t smem_desc_sw(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = (addr >> 4) & 0x3FFFull;                          // start address
  d |= 1ull << 16;                                               // leading byte offset (unused for this layout)
  d |= static_cast<uint64_t>(TcShape<K, 16>::kAtom >> 4) << 32;  // stride byte offset: next 8-row atom
  d |= 1ull << 46;                                               // descriptor version
  d |= TcShape<K, 16>::kLayout << 61;                            // swizzle mode
  return d;
}

// Instruction descriptor for kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[N]) {
  if constexpr (N == 32) tmem_ld32(taddr, r);
  else tmem_ld16(taddr, r);
}

// Median network (same construction as the FP32 λ kernel).
template <int P>
struct TcNet {
  int lo[1024], hi[1024], count;
  constexpr TcNet() : lo(), hi(), count(0) {
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
struct TcNetOf {
  static constexpr TcNet<P> value{};
};
template <int P, int I>
__device__ __forceinline__ void tc_cmpx(float (&a)[P]) {
  constexpr int l = TcNetOf<P>::value.lo[I];
  constexpr int h = TcNetOf<P>::value.hi[I];
  const float x = a[l], y = a[h];
  a[l] = fminf(x, y);
  a[h] = fmaxf(x, y);
}
template <int P, int... I>
__device__ __forceinline__ void tc_apply(float (&a)[P], std::integer_sequence<int, I...>) {
  (tc_cmpx<P, I>(a), ...);
}

struct TcArgs {
  const float* b;
  int64_t n;
  int64_t tiles;
  float* lam;
  double* block_sums;
  uint32_t* flags;
  float* raw;         // optional: the 32 accumulator columns of every row (checks of the MMA layout)
  const float* mb;    // M's last row (the b column), FP32, r2 values
};

template <int K, int N>
__global__ void __launch_bounds__(kTcThreads, 3) lambda_tc_kernel(const __grid_constant__ CUtensorMap mapA,
                                                                  const __grid_constant__ CUtensorMap mapB,
                                                                  const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ uint64_t full[kTcStages], empty[kTcStages], accfull[2], accempty[2], bfull;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ double wsum[4];
  // 1024-byte aligned tiles (the swizzle atom repeats every 512 bytes)
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem) + 1023) & ~uintptr_t(1023));
  unsigned char* stageA = base;
  using S = TcShape<K, N>;
  unsigned char* tileB = base + kTcStages * S::kTileBytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&accfull[k], 1);
      mbar_init(&accempty[k], 4);
    }
    mbar_init(&bfull, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(S::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      mbar_arrive_expect_tx(&bfull, S::kBBytes);
      tma_load_2d(tileB, &mapB, 0, 0, &bfull);
      int64_t i = 0;
      for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x, ++i) {
        const int s = static_cast<int>(i % kTcStages);
        const uint32_t ph = static_cast<uint32_t>((i / kTcStages) & 1);
        if (!mbar_wait_bounded(&empty[s], ph ^ 1u, kWaitCycles) || s_abort) {
          s_abort = 1;
          break;
        }
        mbar_arrive_expect_tx(&full[s], S::kTileBytes);
        tma_load_2d(stageA + s * S::kTileBytes, &mapA, 0, static_cast<int>(t * kTcTile), &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kTcTile, N);
      bool ok = mbar_wait_bounded(&bfull, 0, kWaitCycles);
      if (!ok) s_abort = 1;
      const uint64_t bdesc = smem_desc_sw<K>(tileB);
      int64_t i = 0;
      for (int64_t t = blockIdx.x; ok && t < a.tiles; t += gridDim.x, ++i) {
        const int s = static_cast<int>(i % kTcStages);
        const int acc = static_cast<int>(i & 1);
        if (!mbar_wait_bounded(&accempty[acc], static_cast<uint32_t>(((i >> 1) & 1) ^ 1), kWaitCycles) ||
            !mbar_wait_bounded(&full[s], static_cast<uint32_t>((i / kTcStages) & 1), kWaitCycles) || s_abort) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint64_t adesc = smem_desc_sw<K>(stageA + s * S::kTileBytes);
        const uint32_t d = tmem + static_cast<uint32_t>(acc * N);
        // K in steps of 16: step k starts 32·k bytes into each swizzled row.
#pragma unroll
        for (int k = 0; k < K / 16; ++k) mma_bf16(d, adesc + 2 * k, bdesc + 2 * k, idesc, k > 0 ? 1u : 0u);
        mma_commit(&empty[s]);
        mma_commit(&accfull[acc]);
      }
    }
  } else {
    // epilogue: warps 2..5; warp w reads TMEM lanes 32·(w mod 4) … +31
    const int quarter = warp & 3;
    float sum_s = 0.f, sum_c = 0.f;
    float mb[N];
#pragma unroll
    for (int j = 0; j < N; ++j) mb[j] = __ldg(a.mb + j);   // M's last row (b column), FP32
    int64_t i = 0;
    for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x, ++i) {
      const int acc = static_cast<int>(i & 1);
      if (!mbar_wait_bounded(&accfull[acc], static_cast<uint32_t>((i >> 1) & 1), kWaitCycles) || s_abort) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
      uint32_t r[N];
      tmem_ld<N>(tmem + static_cast<uint32_t>(acc * N) + (static_cast<uint32_t>(quarter * 32) << 16), r);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[acc]);
      const int64_t row = t * kTcTile + quarter * 32 + lane;
      if (a.raw && row < a.n) {
#pragma unroll
        for (int j = 0; j < N; ++j) a.raw[row * N + j] = __uint_as_float(r[j]);
      }
      if (row < a.n) {
        const float xb = -__ldg(a.b + row);
        float v[N];
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = fabsf(fmaf(xb, mb[j], __uint_as_float(r[j])));
        tc_apply<N>(v, std::make_integer_sequence<int, TcNetOf<N>::value.count>{});
        const float med = v[(N - 1) / 2];
        a.lam[row] = med;
        const float tt = sum_s + med, bp = tt - sum_s;
        sum_c += (sum_s - (tt - bp)) + (med - bp);
        sum_s = tt;
      }
    }
    // Σλ of this block: fixed-order reduction over the 128 epilogue threads
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, sum_s, off);
      const float c2 = __shfl_xor_sync(0xffffffffu, sum_c, off);
      const float tt = sum_s + s2, bp = tt - sum_s;
      const float e = (sum_s - (tt - bp)) + (s2 - bp);
      sum_s = tt;
      sum_c = (sum_c + c2) + e;
    }
    if (lane == 0) wsum[warp - 2] = static_cast<double>(sum_s) + static_cast<double>(sum_c);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    a.block_sums[blockIdx.x] = ((wsum[0] + wsum[1]) + wsum[2]) + wsum[3];
    if (s_abort) raise_flag(a.flags, L1S_ERR_TIMEOUT);
  }
  if (s_abort) {
    // Give copies and MMAs still in flight time to land (bounded) before releasing memory.
    if (threadIdx.x == 0) {
      const long long t0 = clock64();
      while (clock64() - t0 < 20000000LL) {
      }
    }
    __syncthreads();
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::kTmemCols) : "memory");
  }
}

// M_Aᵀ in BF16 ([r2][K], K-major for the MMA's B operand) from the FP32 M (row-major q × r2);
// entries k ≥ d are zero (they meet the zero columns the tensor map reads beyond d).
__global__ void m_bf16_kernel(const float* __restrict__ m32, int d, int K, int r2, uint16_t* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K * r2) return;
  const int n = e / K, k = e - n * K;
  if (k >= d) {
    out[e] = 0;
    return;
  }
  const float v = m32[k * r2 + n];
  // round to nearest even (M is finite here)
  const uint32_t u = __float_as_uint(v);
  const uint32_t rounded = u + 0x7FFFu + ((u >> 16) & 1u);
  out[e] = static_cast<uint16_t>(rounded >> 16);
}

// ----------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

static bool encode_bf16_2d(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t row_bytes,
                           uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swizzle) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return set_error("cuTensorMapEncodeTiled is not available"), false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error("cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r)), false;
  return true;
}

// A 2-D tiled tensor map over a row-major matrix (rows × cols elements, row pitch row_bytes),
// box of box_cols × box_rows elements, rows and columns outside the matrix read as zeros.
bool encode_tiled_2d(CUtensorMap* map, CUtensorMapDataType dtype, const void* base, uint64_t rows, uint64_t cols,
                     uint64_t row_bytes, uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swizzle) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return set_error("cuTensorMapEncodeTiled is not available"), false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error("cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r)), false;
  return true;
}

// K of the tensor-core form for d columns (0 when it does not apply).
static int tc_k_for(int d) { return d > 16 && d <= 32 ? 32 : (d > 32 && d <= 64 ? 64 : 0); }

// The tensor-core λ applies to BF16 A with 16 < d ≤ 64, r2 ∈ {16, 32}, a 16-byte aligned
// base and a row pitch that is a multiple of 16 bytes.
bool lambda_tc_applies(int d, int r2, int64_t lda, const void* A, l1s_dtype dt) {
  return dt == L1S_BF16 && tc_k_for(d) && (r2 == 16 || r2 == 32) && (lda * 2) % 16 == 0 &&
         (reinterpret_cast<uintptr_t>(A) % 16 == 0);
}

template <int K, int N>
static size_t tc_smem_bytes() {
  return 1024 + kTcStages * TcShape<K, N>::kTileBytes + TcShape<K, N>::kBBytes;
}

template <int K, int N>
static bool launch_tc(const TcArgs& args, const void* A, int64_t lda, int d, const uint16_t* mt, int blocks,
                      cudaStream_t st) {
  CUtensorMap mapA, mapB;
  const CUtensorMapSwizzle sw = K == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  if (!encode_bf16_2d(&mapA, A, static_cast<uint64_t>(args.n), static_cast<uint64_t>(d), static_cast<uint64_t>(lda) * 2,
                      K, kTcTile, sw) ||
      !encode_bf16_2d(&mapB, mt, N, K, K * 2, K, N, sw))
    return false;
  const size_t smem = tc_smem_bytes<K, N>();
  if (!allow_dynamic_smem(reinterpret_cast<const void*>(lambda_tc_kernel<K, N>), smem, "lambda_tc smem"))
    return false;
  lambda_tc_kernel<K, N><<<blocks, kTcThreads, smem, st>>>(mapA, mapB, args);
  return true;
}

// Bytes of the BF16 M_Aᵀ tile for (d, r2).
size_t lambda_tc_mt_bytes(int d, int r2) { return static_cast<size_t>(tc_k_for(d)) * r2 * 2; }

// m32 is M in FP32 (q × r2 in device memory); mt_bf16 is workspace for M_Aᵀ (r2 × K BF16).
bool launch_lambda_tc(int64_t n, int d, int r2, const void* A, int64_t lda, const float* b, const float* m32,
                      uint16_t* mt_bf16, float* lam, double* block_sums, int blocks, uint32_t* flags, cudaStream_t st) {
  const int K = tc_k_for(d);
  m_bf16_kernel<<<(K * r2 + 255) / 256, 256, 0, st>>>(m32, d, K, r2, mt_bf16);
  count_launch(1);
  if (!cuda_ok(cudaGetLastError(), "launch m_bf16")) return false;
  TcArgs args;
  args.b = b;
  args.n = n;
  args.tiles = (n + kTcTile - 1) / kTcTile;
  args.lam = lam;
  args.block_sums = block_sums;
  args.flags = flags;
  args.raw = nullptr;
  args.mb = m32 + static_cast<size_t>(d) * r2;
  bool ok;
  if (K == 32) ok = r2 == 32 ? launch_tc<32, 32>(args, A, lda, d, mt_bf16, blocks, st)
                             : launch_tc<32, 16>(args, A, lda, d, mt_bf16, blocks, st);
  else ok = r2 == 32 ? launch_tc<64, 32>(args, A, lda, d, mt_bf16, blocks, st)
                     : launch_tc<64, 16>(args, A, lda, d, mt_bf16, blocks, st);
  if (!ok) return false;
  count_launch(1);
  return cuda_ok(cudaGetLastError(), "launch lambda_tc");
}

}  // namespace l1s
