// Step 8 of Figure 2: x̂ = argmin_x ‖D·(A·x − b)‖₁ on the coreset, in FP64, and
// the objective ‖A·x − b‖₁ over all rows (problem statement, §4.2).
//
// The paper solves the small problem by linear programming; here it is solved
// by iteratively reweighted least squares: with residuals r_k = X_k·[x; 1] of
// the coreset rows X_k = [A_k, −b_k] and sampling weights w_k,
//   x ← argmin Σ_k ω_k r_k²,  ω_k = w_k / max(|r_k|, η),  η = 10⁻⁶·Σ w|r| / Σ w,
// starting from ω = w.  The iterate with the smallest objective is kept; the
// loop stops early once the objective changes by less than 10⁻¹² relative.
// An ℓ1 optimum is attained at a vertex where d residuals vanish, so the result
// is then finished by simplex pivots of the LAD linear program, starting from the
// d rows with the smallest |r_k| whose A parts are linearly independent, until the
// dual multipliers certify the vertex
// optimal; the vertex replaces the iterate when its objective is not larger.
//
// Kernels: irls_accum (many blocks: objective and the weighted normal
// equations, per-block partials), irls_step (one block: fixed-order sum,
// Cholesky solve, bookkeeping), irls_residuals (many blocks), irls_polish (one
// block: the vertex finish), objective (many blocks + fixed-order finish).  A device flag turns
// the remaining iterations into no-ops after convergence, so the whole solve is
// enqueued without host synchronisation.
#include "l1s_common.cuh"

namespace l1s {

constexpr int kIrlsThreads = 256;
constexpr int kIrlsTile = 64;
constexpr int kIrlsSlots = 33;  // ⌈(129·130/2)/256⌉ entries per thread at most

// State kept in the workspace between kernels.
struct IrlsState {
  double x[kMaxD + 1];      // current iterate, x[d] = 1
  double best_x[kMaxD + 1];
  double best_f;
  double w_total;
};

struct IrlsArgs {
  const double* X;        // coreset rows, q per row
  const double* w;
  const int64_t* count;
  int64_t capacity;
  int d, q;
  double* partials;       // [blocks][entries + 2]
  IrlsState* state;
  StatusBlock* status;
  float* scratch;         // |r| per row (polish)
  double* x_out;
  double* obj_out;
  int max_iter;
  // k coresets solved side by side (blockIdx.y = coreset j): coreset j's rows, weights,
  // count, partials, state, status, scratch and outputs start j strides further on.
  int64_t x_stride;       // doubles between coresets' rows (capacity·q)
  int64_t part_stride;    // doubles between coresets' partials
  int64_t scratch_stride; // floats between coresets' scratch
  uint32_t* flags_out;    // per-coreset status flags (may be null)
};

__device__ __forceinline__ IrlsArgs for_coreset(IrlsArgs a) {
  const int64_t j = blockIdx.y;
  a.X += j * a.x_stride;
  a.w += j * a.capacity;
  a.count += j;
  a.partials += j * a.part_stride;
  a.state += j;
  a.status += j;
  a.scratch += j * a.scratch_stride;
  a.x_out += j * a.d;
  if (a.obj_out) a.obj_out += j;
  if (a.flags_out) a.flags_out += j;
  return a;
}

__device__ __forceinline__ int64_t coreset_rows(const IrlsArgs& a) {
  const int64_t c = *a.count;
  return c < a.capacity ? c : a.capacity;
}

__device__ __forceinline__ int pair_count(int q) { return q * (q + 1) / 2 - 1; }

// Entry e → (j, l), 0 ≤ j ≤ l < q, (j, l) ≠ (d, d), row-major over the upper triangle.
__device__ __forceinline__ void pair_of(int e, int q, int& j, int& l) {
  int row = 0, left = e;
  while (left >= q - row) {
    left -= q - row;
    ++row;
  }
  j = row;
  l = row + left;
}

__global__ void __launch_bounds__(kIrlsThreads) irls_accum_kernel(const IrlsArgs a0) {
  const IrlsArgs a = for_coreset(a0);
  if (a.status->irls_done) return;
  extern __shared__ __align__(16) double sm[];
  const int q = a.q;
  double* tile = sm;                      // kIrlsTile × q
  double* om = tile + kIrlsTile * q;      // kIrlsTile
  double* xs = om + kIrlsTile;            // q
  __shared__ double red_f[kIrlsThreads], red_w[kIrlsThreads];
  const int tid = threadIdx.x;
  const int64_t S = coreset_rows(a);
  const int64_t chunk = (S + gridDim.x - 1) / gridDim.x;
  const int64_t start = blockIdx.x * chunk;
  const int64_t stop = min(S, start + chunk);
  for (int k = tid; k < q; k += blockDim.x) xs[k] = a.state->x[k];
  const bool first = a.status->irls_iters == 0;
  const double eta = a.status->irls_eta;
  const int np = pair_count(q);
  int pj[kIrlsSlots], pl[kIrlsSlots];
  double acc[kIrlsSlots];
#pragma unroll
  for (int s = 0; s < kIrlsSlots; ++s) {
    acc[s] = 0.0;
    const int e = tid + s * blockDim.x;
    if (e < np) pair_of(e, q, pj[s], pl[s]);
    else pj[s] = pl[s] = 0;
  }
  double f_acc = 0.0, w_acc = 0.0;
  __syncthreads();
  for (int64_t t0 = start; t0 < stop; t0 += kIrlsTile) {
    const int rows = static_cast<int>(min(static_cast<int64_t>(kIrlsTile), stop - t0));
    for (int i = tid; i < rows * q; i += blockDim.x) tile[i] = a.X[t0 * q + i];
    __syncthreads();
    if (tid < rows) {
      double r = 0.0;
      for (int k = 0; k < q; ++k) r = fma(tile[tid * q + k], xs[k], r);
      const double ar = fabs(r);
      const double wk = a.w[t0 + tid];
      f_acc += wk * ar;
      w_acc += wk;
      om[tid] = first ? wk : wk / fmax(ar, eta);
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kIrlsSlots; ++s) {
      if (tid + s * static_cast<int>(blockDim.x) < np) {
        const int j = pj[s], l = pl[s];
        double v = 0.0;
        for (int t = 0; t < rows; ++t) v = fma(om[t] * tile[t * q + j], tile[t * q + l], v);
        acc[s] += v;
      }
    }
    __syncthreads();
  }
  const int ne = np + 2;
  double* out = a.partials + static_cast<size_t>(blockIdx.x) * ne;
#pragma unroll
  for (int s = 0; s < kIrlsSlots; ++s) {
    const int e = tid + s * blockDim.x;
    if (e < np) out[e] = acc[s];
  }
  red_f[tid] = f_acc;
  red_w[tid] = w_acc;
  __syncthreads();
  if (tid == 0) {
    double f = 0.0, w = 0.0;
    for (int i = 0; i < static_cast<int>(blockDim.x); ++i) {
      f += red_f[i];
      w += red_w[i];
    }
    out[np] = f;
    out[np + 1] = w;
  }
}

// One block: totals, bookkeeping, Cholesky solve of the weighted normal equations.
__global__ void __launch_bounds__(kIrlsThreads) irls_step_kernel(const IrlsArgs a0, int nblocks, int final_pass) {
  const IrlsArgs a = for_coreset(a0);
  StatusBlock* st = a.status;
  if (st->irls_done && !final_pass) return;
  extern __shared__ __align__(16) double sm[];
  const int q = a.q, d = a.d, tid = threadIdx.x;
  const int np = pair_count(q), ne = np + 2;
  double* tot = sm;                 // ne
  double* G = tot + ne;             // d × d (lower Cholesky factor in place)
  double* y = G + d * d;            // d
  __shared__ int s_fail;
  for (int e = tid; e < ne; e += blockDim.x) {
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += a.partials[static_cast<size_t>(b) * ne + e];
    tot[e] = v;
  }
  __syncthreads();
  if (tid == 0) {
    const double f = tot[np];
    IrlsState* S = a.state;
    if (st->irls_iters == 0) {
      S->w_total = tot[np + 1];
      S->best_f = INFINITY;
    }
    if (f < S->best_f) {
      S->best_f = f;
      for (int k = 0; k < q; ++k) S->best_x[k] = S->x[k];
    }
    if (st->irls_iters > 0 && fabs(st->irls_obj - f) <= 1e-12 * f) st->irls_done = 1;
    st->irls_prev_obj = st->irls_obj;
    st->irls_obj = f;
    st->irls_eta = 1e-6 * f / fmax(S->w_total, 1e-300);
    s_fail = 0;
  }
  __syncthreads();
  if (final_pass || st->irls_done) return;
  // Scatter the upper-triangle entries into a full symmetric G and the right-hand side.
  for (int e = tid; e < np; e += blockDim.x) {
    int j, l;
    pair_of(e, q, j, l);
    if (l < d) {
      G[j * d + l] = tot[e];
      G[l * d + j] = tot[e];
    } else {
      y[j] = -tot[e];  // Σ ω a_j b = −Σ ω X_j X_d
    }
  }
  __syncthreads();
  for (int k = 0; k < d; ++k) {
    if (tid == 0) {
      const double piv = G[k * d + k];
      if (!(piv > 0.0) || !isfinite(piv)) s_fail = 1;
      G[k * d + k] = sqrt(fmax(piv, 1e-300));
    }
    __syncthreads();
    const double gkk = G[k * d + k];
    for (int i = k + 1 + tid; i < d; i += blockDim.x) G[i * d + k] /= gkk;
    __syncthreads();
    for (int e = tid; e < (d - k - 1) * (d - k - 1); e += blockDim.x) {
      const int i = k + 1 + e / (d - k - 1), j = k + 1 + e % (d - k - 1);
      if (j <= i) G[i * d + j] -= G[i * d + k] * G[j * d + k];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (s_fail) {
      st->irls_done = 1;
    } else {
      for (int i = 0; i < d; ++i) {  // L·z = y
        double v = y[i];
        for (int j = 0; j < i; ++j) v -= G[i * d + j] * y[j];
        y[i] = v / G[i * d + i];
      }
      for (int i = d - 1; i >= 0; --i) {  // Lᵀ·x = z
        double v = y[i];
        for (int j = i + 1; j < d; ++j) v -= G[j * d + i] * y[j];
        y[i] = v / G[i * d + i];
      }
      bool ok = true;
      for (int i = 0; i < d; ++i) ok &= isfinite(y[i]);
      if (ok) {
        for (int i = 0; i < d; ++i) a.state->x[i] = y[i];
        a.state->x[d] = 1.0;
      } else {
        st->irls_done = 1;
      }
    }
    st->irls_iters += 1;
  }
}

__global__ void irls_init_kernel(const IrlsArgs a0) {
  const IrlsArgs a = for_coreset(a0);
  const int tid = threadIdx.x;
  for (int k = tid; k < a.q; k += blockDim.x) a.state->x[k] = k == a.d ? 1.0 : 0.0;
  if (tid == 0) {
    a.status->irls_done = 0;
    a.status->irls_iters = 0;
    a.status->irls_obj = 0.0;
    a.status->irls_prev_obj = 0.0;
    a.status->irls_eta = 0.0;
  }
}

__global__ void irls_residuals_kernel(const IrlsArgs a0) {
  const IrlsArgs a = for_coreset(a0);
  const int64_t S = coreset_rows(a);
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < S;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double r = 0.0;
    for (int j = 0; j < a.q; ++j) r = fma(a.X[k * a.q + j], a.state->best_x[j], r);
    a.scratch[k] = static_cast<float>(fabs(r));
  }
}

// ----------------------------------------------------------------- vertex finish
// Block-parallel dense LU (partial pivoting) of the d × d matrix B of the active
// rows, and the two triangular solves a simplex pivot needs (B·v = rhs and
// Bᵀ·v = rhs).  Row i of P·B is row perm[i] of B.
__device__ bool block_lu(double* LU, int* perm, int d, int* s_ok) {
  const int tid = threadIdx.x;
  for (int c = 0; c < d; ++c) {
    if (tid == 0) {
      int piv = c;
      for (int r = c + 1; r < d; ++r)
        if (fabs(LU[r * d + c]) > fabs(LU[piv * d + c])) piv = r;
      if (!(fabs(LU[piv * d + c]) > 0.0)) {
        *s_ok = 0;
      } else if (piv != c) {
        for (int j = 0; j < d; ++j) {
          const double t = LU[c * d + j];
          LU[c * d + j] = LU[piv * d + j];
          LU[piv * d + j] = t;
        }
        const int t = perm[c];
        perm[c] = perm[piv];
        perm[piv] = t;
      }
    }
    __syncthreads();
    if (!*s_ok) return false;
    for (int r = c + 1 + tid; r < d; r += blockDim.x) LU[r * d + c] /= LU[c * d + c];
    __syncthreads();
    const int w = d - c - 1;
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int r = c + 1 + e / w, j = c + 1 + e % w;
      LU[r * d + j] = fma(-LU[r * d + c], LU[c * d + j], LU[r * d + j]);
    }
    __syncthreads();
  }
  return true;
}

// v ← B⁻¹·v (transposed = false) or B⁻ᵀ·v (transposed = true); tmp holds d doubles.
__device__ void block_lu_solve(const double* LU, const int* perm, int d, double* v, double* tmp,
                               bool transposed) {
  const int tid = threadIdx.x;
  if (!transposed) {
    for (int i = tid; i < d; i += blockDim.x) tmp[i] = v[perm[i]];
    __syncthreads();
    for (int r = 0; r < d; ++r) {          // L (unit lower)
      for (int k = r + 1 + tid; k < d; k += blockDim.x) tmp[k] = fma(-LU[k * d + r], tmp[r], tmp[k]);
      __syncthreads();
    }
    for (int r = d - 1; r >= 0; --r) {     // U
      if (tid == 0) tmp[r] /= LU[r * d + r];
      __syncthreads();
      for (int k = tid; k < r; k += blockDim.x) tmp[k] = fma(-LU[k * d + r], tmp[r], tmp[k]);
      __syncthreads();
    }
    for (int i = tid; i < d; i += blockDim.x) v[i] = tmp[i];
  } else {
    for (int i = tid; i < d; i += blockDim.x) tmp[i] = v[i];
    __syncthreads();
    for (int r = 0; r < d; ++r) {          // Uᵀ (lower, diagonal of U)
      if (tid == 0) tmp[r] /= LU[r * d + r];
      __syncthreads();
      for (int k = r + 1 + tid; k < d; k += blockDim.x) tmp[k] = fma(-LU[r * d + k], tmp[r], tmp[k]);
      __syncthreads();
    }
    for (int r = d - 1; r >= 0; --r) {     // Lᵀ (unit upper)
      for (int k = tid; k < r; k += blockDim.x) tmp[k] = fma(-LU[r * d + k], tmp[r], tmp[k]);
      __syncthreads();
    }
    for (int i = tid; i < d; i += blockDim.x) v[perm[i]] = tmp[i];
  }
  __syncthreads();
}

// Fixed-order block sum of one value per thread (thread 0's result is broadcast).
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (static_cast<int>(threadIdx.x) < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const double t = red[0];
  __syncthreads();
  return t;
}

constexpr int kMaxPivots = 64;

// One block.  Start from the d coreset rows with the smallest |r| at the best IRLS
// iterate, and walk vertex to vertex (simplex pivots of the LAD linear program):
// at a vertex with active rows Z (r_Z = 0) and B = A_Z, the objective along the edge
// that frees active row j is, to first order, sgn·y_j + w_{Z_j} with y = B⁻ᵀ·c and
// c = Σ_{i∉Z} w_i sign(r_i)·A_i.  The vertex is optimal when |y_j| ≤ w_{Z_j} for
// every j (the multipliers −y certify it); otherwise step along the steepest such
// edge to the minimiser of the piecewise-linear objective on it (a weighted median
// of the breakpoints −r_i/g_i, found by bisection on their bit patterns), where the
// row with that breakpoint enters Z.  The better of this vertex and the IRLS iterate
// is returned.
__global__ void __launch_bounds__(kIrlsThreads) irls_polish_kernel(const IrlsArgs a0) {
  const IrlsArgs a = for_coreset(a0);
  extern __shared__ __align__(16) double sm[];
  const int q = a.q, d = a.d, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  double* LU = sm;                 // d × d
  double* xs = LU + d * d;         // q: current vertex
  double* xb = xs + q;             // q: best vertex
  double* cv = xb + q;             // d: c, then y
  double* dv = cv + d;             // d: edge direction
  double* tmp = dv + d;            // d
  int64_t* Z = reinterpret_cast<int64_t*>(tmp + d);  // d active rows
  int* perm = reinterpret_cast<int*>(Z + d);         // d
  __shared__ float rv[kIrlsThreads];
  __shared__ int64_t ri[kIrlsThreads];
  __shared__ double red[kIrlsThreads];
  __shared__ int s_ok, s_more, s_j, s_certified;
  __shared__ double s_sgn, s_h, s_fb;
  const int64_t S = coreset_rows(a);
  double* rs = reinterpret_cast<double*>(a.scratch);   // S doubles: r, then breakpoints
  double* vs = rs + a.capacity;                        // S doubles: breakpoint weights
  IrlsState* st = a.state;
  if (tid == 0) {
    s_ok = S >= d ? 1 : 0;
    s_certified = 0;
    s_fb = INFINITY;
  }
  __syncthreads();
  // The d rows with the smallest |r| at the IRLS iterate (the float |r| sit in scratch)
  // whose A parts are linearly independent, so that B = A_Z is invertible: a row whose A
  // part lies within 1e-10 relative of the span of the rows taken so far (an exact copy,
  // or another canonical row e_j of a j already taken) is passed over.  Where many rows
  // are passed over (hundreds in a canonical-row design), taking one row per pass over the
  // coreset would be slow, so each round takes every thread's smallest remaining |r|,
  // orders these candidates by (|r|, index), and warp 0 tests them in that order, keeping
  // an orthonormal basis of the taken A parts (Gram–Schmidt, twice) in LU's space, which
  // is free until the first vertex.  Every tested candidate leaves the pool.
  __shared__ int s_k, s_rounds;
  __shared__ int64_t cand[kIrlsThreads];
  if (tid == 0) {
    s_k = 0;
    s_rounds = 0;
  }
  __syncthreads();
  constexpr int kMaxStartRounds = 64;
  while (s_ok && s_k < d && s_rounds < kMaxStartRounds) {
    float best = INFINITY;
    int64_t bi = -1;
    for (int64_t i = tid; i < S; i += blockDim.x) {
      const float v = a.scratch[i];
      if (v < best) {
        best = v;
        bi = i;
      }
    }
    rv[tid] = best;
    ri[tid] = bi;
    const int nvalid = __syncthreads_count(bi >= 0 && best < INFINITY);
    if (nvalid == 0) {
      if (tid == 0) s_ok = 0;
      break;
    }
    if (bi >= 0 && best < INFINITY) {
      int rank = 0;
      for (int t = 0; t < static_cast<int>(blockDim.x); ++t)
        rank += (ri[t] >= 0 && rv[t] < INFINITY && (rv[t] < best || (rv[t] == best && ri[t] < bi))) ? 1 : 0;
      cand[rank] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      constexpr int kPer = (kMaxD + 31) / 32;
      int k = s_k;
      for (int t = 0; t < nvalid && k < d; ++t) {
        const int64_t c = cand[t];
        double v[kPer], n0 = 0.0;
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
          const int e = lane + 32 * u;
          v[u] = e < d ? a.X[c * q + e] : 0.0;
          n0 = fma(v[u], v[u], n0);
        }
        for (int o = 16; o > 0; o >>= 1) n0 += __shfl_xor_sync(0xffffffffu, n0, o);
        for (int pass = 0; pass < 2; ++pass)
          for (int m = 0; m < k; ++m) {
            double dot = 0.0;
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
              const int e = lane + 32 * u;
              if (e < d) dot = fma(v[u], LU[m * d + e], dot);
            }
            for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
              const int e = lane + 32 * u;
              if (e < d) v[u] = fma(-dot, LU[m * d + e], v[u]);
            }
          }
        double n1 = 0.0;
#pragma unroll
        for (int u = 0; u < kPer; ++u) n1 = fma(v[u], v[u], n1);
        for (int o = 16; o > 0; o >>= 1) n1 += __shfl_xor_sync(0xffffffffu, n1, o);
        if (n1 > 1e-20 * n0 && n0 > 0.0) {            // the same decision in every lane
          const double inv = 1.0 / sqrt(n1);
#pragma unroll
          for (int u = 0; u < kPer; ++u) {
            const int e = lane + 32 * u;
            if (e < d) LU[k * d + e] = v[u] * inv;   // each lane reads back only its own entries
          }
          if (lane == 0) Z[k] = c;
          ++k;
        }
        if (lane == 0) a.scratch[c] = INFINITY;
      }
      if (lane == 0) {
        s_k = k;
        s_rounds += 1;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (tid == 0 && s_k < d) s_ok = 0;
  __syncthreads();

  for (int piv = 0; piv < kMaxPivots && s_ok; ++piv) {
    // Vertex of the active rows: B·x = b_Z with B = A_Z (first d columns of X_Z), b = −X_{:,d}.
    for (int e = tid; e < d * d; e += blockDim.x) LU[e] = a.X[Z[e / d] * q + e % d];
    for (int i = tid; i < d; i += blockDim.x) {
      perm[i] = i;
      xs[i] = -a.X[Z[i] * q + d];
    }
    __syncthreads();
    if (!block_lu(LU, perm, d, &s_ok)) break;
    block_lu_solve(LU, perm, d, xs, tmp, false);
    if (tid == 0) {
      xs[d] = 1.0;
      for (int j = 0; j < d; ++j) s_ok &= isfinite(xs[j]) ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) break;
    // Residuals and objective; active rows are exactly on the vertex.
    double facc = 0.0;
    for (int64_t i = tid; i < S; i += blockDim.x) {
      double r = 0.0;
      for (int k = 0; k < q; ++k) r = fma(a.X[i * q + k], xs[k], r);
      rs[i] = r;
      facc += a.w[i] * fabs(r);
    }
    const double f = block_sum(facc, red);
    for (int i = tid; i < d; i += blockDim.x) rs[Z[i]] = 0.0;
    if (!(f < s_fb)) break;   // no further decrease (rounding): keep the best vertex
    for (int k = tid; k < q; k += blockDim.x) xb[k] = xs[k];
    __syncthreads();
    if (tid == 0) s_fb = f;
    // c_k = Σ_{i∉Z} w_i·sign(r_i)·A_ik, one warp per column, lanes over rows.
    for (int k = warp; k < d; k += nwarps) {
      double acc = 0.0;
      for (int64_t i = lane; i < S; i += 32) {
        const double r = rs[i];
        const double sg = r > 0.0 ? 1.0 : (r < 0.0 ? -1.0 : 0.0);
        acc = fma(a.w[i] * sg, a.X[i * q + k], acc);
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) cv[k] = acc;
    }
    __syncthreads();
    block_lu_solve(LU, perm, d, cv, tmp, true);   // y = B⁻ᵀ·c
    if (tid == 0) {
      int jb = -1;
      double worst = 0.0;
      for (int j = 0; j < d; ++j) {
        const double wz = a.w[Z[j]];
        const double slope = wz - fabs(cv[j]);
        if (slope < -1e-12 * (wz + fabs(cv[j])) && slope < worst) {
          worst = slope;
          jb = j;
        }
      }
      s_more = jb >= 0 ? 1 : 0;
      if (jb < 0) s_certified = 1;
      s_j = jb;
      s_sgn = jb >= 0 ? (cv[jb] > 0.0 ? -1.0 : 1.0) : 0.0;
      s_h = -0.5 * worst;
    }
    __syncthreads();
    if (!s_more) break;
    // Edge direction: B·dv = sgn·e_j.
    for (int i = tid; i < d; i += blockDim.x) dv[i] = i == s_j ? s_sgn : 0.0;
    __syncthreads();
    block_lu_solve(LU, perm, d, dv, tmp, false);
    // Breakpoints t_i = −r_i/g_i > 0 with weights w_i·|g_i| (others: +inf, weight 0).
    for (int64_t i = tid; i < S; i += blockDim.x) {
      double g = 0.0;
      for (int k = 0; k < d; ++k) g = fma(a.X[i * q + k], dv[k], g);
      double t = g != 0.0 ? -rs[i] / g : 0.0;
      const bool live = t > 0.0 && isfinite(t);
      rs[i] = live ? t : INFINITY;
      vs[i] = live ? a.w[i] * fabs(g) : 0.0;
    }
    __syncthreads();
    // Smallest breakpoint T with Σ_{t_i ≤ T} w_i|g_i| ≥ h: bisection on the bit patterns
    // of positive doubles (their order is the order of the values).
    long long lo = 0, hi = 0x7FF0000000000000LL;
    {
      double wtot = 0.0;
      for (int64_t i = tid; i < S; i += blockDim.x) wtot += vs[i];
      if (!(block_sum(wtot, red) >= s_h)) break;   // no finite minimiser on this edge
    }
    while (lo < hi) {
      const long long mid = lo + (hi - lo) / 2;
      const double T = __longlong_as_double(mid);
      double acc = 0.0;
      for (int64_t i = tid; i < S; i += blockDim.x)
        if (rs[i] <= T) acc += vs[i];
      if (block_sum(acc, red) >= s_h)
        hi = mid;
      else
        lo = mid + 1;
    }
    const double T = __longlong_as_double(lo);
    int64_t enter = S;
    for (int64_t i = tid; i < S; i += blockDim.x)
      if (rs[i] == T) {
        enter = i;
        break;
      }
    ri[tid] = enter;
    __syncthreads();
    if (tid == 0) {
      int64_t k = S;
      for (int t = 0; t < static_cast<int>(blockDim.x); ++t) k = ri[t] < k ? ri[t] : k;
      if (k >= S) s_ok = 0;
      else Z[s_j] = k;
    }
    __syncthreads();
  }
  __syncthreads();
  if (tid == 0) {
    const bool use = isfinite(s_fb) && s_fb <= st->best_f;
    for (int j = 0; j < d; ++j) a.x_out[j] = use ? xb[j] : st->best_x[j];
    if (a.obj_out) *a.obj_out = use ? s_fb : st->best_f;
    if (!a.status->irls_done && !(use && s_certified)) raise_flag(&a.status->flags, L1S_ERR_NOT_CONVERGED);
    if (a.flags_out) *a.flags_out = atomicOr(&a.status->flags, 0u);
  }
}

size_t polish_smem_bytes(int d) {
  const int q = d + 1;
  return sizeof(double) * (static_cast<size_t>(d) * d + 2 * q + 3 * d) + sizeof(int64_t) * d + sizeof(int) * d;
}

size_t solve_scratch_bytes(int64_t capacity) { return 2 * sizeof(double) * static_cast<size_t>(capacity); }

int irls_entries(int q) { return q * (q + 1) / 2 + 1; }
size_t irls_state_bytes() { return sizeof(IrlsState); }

// k coresets at once: coreset j at X + j·capacity·q, w + j·capacity, count + j; its
// partials, state, status block and scratch are the j-th of arrays of k; outputs
// x_out + j·d, obj_out + j, flags_out + j.  nblocks accumulation blocks per coreset.
bool launch_solve(const double* X, const double* w, const int64_t* count, int64_t capacity, int d,
                  int max_iter, double* x_out, double* obj_out, int nblocks, double* partials,
                  void* state, float* scratch, StatusBlock* status, cudaStream_t st, int k,
                  uint32_t* flags_out) {
  IrlsArgs a;
  a.X = X;
  a.w = w;
  a.count = count;
  a.capacity = capacity;
  a.d = d;
  a.q = d + 1;
  a.partials = partials;
  a.state = static_cast<IrlsState*>(state);
  a.status = status;
  a.scratch = scratch;
  a.x_out = x_out;
  a.obj_out = obj_out;
  a.max_iter = max_iter;
  const int q = d + 1;
  a.x_stride = capacity * q;
  a.part_stride = static_cast<int64_t>(nblocks) * (irls_entries(q) + 1);
  a.scratch_stride = static_cast<int64_t>(solve_scratch_bytes(capacity) / sizeof(float));
  a.flags_out = flags_out;
  const size_t acc_smem = sizeof(double) * (kIrlsTile * q + kIrlsTile + q);
  const size_t step_smem = sizeof(double) * (irls_entries(q) + d * d + d);
  const size_t pol_smem = polish_smem_bytes(d);
  if (!allow_dynamic_smem(reinterpret_cast<const void*>(irls_step_kernel), step_smem, "irls_step smem") ||
      !allow_dynamic_smem(reinterpret_cast<const void*>(irls_accum_kernel), acc_smem, "irls_accum smem") ||
      !allow_dynamic_smem(reinterpret_cast<const void*>(irls_polish_kernel), pol_smem, "irls_polish smem"))
    return false;
  const dim3 many(nblocks, k), one(1, k);
  irls_init_kernel<<<one, 256, 0, st>>>(a);
  for (int it = 0; it < max_iter; ++it) {
    irls_accum_kernel<<<many, kIrlsThreads, acc_smem, st>>>(a);
    irls_step_kernel<<<one, kIrlsThreads, step_smem, st>>>(a, nblocks, 0);
  }
  // Objective of the last iterate, then the vertex polish.
  irls_accum_kernel<<<many, kIrlsThreads, acc_smem, st>>>(a);
  irls_step_kernel<<<one, kIrlsThreads, step_smem, st>>>(a, nblocks, 1);
  irls_residuals_kernel<<<many, 256, 0, st>>>(a);
  irls_polish_kernel<<<one, kIrlsThreads, pol_smem, st>>>(a);
  count_launch(2 * max_iter + 5);
  return cuda_ok(cudaGetLastError(), "launch l1_solve kernels");
}

// ----------------------------------------------------------------- objective
template <typename TA>
__global__ void __launch_bounds__(256) objective_kernel(const TA* __restrict__ A, int64_t lda,
                                                        const float* __restrict__ b, int64_t n, int d,
                                                        const double* __restrict__ x,
                                                        double* __restrict__ partials) {
  __shared__ double xs[kMaxD];
  __shared__ double red[256];
  for (int k = threadIdx.x; k < d; k += blockDim.x) xs[k] = x[k];
  __syncthreads();
  double acc = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const TA* p = A + i * lda;
    double r = -static_cast<double>(b[i]);
    for (int k = 0; k < d; ++k) r = fma(static_cast<double>(load_elem<TA>(p + k)), xs[k], r);
    acc += fabs(r);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < static_cast<int>(blockDim.x); ++k) t += red[k];
    partials[blockIdx.x] = t;
  }
}

__global__ void sum_partials_kernel(const double* __restrict__ partials, int count, double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < static_cast<int>(blockDim.x); ++k) t += red[k];
    *out = t;
  }
}

bool launch_objective(const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n, int d,
                      const double* x, double* out, int nblocks, double* partials, cudaStream_t st) {
  if (dt == L1S_BF16)
    objective_kernel<uint16_t><<<nblocks, 256, 0, st>>>(static_cast<const uint16_t*>(A), lda, b, n, d, x,
                                                       partials);
  else
    objective_kernel<float><<<nblocks, 256, 0, st>>>(static_cast<const float*>(A), lda, b, n, d, x,
                                                    partials);
  sum_partials_kernel<<<1, 256, 0, st>>>(partials, nblocks, out);
  count_launch(2);
  return cuda_ok(cudaGetLastError(), "launch objective");
}

}  // namespace l1s
