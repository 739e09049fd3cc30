// als.cu -- one CP-ALS sweep (Sec. II-A5) on top of the spMTTKRP kernels.
//
// Per mode d (Gauss-Seidel over d = 0..N-1, Algorithm 1's mode loop):
//   M      = spMTTKRP_d(Y)                                   (mttkrp.cu)
//   V      = Hadamard over w != d of G_w,  G_w = Y_w^T Y_w    (R x R, FP64)
//   L      = Cholesky(V) (FP64); W = V^{-1} = L^{-T} L^{-1}   (FP64, one block)
//   Z      = M W, accumulated in double-float (FP32 pairs)    (all SMs)
//   lambda = column 2-norms of Z;  Y_d = Z / lambda stored as FP32 or BF16
//   G_d    = Gram of the stored Y_d, exact FP32 products summed in
//            double-float per block, blocks summed in FP64 in a fixed order.
// After the last mode: fit = 1 - sqrt(max(0, |X|^2 + |Xhat|^2 - 2<X,Xhat>))/|X|
// with |Xhat|^2 = lambda^T (Hadamard of all G_w) lambda and
// <X,Xhat> = sum_r lambda_r sum_i M(i,r) Y_{N-1}(i,r)  (Kolda & Bader).
//
// FP64 arithmetic is confined to O(R^2)-O(R^3) work (the R x R system): FP64
// throughput on GB300 is a small fraction of FP32, so the O(I R^2) passes use
// error-free FP32 transformations (two-product via FMA, two-sum) instead.
#include <algorithm>

#include "plan.cuh"

namespace spm {
namespace {

constexpr int ALS_THREADS = 256;
constexpr int GRAM_TILE_ROWS = 32;

// ---- double-float helpers (Dekker / Knuth error-free transformations) ----
struct df {
  float hi, lo;
};
__device__ __forceinline__ void df_add_prod(df& acc, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);  // exact: a*b = p + e
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  const float err = (acc.hi - (s - bb)) + (p - bb);
  acc.hi = s;
  acc.lo += err + e;
}
__device__ __forceinline__ void df_add_prod2(df& acc, float a, float bh, float bl) {
  const float p = a * bh;
  float e = fmaf(a, bh, -p);
  e = fmaf(a, bl, e);
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  const float err = (acc.hi - (s - bb)) + (p - bb);
  acc.hi = s;
  acc.lo += err + e;
}
__device__ __forceinline__ double df_value(const df& a) { return (double)a.hi + (double)a.lo; }

template <typename FT>
__device__ __forceinline__ float load_f(const FT* p, int64_t i);
template <>
__device__ __forceinline__ float load_f<float>(const float* p, int64_t i) { return p[i]; }
template <>
__device__ __forceinline__ float load_f<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}
template <typename FT>
__device__ __forceinline__ FT store_cvt(float x);
template <>
__device__ __forceinline__ float store_cvt<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 store_cvt<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}

// ---------------------------------------------------------------------------
// Gram partials: block b sums rows [i0, i1) of Y; thread (tr, ts) of a 16x16
// grid owns entries (tr + 16 a, ts + 16 b).  Requires R <= 16 * GT.
// ---------------------------------------------------------------------------
template <typename FT, int GT>
__global__ void __launch_bounds__(ALS_THREADS)
    gram_partial_kernel(const FT* __restrict__ Y, int64_t I, int R, int64_t rows_per_block,
                        double* __restrict__ part) {
  __shared__ float tile[GRAM_TILE_ROWS][16 * GT + 1];
  const int tr = threadIdx.x / 16, ts = threadIdx.x % 16;
  const int64_t i0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t i1 = std::min<int64_t>(I, i0 + rows_per_block);
  df acc[GT][GT];
#pragma unroll
  for (int a = 0; a < GT; ++a)
#pragma unroll
    for (int b = 0; b < GT; ++b) acc[a][b] = {0.f, 0.f};
  for (int64_t t0 = i0; t0 < i1; t0 += GRAM_TILE_ROWS) {
    const int nrow = (int)std::min<int64_t>(GRAM_TILE_ROWS, i1 - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < GRAM_TILE_ROWS * 16 * GT; e += ALS_THREADS) {
      const int rr = e / (16 * GT), cc = e % (16 * GT);
      tile[rr][cc] = (rr < nrow && cc < R) ? load_f<FT>(Y, (t0 + rr) * R + cc) : 0.f;
    }
    __syncthreads();
    for (int rr = 0; rr < nrow; ++rr) {
      float ya[GT], yb[GT];
#pragma unroll
      for (int a = 0; a < GT; ++a) ya[a] = tile[rr][tr + 16 * a];
#pragma unroll
      for (int b = 0; b < GT; ++b) yb[b] = tile[rr][ts + 16 * b];
#pragma unroll
      for (int a = 0; a < GT; ++a)
#pragma unroll
        for (int b = 0; b < GT; ++b) df_add_prod(acc[a][b], ya[a], yb[b]);
    }
  }
  double* out = part + (int64_t)blockIdx.x * R * R;
#pragma unroll
  for (int a = 0; a < GT; ++a)
#pragma unroll
    for (int b = 0; b < GT; ++b) {
      const int r = tr + 16 * a, s = ts + 16 * b;
      if (r < R && s < R) out[r * R + s] = df_value(acc[a][b]);
    }
}

// G = sum over blocks of the partials (fixed order, FP64).
__global__ void gram_reduce_kernel(const double* __restrict__ part, int nblocks, int R,
                                   double* __restrict__ G, const int* __restrict__ err) {
  if (*err) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < R * R; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * R * R + e];
    G[e] = s;
  }
}

// ---------------------------------------------------------------------------
// V = Hadamard of the other Grams; Cholesky; W = V^{-1} as FP32 hi/lo pairs.
// One block.  `chol` (R*R doubles) is the working matrix.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(ALS_THREADS)
    system_kernel(const double* __restrict__ grams, int N, int d, int R,
                  double* __restrict__ V, float* __restrict__ winv, int* __restrict__ err) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = *err ? 1 : 0;
  __syncthreads();
  if (bad) return;
  const int RR = R * R;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    double v = 1.0;
    for (int w = 0; w < N; ++w)
      if (w != d) v *= grams[(int64_t)w * RR + e];
    V[e] = v;
  }
  __syncthreads();
  // right-looking Cholesky, lower triangle of V becomes L
  for (int j = 0; j < R; ++j) {
    if (threadIdx.x == 0) {
      const double piv = V[j * R + j];
      if (!(piv > 0.0) || !isfinite(piv)) bad = 1;
      else V[j * R + j] = sqrt(piv);
    }
    __syncthreads();
    if (bad) break;
    const double ljj = V[j * R + j];
    for (int i = j + 1 + threadIdx.x; i < R; i += blockDim.x) V[i * R + j] /= ljj;
    __syncthreads();
    const int m = R - j - 1;  // trailing (m x m) lower triangle update
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) V[i * R + k] -= V[i * R + j] * V[k * R + j];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicOr(err, DEV_ERR_NUMERIC);
    return;
  }
  // X = L^{-1} column by column (thread c owns column c), stored in the upper
  // triangle positions transposed: Xt[c][i] = X[i][c] at V[c*R + i] for i > c
  // would clash with L, so X goes to winv's scratch as doubles is avoided:
  // each thread keeps its column in the (unused) strictly upper part of V
  // reversed: X[i][c] for i >= c is written to V[c * R + i] only for i > c,
  // and the diagonal 1/L[c][c] is recomputed when needed.
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    // forward substitution L x = e_c, x_i = 0 for i < c
    for (int i = c; i < R; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) {
        const double xk = (k == c) ? 1.0 / V[c * R + c] : V[c * R + k];
        s -= V[i * R + k] * xk;
      }
      const double xi = s / V[i * R + i];
      if (i > c) V[c * R + i] = xi;
    }
  }
  __syncthreads();
  // W = X^T X:  W[r][s] = sum_{k >= max(r,s)} X[k][r] X[k][s]
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int r = e / R, s = e % R;
    const int k0 = r > s ? r : s;
    double acc = 0.0;
    for (int k = k0; k < R; ++k) {
      const double xr = (k == r) ? 1.0 / V[r * R + r] : V[r * R + k];
      const double xs = (k == s) ? 1.0 / V[s * R + s] : V[s * R + k];
      acc += xr * xs;
    }
    const float hi = (float)acc;
    winv[e] = hi;
    winv[RR + e] = (float)(acc - (double)hi);
  }
}

// ---------------------------------------------------------------------------
// Z = M W (double-float), column sums of Z^2 per block.  One warp handles
// ROWS rows at a time; lane owns ranks lane + 32 j (j < RPL).
// ---------------------------------------------------------------------------
template <int RPL>
__global__ void __launch_bounds__(ALS_THREADS)
    solve_kernel(const float* __restrict__ M, const float* __restrict__ winv, int64_t I, int R,
                 float* __restrict__ Z, double* __restrict__ colsq_part,
                 const int* __restrict__ err) {
  constexpr int ROWS = 4;
  __shared__ double red[ALS_THREADS / 32][32 * RPL];
  if (*err) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int RR = R * R;
  const int64_t gwarp = (int64_t)blockIdx.x * (ALS_THREADS / 32) + warp;
  const int64_t nwarps = (int64_t)gridDim.x * (ALS_THREADS / 32);
  df sq[RPL];
#pragma unroll
  for (int j = 0; j < RPL; ++j) sq[j] = {0.f, 0.f};
  for (int64_t i0 = gwarp * ROWS; i0 < I; i0 += nwarps * ROWS) {
    df acc[ROWS][RPL];
#pragma unroll
    for (int q = 0; q < ROWS; ++q)
#pragma unroll
      for (int j = 0; j < RPL; ++j) acc[q][j] = {0.f, 0.f};
    for (int s = 0; s < R; ++s) {
      float m[ROWS];
#pragma unroll
      for (int q = 0; q < ROWS; ++q) m[q] = (i0 + q < I) ? M[(i0 + q) * R + s] : 0.f;
#pragma unroll
      for (int j = 0; j < RPL; ++j) {
        const int r = lane + 32 * j;
        if (r < R) {
          const float wh = winv[s * R + r], wl = winv[RR + s * R + r];
#pragma unroll
          for (int q = 0; q < ROWS; ++q) df_add_prod2(acc[q][j], m[q], wh, wl);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      if (i0 + q >= I) break;
#pragma unroll
      for (int j = 0; j < RPL; ++j) {
        const int r = lane + 32 * j;
        if (r < R) {
          const float z = acc[q][j].hi + acc[q][j].lo;
          Z[(i0 + q) * R + r] = z;
          df_add_prod(sq[j], z, z);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < RPL; ++j) red[warp][lane + 32 * j] = df_value(sq[j]);
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < ALS_THREADS / 32; ++w) s += red[w][r];
    colsq_part[(int64_t)blockIdx.x * R + r] = s;
  }
}

__global__ void lambda_kernel(const double* __restrict__ colsq_part, int nblocks, int R,
                              double* __restrict__ lambda, const int* __restrict__ err) {
  if (*err) return;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += colsq_part[(int64_t)b * R + r];
    lambda[r] = sqrt(s);
  }
}

// Y_d = Z / lambda (stored type FT); optionally sums M .* Y per column.
template <typename FT>
__global__ void __launch_bounds__(ALS_THREADS)
    scale_kernel(const float* __restrict__ Z, const double* __restrict__ lambda, int64_t I, int R,
                 FT* __restrict__ Y, const float* __restrict__ M, double* __restrict__ inner_part,
                 const int* __restrict__ err) {
  __shared__ double red[ALS_THREADS];
  if (*err) return;
  // each thread walks a fixed rank r = t % R over rows (t / R) + k * stride
  // (requires R <= ALS_THREADS)
  const int per = ALS_THREADS / R;
  const int r = threadIdx.x % R;
  const int sub = threadIdx.x / R;
  const bool active = sub < per;
  const double lam = lambda[r];
  const float inv = lam > 0.0 ? (float)(1.0 / lam) : 1.f;
  df in = {0.f, 0.f};
  if (active) {
    const int64_t stride = (int64_t)gridDim.x * per;
    for (int64_t i = (int64_t)blockIdx.x * per + sub; i < I; i += stride) {
      const float z = Z[i * R + r];
      const float y = lam > 0.0 ? z * inv : z;
      const FT ys = store_cvt<FT>(y);
      Y[i * R + r] = ys;
      if (M) df_add_prod(in, M[i * R + r], load_f<FT>(&ys, 0));
    }
  }
  if (!M) return;
  red[threadIdx.x] = active ? df_value(in) : 0.0;
  __syncthreads();
  if (threadIdx.x < R) {
    double s = 0.0;
    for (int q = 0; q < per; ++q) s += red[q * R + threadIdx.x];
    inner_part[(int64_t)blockIdx.x * R + threadIdx.x] = s;
  }
}

// fit from |X|^2, lambda, all Grams and the inner-product partials.
__global__ void fit_kernel(const double* __restrict__ grams, int N, int R,
                           const double* __restrict__ lambda,
                           const double* __restrict__ inner_part, int nblocks,
                           const double* __restrict__ normX2, double* __restrict__ fit,
                           double* __restrict__ lambda_out, const int* __restrict__ err) {
  __shared__ double red[ALS_THREADS];
  __shared__ double red2[ALS_THREADS];
  const int RR = R * R;
  double xh = 0.0, inn = 0.0;
  if (!*err) {
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
      double h = 1.0;
      for (int w = 0; w < N; ++w) h *= grams[(int64_t)w * RR + e];
      xh += lambda[e / R] * lambda[e % R] * h;
    }
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      double s = 0.0;
      for (int b = 0; b < nblocks; ++b) s += inner_part[(int64_t)b * R + r];
      inn += lambda[r] * s;
      lambda_out[r] = lambda[r];
    }
  }
  red[threadIdx.x] = xh;
  red2[threadIdx.x] = inn;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x] += red[threadIdx.x + o];
      red2[threadIdx.x] += red2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && fit && !*err) {
    const double nx = *normX2;
    double res = nx + red[0] - 2.0 * red2[0];
    if (res < 0.0) res = 0.0;
    *fit = nx > 0.0 ? 1.0 - sqrt(res) / sqrt(nx) : 1.0;
  }
}

__global__ void copy_lambda_kernel(const double* __restrict__ src, int R, double* __restrict__ dst,
                                   const int* __restrict__ err) {
  if (*err) return;
  for (int r = threadIdx.x; r < R; r += blockDim.x) dst[r] = src[r];
}

// ---------------------------------------------------------------------------

int gram_tile(int R) { return R <= 16 ? 1 : R <= 32 ? 2 : R <= 64 ? 4 : 0; }

int work_blocks(int64_t I, int64_t rows_per_block_min, int cap) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(cap, ceil_div<int64_t>(I, rows_per_block_min)));
}

template <typename FT>
spm_status launch_gram(spmttkrp_plan_s* p, const void* Y, int64_t I, double* G, cudaStream_t s) {
  const int R = p->R;
  spm_als_state& A = p->als;
  const int nb = work_blocks(I, GRAM_TILE_ROWS, A.gram_blocks);
  const int64_t rpb = ceil_div<int64_t>(I, nb);
  const FT* y = static_cast<const FT*>(Y);
  switch (gram_tile(R)) {
    case 1: gram_partial_kernel<FT, 1><<<nb, ALS_THREADS, 0, s>>>(y, I, R, rpb, A.gram_part); break;
    case 2: gram_partial_kernel<FT, 2><<<nb, ALS_THREADS, 0, s>>>(y, I, R, rpb, A.gram_part); break;
    case 4: gram_partial_kernel<FT, 4><<<nb, ALS_THREADS, 0, s>>>(y, I, R, rpb, A.gram_part); break;
    default: return SPM_ERR_UNSUPPORTED;
  }
  gram_reduce_kernel<<<std::max(1, std::min(64, R * R / 256 + 1)), 256, 0, s>>>(
      A.gram_part, nb, R, G, p->dev_err);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

spm_status gram(spmttkrp_plan_s* p, const void* Y, int64_t I, double* G, cudaStream_t s) {
  return p->bf16 ? launch_gram<__nv_bfloat16>(p, Y, I, G, s) : launch_gram<float>(p, Y, I, G, s);
}

spm_status ensure_als_state(spmttkrp_plan_s* p) {
  spm_als_state& A = p->als;
  if (A.M) return SPM_OK;
  const int R = p->R;
  int64_t Imax = 1;
  for (int w = 0; w < p->N; ++w) Imax = std::max(Imax, p->dims[w]);
  A.gram_blocks = std::max(1, sm_count()) * 4;
  const size_t RR = (size_t)R * R;
  SPM_TRY(plan_alloc(p, (void**)&A.gram, sizeof(double) * RR * p->N));
  SPM_TRY(plan_alloc(p, (void**)&A.gram_part, sizeof(double) * RR * A.gram_blocks));
  SPM_TRY(plan_alloc(p, (void**)&A.chol, sizeof(double) * RR));
  SPM_TRY(plan_alloc(p, (void**)&A.winv, sizeof(float) * 2 * RR));
  SPM_TRY(plan_alloc(p, (void**)&A.colsq_part, sizeof(double) * R * A.gram_blocks));
  SPM_TRY(plan_alloc(p, (void**)&A.inner_part, sizeof(double) * R * A.gram_blocks));
  SPM_TRY(plan_alloc(p, (void**)&A.lambda_ws, sizeof(double) * R));
  SPM_TRY(plan_alloc(p, (void**)&A.Z, sizeof(float) * (size_t)Imax * R));
  SPM_TRY(plan_alloc(p, (void**)&A.M, sizeof(float) * (size_t)Imax * R));
  return SPM_OK;
}

}  // namespace

spm_status als_sweep(spmttkrp_plan_s* p, void* const* factors, double* lambda, double* fit,
                     cudaStream_t s) {
  const int N = p->N, R = p->R;
  if (gram_tile(R) == 0 || R > ALS_THREADS) return SPM_ERR_UNSUPPORTED;
  for (int w = 0; w < N; ++w)
    if (!factors[w] || (reinterpret_cast<uintptr_t>(factors[w]) & 15u)) return SPM_ERR_INVALID_ARG;
  SPM_TRY(ensure_als_state(p));
  spm_als_state& A = p->als;
  bool same = A.ready;
  for (int w = 0; w < N; ++w) same = same && A.fac_ptr[w] == factors[w];
  if (!same) {
    for (int w = 0; w < N; ++w) {
      SPM_TRY(gram(p, factors[w], p->dims[w], A.gram + (size_t)w * R * R, s));
      A.fac_ptr[w] = factors[w];
    }
    A.ready = true;
  }
  const int nb_solve = A.gram_blocks;
  for (int d = 0; d < N; ++d) {
    const int64_t I = p->dims[d];
    SPM_TRY(run_mttkrp(p, d, factors, A.M, s));
    system_kernel<<<1, ALS_THREADS, 0, s>>>(A.gram, N, d, R, A.chol, A.winv, p->dev_err);
    const int nb = work_blocks(I, 4 * (ALS_THREADS / 32), nb_solve);
    if (R <= 32) solve_kernel<1><<<nb, ALS_THREADS, 0, s>>>(A.M, A.winv, I, R, A.Z, A.colsq_part, p->dev_err);
    else solve_kernel<2><<<nb, ALS_THREADS, 0, s>>>(A.M, A.winv, I, R, A.Z, A.colsq_part, p->dev_err);
    lambda_kernel<<<1, 256, 0, s>>>(A.colsq_part, nb, R, A.lambda_ws, p->dev_err);
    const bool last = d == N - 1;
    const int nbs = work_blocks(I, ALS_THREADS / R, nb_solve);
    if (p->bf16)
      scale_kernel<__nv_bfloat16><<<nbs, ALS_THREADS, 0, s>>>(
          A.Z, A.lambda_ws, I, R, static_cast<__nv_bfloat16*>(factors[d]), last ? A.M : nullptr,
          A.inner_part, p->dev_err);
    else
      scale_kernel<float><<<nbs, ALS_THREADS, 0, s>>>(A.Z, A.lambda_ws, I, R,
                                                       static_cast<float*>(factors[d]),
                                                       last ? A.M : nullptr, A.inner_part,
                                                       p->dev_err);
    SPM_CUDA_TRY(cudaGetLastError());
    SPM_TRY(gram(p, factors[d], I, A.gram + (size_t)d * R * R, s));
    if (last) {
      fit_kernel<<<1, ALS_THREADS, 0, s>>>(A.gram, N, R, A.lambda_ws, A.inner_part, nbs,
                                           p->normX2, fit, lambda, p->dev_err);
    }
  }
  if (!fit) copy_lambda_kernel<<<1, 256, 0, s>>>(A.lambda_ws, R, lambda, p->dev_err);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

}  // namespace spm
