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

#include "als_tc.cuh"

namespace spm {
namespace {

template <typename FT, int GT>
__global__ void __launch_bounds__(ALS_THREADS)
    gram_partial_kernel(const FT* __restrict__ Y, int64_t I, int R, int64_t rows_per_block,
                        double* __restrict__ part, const uint32_t* __restrict__ mask) {
  gram_partial_body<FT, GT>(Y, I, R, rows_per_block, part, blockIdx.x, mask);
}

__global__ void gram_reduce_kernel(const double* __restrict__ part, int nblocks, int R,
                                   double* __restrict__ G, const int* __restrict__ err) {
  gram_reduce_body(part, nblocks, R, G, err, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(SYS_THREADS)
    system_kernel(const double* __restrict__ grams, int N, int d, int R,
                  double* __restrict__ V, float* __restrict__ winv,
                  unsigned char* __restrict__ wdig, int* __restrict__ err) {
  system_col_body(grams, N, d, R, blockIdx.x, blockIdx.x + 1, V, winv, wdig, err);
}

template <int RPL, int LPR>
__global__ void __launch_bounds__(ALS_THREADS)
    solve_kernel(const float* __restrict__ M, const float* __restrict__ winv, int64_t I, int R,
                 float* __restrict__ Z, double* __restrict__ colsq_part,
                 const int* __restrict__ err, const uint32_t* __restrict__ mask) {
  solve_body<RPL, LPR>(M, winv, I, R, Z, colsq_part, err, blockIdx.x, gridDim.x, mask);
}

template <int R>
__global__ void __launch_bounds__(TC_THREADS)
    tc_solve_kernel(const float* __restrict__ M, const unsigned char* __restrict__ wdig, int64_t I,
                    float* __restrict__ Z, double* __restrict__ colsq_part,
                    float* __restrict__ colmax_part, const int* __restrict__ err, int nvb,
                    const uint32_t* __restrict__ mask) {
  tc_solve_body<R>(M, wdig, I, Z, colsq_part, colmax_part, err, blockIdx.x, nvb, mask);
}

__global__ void lambda_kernel(const double* __restrict__ colsq_part,
                              const float* __restrict__ colmax_part, int nblocks, int R,
                              double* __restrict__ lambda, const int* __restrict__ err) {
  lambda_body(colsq_part, colmax_part, nblocks, R, lambda, err, blockIdx.x);
}

template <typename FT, int R>
__global__ void __launch_bounds__(TC_THREADS)
    tc_scale_gram_kernel(const float* __restrict__ Z, const double* __restrict__ lam, int64_t I,
                         FT* __restrict__ Y, const float* __restrict__ M,
                         double* __restrict__ gram_part, double* __restrict__ inner_part,
                         const int* __restrict__ err, const uint32_t* __restrict__ mask) {
  tc_scale_gram_body<FT, R>(Z, lam, I, Y, M, gram_part, inner_part, err, blockIdx.x, gridDim.x,
                            mask);
}

template <typename FT>
__global__ void __launch_bounds__(ALS_THREADS)
    scale_kernel(const float* __restrict__ Z, const double* __restrict__ lambda, int64_t I, int R,
                 FT* __restrict__ Y, const float* __restrict__ M, double* __restrict__ inner_part,
                 const int* __restrict__ err, const uint32_t* __restrict__ mask) {
  scale_body<FT>(Z, lambda, I, R, Y, M, inner_part, err, blockIdx.x, gridDim.x, mask);
}

__global__ void fit_kernel(const double* __restrict__ grams, int N, int R,
                           const double* __restrict__ lambda,
                           const double* __restrict__ inner_part, int nblocks,
                           const double* __restrict__ normX2, double* __restrict__ fit,
                           double* __restrict__ lambda_out, const int* __restrict__ err) {
  fit_body(grams, N, R, lambda, inner_part, nblocks, normX2, fit, lambda_out, err);
}

__global__ void copy_lambda_kernel(const double* __restrict__ src, int R, double* __restrict__ dst,
                                   const int* __restrict__ err) {
  copy_lambda_body(src, R, dst, err);
}

template <typename FT>
spm_status launch_gram(spmttkrp_plan_s* p, const void* Y, int64_t I, double* G, cudaStream_t s,
                       const uint32_t* mask) {
  const int R = p->R;
  spm_als_state& A = p->als;
  const int nb = als_row_blocks(I, A.gram_blocks);
  const int64_t rpb = ceil_div<int64_t>(I, nb);
  const FT* y = static_cast<const FT*>(Y);
  switch (gram_tile(R)) {
    case 1: gram_partial_kernel<FT, 1><<<nb, ALS_THREADS, 0, s>>>(y, I, R, rpb, A.gram_part, mask); break;
    case 2: gram_partial_kernel<FT, 2><<<nb, ALS_THREADS, 0, s>>>(y, I, R, rpb, A.gram_part, mask); break;
    case 4: gram_partial_kernel<FT, 4><<<nb, ALS_THREADS, 0, s>>>(y, I, R, rpb, A.gram_part, mask); break;
    default: return SPM_ERR_UNSUPPORTED;
  }
  gram_reduce_kernel<<<std::max(1, std::min(1024, R * R / 8)), 256, 0, s>>>(
      A.gram_part, nb, R, G, p->dev_err);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

}  // namespace

// The tensor-core row solve over `nb` virtual blocks (R = 16, 32 or 64).
template <int R>
spm_status launch_tc_solve_r(int nb, const float* M, const unsigned char* wdig, int64_t I, float* Z,
                             double* colsq_part, float* colmax_part, const int* err,
                             const uint32_t* mask, cudaStream_t s) {
  constexpr int smem = (int)TcSolveShape<R>::SMEM;
  SPM_CUDA_TRY(cudaFuncSetAttribute(tc_solve_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  tc_solve_kernel<R><<<nb, TC_THREADS, smem, s>>>(M, wdig, I, Z, colsq_part, colmax_part, err, nb, mask);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

// The row solve of one mode: tensor cores for R = 16, 32 and 64, else the
// CUDA-core double-float solve in the lane layout of R.  Kept out of line:
// inlined into the sweep loop, the equivalent if-chain launched the next
// variant's instantiation on the aarch64 host build (gcc 13.3, -O2), which
// the bitwise batch-versus-single sweep test exposed.
__attribute__((noinline)) spm_status launch_solve(int R, int nb, const spm_als_state& A, int64_t I,
                                                  const int* err, const uint32_t* mask,
                                                  cudaStream_t s) {
  switch (tc_solve_rank(R) ? R : 0) {
    case 16: return launch_tc_solve_r<16>(nb, A.M, A.wdig, I, A.Z, A.colsq_part, A.colmax_part, err, mask, s);
    case 32: return launch_tc_solve_r<32>(nb, A.M, A.wdig, I, A.Z, A.colsq_part, A.colmax_part, err, mask, s);
    case 64: return launch_tc_solve_r<64>(nb, A.M, A.wdig, I, A.Z, A.colsq_part, A.colmax_part, err, mask, s);
    default: break;
  }
  switch (R <= 8 ? 0 : R <= 16 ? 1 : R <= 32 ? 2 : 3) {
    case 0: solve_kernel<1, 8><<<nb, ALS_THREADS, 0, s>>>(A.M, A.winv, I, R, A.Z, A.colsq_part, err, mask); break;
    case 1: solve_kernel<1, 16><<<nb, ALS_THREADS, 0, s>>>(A.M, A.winv, I, R, A.Z, A.colsq_part, err, mask); break;
    case 2: solve_kernel<1, 32><<<nb, ALS_THREADS, 0, s>>>(A.M, A.winv, I, R, A.Z, A.colsq_part, err, mask); break;
    default: solve_kernel<2, 32><<<nb, ALS_THREADS, 0, s>>>(A.M, A.winv, I, R, A.Z, A.colsq_part, err, mask); break;
  }
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

template <typename FT, int R>
spm_status launch_tc_scale_gram_r(int nb, const spm_als_state& A, int64_t I, void* Y, bool last,
                                  const int* err, const uint32_t* mask, cudaStream_t s) {
  constexpr int smem = (int)TcGramShape<R>::SMEM;
  SPM_CUDA_TRY(cudaFuncSetAttribute(tc_scale_gram_kernel<FT, R>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  tc_scale_gram_kernel<FT, R><<<nb, TC_THREADS, smem, s>>>(A.Z, A.lambda_ws, I, static_cast<FT*>(Y),
                                                          last ? A.M : nullptr, A.gram_part,
                                                          A.inner_part, err, mask);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

// Y = Z / lambda and the Gram partials of the stored Y (and the inner-product
// partials on the last mode) in one tensor-core pass (R = 16, 32).
__attribute__((noinline)) spm_status launch_tc_scale_gram(int R, bool bf16, int nb,
                                                          const spm_als_state& A, int64_t I,
                                                          void* Y, bool last, const int* err,
                                                          const uint32_t* mask, cudaStream_t s) {
  switch ((R == 32 ? 1 : 0) + (bf16 ? 2 : 0)) {
    case 0: return launch_tc_scale_gram_r<float, 16>(nb, A, I, Y, last, err, mask, s);
    case 1: return launch_tc_scale_gram_r<float, 32>(nb, A, I, Y, last, err, mask, s);
    case 2: return launch_tc_scale_gram_r<__nv_bfloat16, 16>(nb, A, I, Y, last, err, mask, s);
    default: return launch_tc_scale_gram_r<__nv_bfloat16, 32>(nb, A, I, Y, last, err, mask, s);
  }
}

spm_status gram(spmttkrp_plan_s* p, const void* Y, int64_t I, double* G, cudaStream_t s,
                const uint32_t* mask) {
  return p->bf16 ? launch_gram<__nv_bfloat16>(p, Y, I, G, s, mask)
                 : launch_gram<float>(p, Y, I, G, s, mask);
}

spm_status ensure_als_state(spmttkrp_plan_s* p) {
  spm_als_state& A = p->als;
  if (!A.side) SPM_CUDA_TRY(cudaStreamCreateWithFlags(&A.side, cudaStreamNonBlocking));
  if (!A.ev_fork) SPM_CUDA_TRY(cudaEventCreateWithFlags(&A.ev_fork, cudaEventDisableTiming));
  if (!A.ev_join) SPM_CUDA_TRY(cudaEventCreateWithFlags(&A.ev_join, cudaEventDisableTiming));
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
  SPM_TRY(plan_alloc(p, (void**)&A.colmax_part, sizeof(float) * R * A.gram_blocks));
  if (als_wdig_bytes(R)) SPM_TRY(plan_alloc(p, (void**)&A.wdig, als_wdig_bytes(R)));
  SPM_TRY(plan_alloc(p, (void**)&A.inner_part, sizeof(double) * R * A.gram_blocks));
  SPM_TRY(plan_alloc(p, (void**)&A.lambda_ws, sizeof(double) * 2 * R));  // lambda, Gram scales
  SPM_TRY(plan_alloc(p, (void**)&A.Z, sizeof(float) * (size_t)Imax * R));
  SPM_TRY(plan_alloc(p, (void**)&A.M, sizeof(float) * (size_t)Imax * R));
  return SPM_OK;
}


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
    // V, its Cholesky factor and V^-1 for mode d need the other modes'
    // Grams (final once the previous mode's Gram is reduced, i.e. at this
    // point of `s`), not M: they are formed on the side stream beside the
    // MTTKRP, and the solve waits for them.  The fork also orders the
    // previous mode's solve (the last reader of V^-1) before the overwrite.
    SPM_CUDA_TRY(cudaEventRecord(A.ev_fork, s));
    SPM_CUDA_TRY(cudaStreamWaitEvent(A.side, A.ev_fork, 0));
    system_kernel<<<R, SYS_THREADS, 0, A.side>>>(A.gram, N, d, R, A.chol, A.winv, A.wdig,
                                                 p->dev_err);
    SPM_CUDA_TRY(cudaGetLastError());
    SPM_CUDA_TRY(cudaEventRecord(A.ev_join, A.side));
    SPM_TRY(run_mttkrp(p, d, factors, A.M, s));
    SPM_CUDA_TRY(cudaStreamWaitEvent(s, A.ev_join, 0));
    const int nb = als_row_blocks(I, nb_solve);
    // rows without nonzeros in mode d have a zero update: passes skip them
    const uint32_t* live = p->mode[d].empty_rows > 0 ? p->mode[d].rowmask : nullptr;
    SPM_TRY(launch_solve(R, nb, A, I, p->dev_err, live, s));
    const bool tcg = tc_gram_rank(R);
    lambda_kernel<<<R, 32, 0, s>>>(A.colsq_part, tcg ? A.colmax_part : nullptr, nb, R,
                                    A.lambda_ws, p->dev_err);
    const bool last = d == N - 1;
    int nin;  // inner-product partials of the last mode
    if (tcg) {
      nin = tc_gram_blocks(I, A.gram_blocks);
      SPM_TRY(launch_tc_scale_gram(R, p->bf16, nin, A, I, factors[d], last, p->dev_err, live, s));
      gram_reduce_kernel<<<std::max(1, std::min(1024, R * R / 8)), 256, 0, s>>>(
          A.gram_part, nin, R, A.gram + (size_t)d * R * R, p->dev_err);
    } else {
      nin = als_row_blocks(I, nb_solve);
      if (p->bf16)
        scale_kernel<__nv_bfloat16><<<nin, ALS_THREADS, 0, s>>>(
            A.Z, A.lambda_ws, I, R, static_cast<__nv_bfloat16*>(factors[d]), last ? A.M : nullptr,
            A.inner_part, p->dev_err, live);
      else
        scale_kernel<float><<<nin, ALS_THREADS, 0, s>>>(A.Z, A.lambda_ws, I, R,
                                                         static_cast<float*>(factors[d]),
                                                         last ? A.M : nullptr, A.inner_part,
                                                         p->dev_err, live);
      SPM_CUDA_TRY(cudaGetLastError());
      SPM_TRY(gram(p, factors[d], I, A.gram + (size_t)d * R * R, s, live));
    }
    if (last) {
      fit_kernel<<<1, ALS_THREADS, 0, s>>>(A.gram, N, R, A.lambda_ws, A.inner_part, nin,
                                           p->normX2, fit, lambda, p->dev_err);
    }
  }
  if (!fit) copy_lambda_kernel<<<1, 256, 0, s>>>(A.lambda_ws, R, lambda, p->dev_err);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

}  // namespace spm

using namespace spm;

extern "C" spm_status spm_selftest_tc_rowpass(int R, int64_t I, const float* M, const double* V,
                                              float* Z, float* Y, double* G, double* lambda,
                                              void* stream) {
  if (!(R == 16 || R == 32 || R == 64) || !tc_solve_rank(R)) return SPM_ERR_UNSUPPORTED;
  if (I < 1 || !M || !V || !Z || !Y || !G || !lambda) return SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int cap = std::max(1, sm_count()) * 4;  // the plans' row-pass partial count
  const size_t RR = (size_t)R * R;
  spm_als_state A;
  double* grams = nullptr;
  int* err = nullptr;
  spm_status st = SPM_OK;
  auto alloc = [&](void** p, size_t bytes) {
    if (st == SPM_OK && cudaMalloc(p, bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      st = SPM_ERR_OOM;
    }
  };
  alloc((void**)&grams, sizeof(double) * 2 * RR);
  alloc((void**)&err, sizeof(int));
  alloc((void**)&A.chol, sizeof(double) * RR);
  alloc((void**)&A.winv, sizeof(float) * 2 * RR);
  alloc((void**)&A.wdig, als_wdig_bytes(R));
  alloc((void**)&A.colsq_part, sizeof(double) * R * cap);
  alloc((void**)&A.colmax_part, sizeof(float) * R * cap);
  alloc((void**)&A.lambda_ws, sizeof(double) * 2 * R);
  alloc((void**)&A.gram_part, sizeof(double) * RR * cap);
  alloc((void**)&A.inner_part, sizeof(double) * R * cap);
  if (st == SPM_OK) {
    A.M = const_cast<float*>(M);
    A.Z = Z;
    A.gram_blocks = cap;
    auto run = [&]() -> spm_status {
      SPM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
      // V = the Hadamard product over the modes other than 0 of a two-mode "tensor": grams[1]
      SPM_CUDA_TRY(cudaMemcpyAsync(grams + RR, V, sizeof(double) * RR, cudaMemcpyDeviceToDevice, s));
      system_kernel<<<R, SYS_THREADS, 0, s>>>(grams, 2, 0, R, A.chol, A.winv, A.wdig, err);
      const int nb = als_row_blocks(I, cap);
      SPM_TRY(launch_solve(R, nb, A, I, err, nullptr, s));
      const bool tcg = tc_gram_rank(R);
      lambda_kernel<<<R, 32, 0, s>>>(A.colsq_part, A.colmax_part, nb, R, A.lambda_ws, err);
      if (tcg) {
        const int nbg = tc_gram_blocks(I, cap);
        SPM_TRY(launch_tc_scale_gram(R, false, nbg, A, I, Y, false, err, nullptr, s));
        gram_reduce_kernel<<<std::max(1, std::min(1024, R * R / 8)), 256, 0, s>>>(A.gram_part, nbg, R,
                                                                                 G, err);
      } else {
        const int nbs = als_row_blocks(I, cap);
        scale_kernel<float><<<nbs, ALS_THREADS, 0, s>>>(A.Z, A.lambda_ws, I, R, Y, nullptr,
                                                         A.inner_part, err, nullptr);
      }
      SPM_CUDA_TRY(cudaMemcpyAsync(lambda, A.lambda_ws, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
      SPM_CUDA_TRY(cudaGetLastError());
      int h = 0;
      SPM_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
      SPM_CUDA_TRY(cudaStreamSynchronize(s));
      if (h & DEV_ERR_NUMERIC) return SPM_ERR_NUMERIC;
      if (h & DEV_ERR_TIMEOUT) return SPM_ERR_TIMEOUT;
      return SPM_OK;
    };
    st = run();
  }
  cudaStreamSynchronize(s);
  for (void* p : {(void*)grams, (void*)err, (void*)A.chol, (void*)A.winv, (void*)A.wdig,
                  (void*)A.colsq_part, (void*)A.colmax_part, (void*)A.lambda_ws,
                  (void*)A.gram_part, (void*)A.inner_part})
    if (p) cudaFree(p);
  (void)cudaGetLastError();
  return st;
}
