// batch.cu -- CP-ALS sweeps over a set of tensors with one launch per step
// for all of them (kernels in batch_kernels.cuh), the nnz-per-partition
// autotuner, and the C ABI of the batch object.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "batch.cuh"

namespace spm {

// grid == 0 only sets the kernel's shared-memory attributes.
spm_status launch_batch_mttkrp_f32(int kc, const BatchTensor* bt, const int2* items, int nitems,
                                   int* queue, int mode, int grid, size_t smem, cudaStream_t s);
spm_status launch_batch_mttkrp_bf16(int kc, const BatchTensor* bt, const int2* items, int nitems,
                                    int* queue, int mode, int grid, size_t smem, cudaStream_t s);

namespace {

constexpr int64_t BATCH_ZERO_WORDS = 1 << 10;  // row-bitmap words per zero-fill item

__global__ void batch_zero_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it,
                                  int mode) {
  const int2 tc = it[blockIdx.x];
  const BatchTensor& b = bt[tc.x];
  if (!b.active) return;
  const int64_t words = (b.dims[mode] + 31) / 32;
  const int64_t w0 = (int64_t)tc.y * BATCH_ZERO_WORDS;
  const int64_t w1 = std::min<int64_t>(words, w0 + BATCH_ZERO_WORDS);
  zero_empty_rows_body(b.rowmask[mode], b.dims[mode], b.R, b.M, w0 + threadIdx.x, w1, blockDim.x);
}

__global__ void batch_fixup_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it,
                                   int nitems, int mode) {
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= nitems) return;
  const int2 tz = it[i];
  const BatchTensor& b = bt[tz.x];
  if (!b.active) return;
  const MttkrpArgs& a = b.margs[mode];
  mttkrp_fixup_body(a.cta_part, a.cta_meta, b.kappa, b.R, b.M, tz.y, threadIdx.x & 31);
}

// One block per tensor: its system factored once, its columns by the warps.
__global__ void __launch_bounds__(SYS_THREADS)
    batch_system_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it, int mode) {
  const BatchTensor& b = bt[it[blockIdx.x].x];
  if (!b.active) return;
  system_col_body(b.gram, b.N, mode, b.R, 0, b.R, b.chol, b.winv, b.wdig, b.err);
}

__global__ void __launch_bounds__(ALS_THREADS)
    batch_solve_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it, int mode) {
  const int2 tv = it[blockIdx.x];
  const BatchTensor& b = bt[tv.x];
  if (!b.active) return;
  if (b.R <= 8)
    solve_body<1, 8>(b.M, b.winv, b.dims[mode], b.R, b.Z, b.colsq_part, b.err, tv.y,
                     b.nb_solve[mode], b.live[mode]);
  else if (b.R <= 16)
    solve_body<1, 16>(b.M, b.winv, b.dims[mode], b.R, b.Z, b.colsq_part, b.err, tv.y,
                      b.nb_solve[mode], b.live[mode]);
  else if (b.R <= 32)
    solve_body<1, 32>(b.M, b.winv, b.dims[mode], b.R, b.Z, b.colsq_part, b.err, tv.y,
                      b.nb_solve[mode], b.live[mode]);
  else
    solve_body<2, 32>(b.M, b.winv, b.dims[mode], b.R, b.Z, b.colsq_part, b.err, tv.y,
                      b.nb_solve[mode], b.live[mode]);
}

template <int R>
__global__ void __launch_bounds__(TC_THREADS)
    batch_tc_solve_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it, int mode) {
  const int2 tv = it[blockIdx.x];
  const BatchTensor& b = bt[tv.x];
  if (!b.active) return;
  tc_solve_body<R>(b.M, b.wdig, b.dims[mode], b.Z, b.colsq_part, b.colmax_part, b.err, tv.y,
                   b.nb_solve[mode], b.live[mode]);
}

template <int R>
spm_status launch_batch_tc_solve_r(const BatchTensor* bt, const int2* it, int n, int mode,
                                   cudaStream_t s) {
  constexpr int smem = (int)TcSolveShape<R>::SMEM;
  SPM_CUDA_TRY(cudaFuncSetAttribute(batch_tc_solve_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  batch_tc_solve_kernel<R><<<n, TC_THREADS, smem, s>>>(bt, it, mode);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

spm_status launch_batch_tc_solve(int R, const BatchTensor* bt, const int2* it, int n, int mode,
                                 cudaStream_t s) {
  switch (R) {
    case 16: return launch_batch_tc_solve_r<16>(bt, it, n, mode, s);
    case 32: return launch_batch_tc_solve_r<32>(bt, it, n, mode, s);
    case 64: return launch_batch_tc_solve_r<64>(bt, it, n, mode, s);
    default: return SPM_ERR_UNSUPPORTED;
  }
}

// Block (x, y): column y of tensor it[x] (one warp).
__global__ void batch_lambda_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it,
                                    int mode) {
  const BatchTensor& b = bt[it[blockIdx.x].x];
  if (!b.active) return;
  lambda_body(b.colsq_part, tc_gram_rank(b.R) ? b.colmax_part : nullptr, b.nb_solve[mode], b.R,
              b.lambda_ws, b.err, blockIdx.y);
}

// Y = Z / lambda with the Gram and inner-product partials on the tensor cores
// (R = 16, 32): item (tensor, virtual block).
template <typename FT, int R>
__global__ void __launch_bounds__(TC_THREADS)
    batch_tc_scale_gram_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it,
                               int mode) {
  const int2 tv = it[blockIdx.x];
  const BatchTensor& b = bt[tv.x];
  if (!b.active) return;
  tc_scale_gram_body<FT, R>(b.Z, b.lambda_ws, b.dims[mode], static_cast<FT*>(b.fac[mode]),
                            mode == b.N - 1 ? b.M : nullptr, b.gram_part, b.inner_part, b.err,
                            tv.y, b.nb_scale[mode], b.live[mode]);
}

template <typename FT, int R>
spm_status launch_batch_tc_scale_gram_r(const BatchTensor* bt, const int2* it, int n, int mode,
                                        cudaStream_t s) {
  constexpr int smem = (int)TcGramShape<R>::SMEM;
  SPM_CUDA_TRY(cudaFuncSetAttribute(batch_tc_scale_gram_kernel<FT, R>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  batch_tc_scale_gram_kernel<FT, R><<<n, TC_THREADS, smem, s>>>(bt, it, mode);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

spm_status launch_batch_tc_scale_gram(int R, bool bf16, const BatchTensor* bt, const int2* it,
                                      int n, int mode, cudaStream_t s) {
  switch ((R == 32 ? 1 : 0) + (bf16 ? 2 : 0)) {
    case 0: return launch_batch_tc_scale_gram_r<float, 16>(bt, it, n, mode, s);
    case 1: return launch_batch_tc_scale_gram_r<float, 32>(bt, it, n, mode, s);
    case 2: return launch_batch_tc_scale_gram_r<__nv_bfloat16, 16>(bt, it, n, mode, s);
    default: return launch_batch_tc_scale_gram_r<__nv_bfloat16, 32>(bt, it, n, mode, s);
  }
}

template <typename FT>
__global__ void __launch_bounds__(ALS_THREADS)
    batch_scale_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it, int mode) {
  const int2 tv = it[blockIdx.x];
  const BatchTensor& b = bt[tv.x];
  if (!b.active) return;
  const bool last = mode == b.N - 1;
  scale_body<FT>(b.Z, b.lambda_ws, b.dims[mode], b.R, static_cast<FT*>(b.fac[mode]),
                 last ? b.M : nullptr, b.inner_part, b.err, tv.y, b.nb_scale[mode], b.live[mode]);
}

// Gram partials of factor `mode` (also used for the initial Grams).
template <typename FT>
__global__ void __launch_bounds__(ALS_THREADS)
    batch_gram_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it, int mode) {
  const int2 tv = it[blockIdx.x];
  const BatchTensor& b = bt[tv.x];
  if (!b.active) return;
  const FT* y = static_cast<const FT*>(b.fac[mode]);
  const int64_t I = b.dims[mode];
  const int64_t rpb = b.gram_rpb[mode];
  switch (gram_tile(b.R)) {
    case 1: gram_partial_body<FT, 1>(y, I, b.R, rpb, b.gram_part, tv.y, b.live[mode]); break;
    case 2: gram_partial_body<FT, 2>(y, I, b.R, rpb, b.gram_part, tv.y, b.live[mode]); break;
    default: gram_partial_body<FT, 4>(y, I, b.R, rpb, b.gram_part, tv.y, b.live[mode]); break;
  }
}

__global__ void batch_gram_reduce_kernel(const BatchTensor* __restrict__ bt,
                                         const int2* __restrict__ it, int mode) {
  const BatchTensor& b = bt[it[blockIdx.x].x];
  if (!b.active) return;
  gram_reduce_body(b.gram_part, b.nb_gram[mode], b.R, b.gram + (int64_t)mode * b.R * b.R, b.err,
                   0, 1);
}

// Fit after the tensor's last mode, then the convergence decision.
__global__ void __launch_bounds__(ALS_THREADS)
    batch_fit_kernel(BatchTensor* __restrict__ bt, const int2* __restrict__ it, int mode) {
  BatchTensor& b = bt[it[blockIdx.x].x];
  if (!b.active) return;
  fit_body(b.gram, b.N, b.R, b.lambda_ws, b.inner_part, b.nb_scale[mode], b.normX2, b.fit_out,
           b.lambda_out, b.err);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double f = *b.fit_out;
    b.sweeps += 1;
    const bool failed = *b.err != 0;
    if (failed || b.sweeps >= b.max_sweeps || fabs(f - b.prev_fit) < b.tol) b.active = 0;
    b.prev_fit = f;
  }
}


template <typename T>
spm_status grow(T** buf, size_t* cap, size_t need) {
  if (need <= *cap) return SPM_OK;
  const size_t n = std::max(need, *cap + *cap / 2);
  if (*buf) {
    cudaFree(*buf);  // synchronises the device: queued work is done with it
    *buf = nullptr;
    *cap = 0;
  }
  cudaError_t e = cudaMalloc((void**)buf, sizeof(T) * n);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *buf = nullptr;
    return e == cudaErrorMemoryAllocation ? SPM_ERR_OOM : SPM_ERR_CUDA;
  }
  *cap = n;
  return SPM_OK;
}

}  // namespace

spm_status batch_add(spm_batch_s* B, spmttkrp_plan_s* p, void* const* factors, double* lambda,
                     double* fit, double tol, int max_sweeps, cudaStream_t s, int start_sweeps,
                     double prev_fit) {
  if (!p || !factors || !lambda || !fit || max_sweeps < 1 || !(tol >= 0.0) || start_sweeps < 0 ||
      start_sweeps >= max_sweeps)
    return SPM_ERR_INVALID_ARG;
  const int kc = batch_kclass(p->N, p->R);
  if (kc == KC_NONE || p->lean || p->fibre || (B->bf16 >= 0 && B->bf16 != (int)p->bf16))
    return SPM_ERR_UNSUPPORTED;
  for (int d = 0; d < p->N; ++d)
    if (p->mode[d].scheme == 1) return SPM_ERR_UNSUPPORTED;
  for (int w = 0; w < p->N; ++w)
    if (!factors[w] || (reinterpret_cast<uintptr_t>(factors[w]) & 15u)) return SPM_ERR_INVALID_ARG;
  if (!B->side) SPM_CUDA_TRY(cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking));
  if (!B->ev_fork) SPM_CUDA_TRY(cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming));
  if (!B->ev_join) SPM_CUDA_TRY(cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming));
  for (const spmttkrp_plan_s* q : B->plans)
    if (q == p) return SPM_ERR_INVALID_ARG;  // one batch slot per plan (shared workspace)
  // the members' convergence state lives on the device between sweeps
  if (!B->dirty) SPM_TRY(batch_pull(B, s));
  SPM_TRY(ensure_als_state(p));
  spm_als_state& A = p->als;
  A.ready = false;  // the batch keeps the Grams from now on
  BatchTensor b{};
  b.N = p->N;
  b.R = p->R;
  b.kappa = p->kappa;
  b.kclass = kc;
  b.gram = A.gram;
  b.gram_part = A.gram_part;
  b.chol = A.chol;
  b.winv = A.winv;
  b.colsq_part = A.colsq_part;
  b.colmax_part = A.colmax_part;
  b.wdig = A.wdig;
  b.inner_part = A.inner_part;
  b.lambda_ws = A.lambda_ws;
  b.M = A.M;
  b.Z = A.Z;
  b.normX2 = p->normX2;
  b.err = p->dev_err;
  b.lambda_out = lambda;
  b.fit_out = fit;
  b.active = 1;
  b.sweeps = start_sweeps;
  b.max_sweeps = max_sweeps;
  b.tol = tol;
  b.prev_fit = prev_fit;
  for (int w = 0; w < p->N; ++w) b.fac[w] = factors[w];
  for (int d = 0; d < p->N; ++d) {
    const int64_t I = p->dims[d];
    b.dims[d] = I;
    b.rowmask[d] = p->mode[d].rowmask;
    b.live[d] = p->mode[d].empty_rows > 0 ? p->mode[d].rowmask : nullptr;
    MttkrpArgs& a = b.margs[d];
    a = MttkrpArgs{};
    a.rec = p->mode[d].rec;
    a.woff = p->mode[d].woff;
    int m = 0;
    for (int w = 0; w < p->N; ++w)
      if (w != d) a.fac[m++] = b.fac[w];
    a.out = A.M;
    a.cta_part = p->cta_part;  // the modes run one after another: one workspace
    a.cta_meta = p->cta_meta;
    a.err = p->dev_err;
    a.nnz = p->nnz;
    a.I = I;
    a.R = p->R;
    a.nin = p->N - 1;
    a.nu = p->nu;
    // the single-tensor sweep's virtual block counts (identical sums)
    b.nb_gram[d] = als_row_blocks(I, A.gram_blocks);
    b.gram_rpb[d] = ceil_div<int64_t>(I, b.nb_gram[d]);
    b.nb_solve[d] = als_row_blocks(I, A.gram_blocks);
    b.nb_scale[d] = als_row_blocks(I, A.gram_blocks);
    if (tc_gram_rank(p->R))  // the tensor-core normalisation/Gram pass: its own split
      b.nb_gram[d] = b.nb_scale[d] = tc_gram_blocks(I, A.gram_blocks);
  }
  for (int w = 0; w < p->N; ++w)
    SPM_TRY(gram(p, factors[w], p->dims[w], A.gram + (size_t)w * p->R * p->R, s));
  B->plans.push_back(p);
  B->host.push_back(b);
  B->bf16 = p->bf16 ? 1 : 0;
  B->dirty = true;
  return SPM_OK;
}

void batch_remove(spm_batch_s* B, int t) {
  B->plans.erase(B->plans.begin() + t);
  B->host.erase(B->host.begin() + t);
  if (B->plans.empty()) B->bf16 = -1;
  B->dirty = true;
}

spm_status batch_pull(spm_batch_s* B, cudaStream_t s) {
  if (B->bt && !B->host.empty() && !B->dirty)
    SPM_CUDA_TRY(cudaMemcpyAsync(B->host.data(), B->bt, sizeof(BatchTensor) * B->host.size(),
                                 cudaMemcpyDeviceToHost, s));
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  return SPM_OK;
}

spm_status batch_commit(spm_batch_s* B, cudaStream_t s) {
  if (!B->dirty) return SPM_OK;
  const int n = (int)B->host.size();
  B->maxN = 0;
  B->maxR = 1;
  for (int kc = 0; kc < KC_NONE; ++kc) B->mtt_smem[kc] = 0;
  for (int t = 0; t < n; ++t) {
    const spmttkrp_plan_s* p = B->plans[t];
    B->maxN = std::max(B->maxN, p->N);
    B->maxR = std::max(B->maxR, p->R);
    // partitions may have changed since the tensor was added (autotuning)
    B->host[t].kappa = p->kappa;
    for (int d = 0; d < p->N; ++d) B->host[t].margs[d].woff = p->mode[d].woff;
    const int kc = B->host[t].kclass;
    B->mtt_smem[kc] =
        std::max(B->mtt_smem[kc], mttkrp_smem_bytes(p->R, record_int4s(p->N), p->nu, p->bf16 ? 2 : 4));
  }
  std::vector<int2>& v = B->stage;
  v.clear();
  for (int d = 0; d < SPM_MAX_MODES; ++d) {
    spm_batch_s::ModeItems& I = B->mi[d];
    I = spm_batch_s::ModeItems{};
    for (int kc = 0; kc < KC_NONE; ++kc) {
      I.mtt_off[kc] = (int)v.size();
      for (int t = 0; t < n; ++t) {
        const spmttkrp_plan_s* p = B->plans[t];
        if (d < p->N && B->host[t].kclass == kc && p->nnz > 0)
          for (int z = 0; z < p->kappa; ++z) v.push_back(make_int2(t, z));
      }
      I.n_mtt[kc] = (int)v.size() - I.mtt_off[kc];
    }
    I.zero_off = (int)v.size();
    for (int t = 0; t < n; ++t) {
      const spmttkrp_plan_s* p = B->plans[t];
      // an empty tensor has no partition items: its row masks are all
      // clear, so the zero-fill items cover its whole output
      if (d < p->N && (p->nnz == 0 || p->mode[d].empty_rows > 0)) {
        const int64_t chunks = ceil_div<int64_t>((p->dims[d] + 31) / 32, BATCH_ZERO_WORDS);
        for (int64_t c = 0; c < chunks; ++c) v.push_back(make_int2(t, (int)c));
      }
    }
    I.n_zero = (int)v.size() - I.zero_off;
    auto per_tensor = [&](int* off, int* cnt, auto count) {
      *off = (int)v.size();
      for (int t = 0; t < n; ++t) {
        if (d >= B->plans[t]->N) continue;
        const int k = count(t);
        for (int j = 0; j < k; ++j) v.push_back(make_int2(t, j));
      }
      *cnt = (int)v.size() - *off;
    };
    per_tensor(&I.tens_off, &I.n_tens, [&](int) { return 1; });
    per_tensor(&I.solve_off, &I.n_solve, [&](int t) {
      return tc_solve_rank(B->plans[t]->R) ? 0 : B->host[t].nb_solve[d];
    });
    for (int k = 0; k < 3; ++k)
      per_tensor(&I.tcs_off[k], &I.n_tcs[k], [&](int t) {
        const int R = B->plans[t]->R;
        return tc_solve_rank(R) && R == (16 << k) ? B->host[t].nb_solve[d] : 0;
      });
    per_tensor(&I.scale_off, &I.n_scale, [&](int t) {
      return tc_gram_rank(B->plans[t]->R) ? 0 : B->host[t].nb_scale[d];
    });
    per_tensor(&I.gram_off, &I.n_gram, [&](int t) {
      return tc_gram_rank(B->plans[t]->R) ? 0 : B->host[t].nb_gram[d];
    });
    for (int k = 0; k < 2; ++k)
      per_tensor(&I.tcg_off[k], &I.n_tcg[k], [&](int t) {
        const int R = B->plans[t]->R;
        return tc_gram_rank(R) && R == (16 << k) ? B->host[t].nb_scale[d] : 0;
      });
    per_tensor(&I.fit_off, &I.n_fit, [&](int t) { return d == B->plans[t]->N - 1 ? 1 : 0; });
  }
  SPM_TRY(grow(&B->bt, &B->bt_cap, std::max<size_t>(1, n)));
  SPM_TRY(grow(&B->items, &B->items_cap, std::max<size_t>(1, v.size())));
  if (!B->queue) SPM_CUDA_TRY(cudaMalloc((void**)&B->queue, sizeof(int) * SPM_MAX_MODES * KC_NONE));
  if (n > 0)
    SPM_CUDA_TRY(cudaMemcpyAsync(B->bt, B->host.data(), sizeof(BatchTensor) * n,
                                 cudaMemcpyHostToDevice, s));
  if (!v.empty())
    SPM_CUDA_TRY(cudaMemcpyAsync(B->items, v.data(), sizeof(int2) * v.size(),
                                 cudaMemcpyHostToDevice, s));
  for (int kc = 0; kc < KC_NONE; ++kc) {
    if (B->mtt_smem[kc] == 0 || B->mtt_smem[kc] <= B->smem_set[kc]) continue;
    SPM_TRY(B->bf16 == 1 ? launch_batch_mttkrp_bf16(kc, nullptr, nullptr, 0, nullptr, 0, 0,
                                                    B->mtt_smem[kc], s)
                         : launch_batch_mttkrp_f32(kc, nullptr, nullptr, 0, nullptr, 0, 0,
                                                   B->mtt_smem[kc], s));
    B->smem_set[kc] = B->mtt_smem[kc];
  }
  if (B->grid == 0) B->grid = std::max(1, sm_count());
  // the staged host vectors must outlive the asynchronous copies
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  B->dirty = false;
  return SPM_OK;
}

spm_status batch_mttkrp(spm_batch_s* B, int d, cudaStream_t s) {
  const spm_batch_s::ModeItems& I = B->mi[d];
  if (I.n_zero > 0) batch_zero_kernel<<<I.n_zero, 256, 0, s>>>(B->bt, B->items + I.zero_off, d);
  int* q = B->queue + d * KC_NONE;
  SPM_CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(int) * KC_NONE, s));
  for (int kc = 0; kc < KC_NONE; ++kc) {
    const int n = I.n_mtt[kc];
    if (n == 0) continue;
    const int grid = std::min(B->grid, n);
    const int2* it = B->items + I.mtt_off[kc];
    SPM_TRY(B->bf16 == 1
                ? launch_batch_mttkrp_bf16(kc, B->bt, it, n, q + kc, d, grid, B->mtt_smem[kc], s)
                : launch_batch_mttkrp_f32(kc, B->bt, it, n, q + kc, d, grid, B->mtt_smem[kc], s));
  }
  for (int kc = 0; kc < KC_NONE; ++kc) {
    const int n = I.n_mtt[kc];
    if (n == 0) continue;
    batch_fixup_kernel<<<(int)ceil_div<int64_t>((int64_t)n * 32, 256), 256, 0, s>>>(
        B->bt, B->items + I.mtt_off[kc], n, d);
  }
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

spm_status batch_sweep(spm_batch_s* B, cudaStream_t s) {
  SPM_TRY(batch_commit(B, s));
  if (B->host.empty()) return SPM_OK;
  const int2* it = B->items;
  for (int d = 0; d < B->maxN; ++d) {
    const spm_batch_s::ModeItems& I = B->mi[d];
    // each member's system for mode d needs its other modes' Grams (final at
    // this point of `s`), not its MTTKRP: formed on the side stream beside
    // the MTTKRP launches; the fork also orders the previous mode's solve
    // before V^-1 is overwritten
    const bool fork = B->side && B->ev_fork && B->ev_join;
    cudaStream_t ss = fork ? B->side : s;
    if (fork) {
      SPM_CUDA_TRY(cudaEventRecord(B->ev_fork, s));
      SPM_CUDA_TRY(cudaStreamWaitEvent(B->side, B->ev_fork, 0));
    }
    batch_system_kernel<<<I.n_tens, SYS_THREADS, 0, ss>>>(B->bt, it + I.tens_off, d);
    SPM_CUDA_TRY(cudaGetLastError());
    if (fork) SPM_CUDA_TRY(cudaEventRecord(B->ev_join, B->side));
    SPM_TRY(batch_mttkrp(B, d, s));
    if (fork) SPM_CUDA_TRY(cudaStreamWaitEvent(s, B->ev_join, 0));
    if (I.n_solve > 0) batch_solve_kernel<<<I.n_solve, ALS_THREADS, 0, s>>>(B->bt, it + I.solve_off, d);
    for (int k = 0; k < 3; ++k)
      if (I.n_tcs[k] > 0) SPM_TRY(launch_batch_tc_solve(16 << k, B->bt, it + I.tcs_off[k], I.n_tcs[k], d, s));
    batch_lambda_kernel<<<dim3(I.n_tens, B->maxR), 32, 0, s>>>(B->bt, it + I.tens_off, d);
    if (I.n_scale > 0) {
      if (B->bf16 == 1)
        batch_scale_kernel<__nv_bfloat16><<<I.n_scale, ALS_THREADS, 0, s>>>(B->bt, it + I.scale_off, d);
      else
        batch_scale_kernel<float><<<I.n_scale, ALS_THREADS, 0, s>>>(B->bt, it + I.scale_off, d);
    }
    if (I.n_gram > 0) {
      if (B->bf16 == 1)
        batch_gram_kernel<__nv_bfloat16><<<I.n_gram, ALS_THREADS, 0, s>>>(B->bt, it + I.gram_off, d);
      else
        batch_gram_kernel<float><<<I.n_gram, ALS_THREADS, 0, s>>>(B->bt, it + I.gram_off, d);
    }
    for (int k = 0; k < 2; ++k)
      if (I.n_tcg[k] > 0)
        SPM_TRY(launch_batch_tc_scale_gram(16 << k, B->bf16 == 1, B->bt, it + I.tcg_off[k],
                                           I.n_tcg[k], d, s));
    batch_gram_reduce_kernel<<<I.n_tens, 256, 0, s>>>(B->bt, it + I.tens_off, d);
    if (I.n_fit > 0) batch_fit_kernel<<<I.n_fit, ALS_THREADS, 0, s>>>(B->bt, it + I.fit_off, d);
    SPM_CUDA_TRY(cudaGetLastError());
  }
  return SPM_OK;
}

void batch_free(spm_batch_s* B) {
  if (!B) return;
  cudaDeviceSynchronize();
  if (B->bt) cudaFree(B->bt);
  if (B->items) cudaFree(B->items);
  if (B->queue) cudaFree(B->queue);
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->ev_join) cudaEventDestroy(B->ev_join);
  if (B->side) cudaStreamDestroy(B->side);
  (void)cudaGetLastError();
  delete B;
}

}  // namespace spm

using namespace spm;

extern "C" {

spm_status spm_batch_create(spm_batch_t* out, int ntensors, const spmttkrp_plan_t* plans,
                            void* const* factors, double* lambdas, double* fits, double tol,
                            int max_sweeps, void* stream) {
  if (!out) return SPM_ERR_INVALID_ARG;
  *out = nullptr;
  if (ntensors < 1 || !plans || !factors || !lambdas || !fits || max_sweeps < 1 || !(tol >= 0.0))
    return SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int t = 0; t < ntensors; ++t) {
    const spmttkrp_plan_s* p = plans[t];
    if (!p) return SPM_ERR_INVALID_ARG;
    if (p->bf16 != plans[0]->bf16 || p->lean || p->fibre || batch_kclass(p->N, p->R) == KC_NONE)
      return SPM_ERR_UNSUPPORTED;
  }
  spm_batch_s* B = new (std::nothrow) spm_batch_s();
  if (!B) return SPM_ERR_OOM;
  cudaGetDevice(&B->device);
  spm_status st = SPM_OK;
  size_t lam_off = 0;
  for (int t = 0; t < ntensors && st == SPM_OK; ++t) {
    st = batch_add(B, plans[t], factors + (size_t)t * SPM_MAX_MODES, lambdas + lam_off, fits + t,
                   tol, max_sweeps, s);
    lam_off += (size_t)plans[t]->R;
  }
  if (st == SPM_OK) st = batch_commit(B, s);
  if (st == SPM_OK && cudaStreamSynchronize(s) != cudaSuccess) st = SPM_ERR_CUDA;
  if (st != SPM_OK) {
    (void)cudaGetLastError();
    batch_free(B);
    return st;
  }
  *out = B;
  return SPM_OK;
}

spm_status spm_batch_sweep(spm_batch_t B, void* stream) {
  NvtxScope nv("spm_batch_sweep");
  if (!B) return SPM_ERR_INVALID_ARG;
  return batch_sweep(B, static_cast<cudaStream_t>(stream));
}

spm_status spm_batch_status(spm_batch_t B, int* active, int* sweeps, void* stream) {
  if (!B || !active) return SPM_ERR_INVALID_ARG;
  SPM_TRY(batch_pull(B, static_cast<cudaStream_t>(stream)));
  for (size_t t = 0; t < B->host.size(); ++t) {
    active[t] = B->host[t].active;
    if (sweeps) sweeps[t] = B->host[t].sweeps;
  }
  return SPM_OK;
}

void spm_batch_destroy(spm_batch_t B) { batch_free(B); }

spm_status spm_batch_autotune(int ntensors, const spmttkrp_plan_t* plans, void* const* factors,
                              const int64_t* candidates, int ncandidates, int reps,
                              int64_t* chosen, float* ms, void* stream) {
  if (ntensors < 1 || !plans || !factors || !candidates || ncandidates < 1 || reps < 1 || !chosen)
    return SPM_ERR_INVALID_ARG;
  for (int c = 0; c < ncandidates; ++c)
    if (candidates[c] < 0) return SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto kappa_for = [&](const spmttkrp_plan_s* p, int64_t target) -> int {
    if (target == 0) return default_kappa();
    return (int)std::max<int64_t>(1, std::min<int64_t>(0xFFFF, ceil_div<int64_t>(p->nnz, target)));
  };
  // scratch weights and fits for the timing batches
  size_t rsum = 0;
  for (int t = 0; t < ntensors; ++t) {
    if (!plans[t]) return SPM_ERR_INVALID_ARG;
    rsum += (size_t)plans[t]->R;
  }
  double* scratch = nullptr;
  SPM_CUDA_TRY(cudaMalloc((void**)&scratch, sizeof(double) * (rsum + ntensors)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  spm_status st = SPM_OK;
  float best_ms = 0.f;
  int best = -1;
  for (int c = 0; c < ncandidates && st == SPM_OK; ++c) {
    for (int t = 0; t < ntensors && st == SPM_OK; ++t)
      st = plan_repartition(plans[t], kappa_for(plans[t], candidates[c]), s);
    spm_batch_s* B = nullptr;
    if (st == SPM_OK)
      st = spm_batch_create(&B, ntensors, plans, factors, scratch, scratch + rsum, 0.0, 1, stream);
    float t_min = 0.f;
    for (int r = 0; r <= reps && st == SPM_OK; ++r) {  // r == 0 warms up
      cudaEventRecord(e0, s);
      for (int d = 0; d < B->maxN && st == SPM_OK; ++d) st = batch_mttkrp(B, d, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = SPM_ERR_CUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r == 1 || (r > 1 && t < t_min)) t_min = t;
    }
    if (B) batch_free(B);
    if (st != SPM_OK) break;
    if (ms) ms[c] = t_min;
    if (best < 0 || t_min < best_ms) {
      best_ms = t_min;
      best = c;
    }
  }
  if (st == SPM_OK) {
    for (int t = 0; t < ntensors && st == SPM_OK; ++t)
      st = plan_repartition(plans[t], kappa_for(plans[t], candidates[best]), s);
    *chosen = candidates[best];
  }
  for (int t = 0; t < ntensors; ++t) plans[t]->als.ready = false;
  if (st == SPM_OK && cudaStreamSynchronize(s) != cudaSuccess) st = SPM_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  (void)cudaGetLastError();
  return st;
}

}  // extern "C"
