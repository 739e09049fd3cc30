// batch.cu -- CP-ALS sweeps over many tensors, one launch per step for all
// of them (see batch_kernels.cuh), and the C ABI of the batch object.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "batch_kernels.cuh"

struct spm_batch_s {
  int n = 0;
  int maxN = 0;
  bool bf16 = false;
  int device = 0;
  std::vector<spmttkrp_plan_s*> plans;
  std::vector<spm::BatchTensor> host;
  spm::BatchTensor* bt = nullptr;  // device copy of `host`
  struct Items {
    int2* mtt[spm::KC_NONE] = {};
    int n_mtt[spm::KC_NONE] = {};  // (tensor, partition) per (N, R) class
    int2* zero = nullptr;
    int n_zero = 0;  // (tensor, element chunk)
    int2* tens = nullptr;
    int n_tens = 0;  // (tensor, 0): tensors that have this mode
    int2* solve = nullptr;
    int n_solve = 0;  // (tensor, virtual block)
    int2* scale = nullptr;
    int n_scale = 0;
    int2* gram = nullptr;
    int n_gram = 0;
    int2* fit = nullptr;
    int n_fit = 0;  // tensors whose last mode is this one
  } items[SPM_MAX_MODES];
  int* queue = nullptr;  // work-queue counters, one per (mode, class)
  size_t mtt_smem[spm::KC_NONE] = {};
  int grid = 0;  // persistent blocks of the MTTKRP launch
  std::vector<void*> allocs;
};

namespace spm {

// grid == 0 only sets the kernel's shared-memory attributes.
spm_status launch_batch_mttkrp_f32(int kc, const BatchTensor* bt, const int2* items, int nitems,
                                   int* queue, int mode, int grid, size_t smem, cudaStream_t s);
spm_status launch_batch_mttkrp_bf16(int kc, const BatchTensor* bt, const int2* items, int nitems,
                                    int* queue, int mode, int grid, size_t smem, cudaStream_t s);

namespace {

constexpr int64_t ZERO_CHUNK = 1 << 16;  // output elements per zero-fill item

__global__ void batch_zero_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it,
                                  int mode) {
  const int2 tc = it[blockIdx.x];
  const BatchTensor& b = bt[tc.x];
  if (!b.active) return;
  const int64_t n = b.dims[mode] * b.R;
  const int64_t x0 = (int64_t)tc.y * ZERO_CHUNK;
  const int64_t x1 = std::min<int64_t>(n, x0 + ZERO_CHUNK);
  zero_empty_rows_body(b.rowmask[mode], b.R, b.M, x0 + threadIdx.x, x1, blockDim.x);
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

__global__ void __launch_bounds__(ALS_THREADS)
    batch_system_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it, int mode) {
  const BatchTensor& b = bt[it[blockIdx.x].x];
  if (!b.active) return;
  system_body(b.gram, b.N, mode, b.R, b.chol, b.winv, b.err);
}

__global__ void __launch_bounds__(ALS_THREADS)
    batch_solve_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it, int mode) {
  const int2 tv = it[blockIdx.x];
  const BatchTensor& b = bt[tv.x];
  if (!b.active) return;
  if (b.R <= 32)
    solve_body<1>(b.M, b.winv, b.dims[mode], b.R, b.Z, b.colsq_part, b.err, tv.y, b.nb_solve[mode]);
  else
    solve_body<2>(b.M, b.winv, b.dims[mode], b.R, b.Z, b.colsq_part, b.err, tv.y, b.nb_solve[mode]);
}

__global__ void batch_lambda_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it,
                                    int mode) {
  const BatchTensor& b = bt[it[blockIdx.x].x];
  if (!b.active) return;
  lambda_body(b.colsq_part, b.nb_solve[mode], b.R, b.lambda_ws, b.err);
}

template <typename FT>
__global__ void __launch_bounds__(ALS_THREADS)
    batch_scale_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ it, int mode) {
  const int2 tv = it[blockIdx.x];
  const BatchTensor& b = bt[tv.x];
  if (!b.active) return;
  const bool last = mode == b.N - 1;
  scale_body<FT>(b.Z, b.lambda_ws, b.dims[mode], b.R, static_cast<FT*>(b.fac[mode]),
                 last ? b.M : nullptr, b.inner_part, b.err, tv.y, b.nb_scale[mode]);
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
    case 1: gram_partial_body<FT, 1>(y, I, b.R, rpb, b.gram_part, tv.y); break;
    case 2: gram_partial_body<FT, 2>(y, I, b.R, rpb, b.gram_part, tv.y); break;
    default: gram_partial_body<FT, 4>(y, I, b.R, rpb, b.gram_part, tv.y); break;
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
spm_status upload(spm_batch_s* B, T** dst, const std::vector<T>& v, cudaStream_t s) {
  *dst = nullptr;
  if (v.empty()) return SPM_OK;
  void* p = nullptr;
  SPM_CUDA_TRY(cudaMalloc(&p, sizeof(T) * v.size()));
  B->allocs.push_back(p);
  SPM_CUDA_TRY(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
  *dst = static_cast<T*>(p);
  return SPM_OK;
}

void free_batch(spm_batch_s* B) {
  if (!B) return;
  cudaDeviceSynchronize();
  for (void* p : B->allocs) cudaFree(p);
  (void)cudaGetLastError();
  delete B;
}

// One batched Gram refresh of factor `mode` for every tensor that has it.
spm_status batch_gram(spm_batch_s* B, int mode, cudaStream_t s) {
  auto& I = B->items[mode];
  if (I.n_gram == 0) return SPM_OK;
  if (B->bf16) batch_gram_kernel<__nv_bfloat16><<<I.n_gram, ALS_THREADS, 0, s>>>(B->bt, I.gram, mode);
  else batch_gram_kernel<float><<<I.n_gram, ALS_THREADS, 0, s>>>(B->bt, I.gram, mode);
  batch_gram_reduce_kernel<<<I.n_tens, 256, 0, s>>>(B->bt, I.tens, mode);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

}  // namespace
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
  const bool bf16 = plans[0] && plans[0]->bf16;
  for (int t = 0; t < ntensors; ++t) {
    const spmttkrp_plan_s* p = plans[t];
    if (!p) return SPM_ERR_INVALID_ARG;
    if (p->bf16 != bf16 || batch_kclass(p->N, p->R) == KC_NONE) return SPM_ERR_UNSUPPORTED;
    for (int d = 0; d < p->N; ++d)
      if (p->mode[d].scheme == 1) return SPM_ERR_UNSUPPORTED;
    for (int w = 0; w < p->N; ++w) {
      const void* f = factors[(size_t)t * SPM_MAX_MODES + w];
      if (!f || (reinterpret_cast<uintptr_t>(f) & 15u)) return SPM_ERR_INVALID_ARG;
    }
  }
  spm_batch_s* B = new (std::nothrow) spm_batch_s();
  if (!B) return SPM_ERR_OOM;
  cudaGetDevice(&B->device);
  B->n = ntensors;
  B->bf16 = bf16;
  B->plans.assign(plans, plans + ntensors);
  B->host.resize(ntensors);
  std::vector<int2> mtt[SPM_MAX_MODES][KC_NONE], zero[SPM_MAX_MODES], tens[SPM_MAX_MODES],
      solve[SPM_MAX_MODES], scale[SPM_MAX_MODES], gram[SPM_MAX_MODES], fit[SPM_MAX_MODES];
  size_t lam_off = 0;
  spm_status st = SPM_OK;
  for (int t = 0; t < ntensors && st == SPM_OK; ++t) {
    spmttkrp_plan_s* p = plans[t];
    st = ensure_als_state(p);
    if (st != SPM_OK) break;
    spm_als_state& A = p->als;
    A.ready = false;  // the batch owns the Grams from now on
    BatchTensor& b = B->host[t];
    b = BatchTensor{};
    b.N = p->N;
    b.R = p->R;
    b.kappa = p->kappa;
    b.kclass = batch_kclass(p->N, p->R);
    B->maxN = std::max(B->maxN, p->N);
    b.gram = A.gram;
    b.gram_part = A.gram_part;
    b.chol = A.chol;
    b.winv = A.winv;
    b.colsq_part = A.colsq_part;
    b.inner_part = A.inner_part;
    b.lambda_ws = A.lambda_ws;
    b.M = A.M;
    b.Z = A.Z;
    b.normX2 = p->normX2;
    b.err = p->dev_err;
    b.lambda_out = lambdas + lam_off;
    lam_off += (size_t)p->R;
    b.fit_out = fits + t;
    b.active = 1;
    b.sweeps = 0;
    b.max_sweeps = max_sweeps;
    b.tol = tol;
    b.prev_fit = -1.0e300;
    for (int w = 0; w < p->N; ++w) b.fac[w] = factors[(size_t)t * SPM_MAX_MODES + w];
    for (int d = 0; d < p->N; ++d) {
      const int64_t I = p->dims[d];
      b.dims[d] = I;
      b.rowmask[d] = p->mode[d].rowmask;
      MttkrpArgs& a = b.margs[d];
      a = MttkrpArgs{};
      a.rec = p->mode[d].rec;
      a.woff = p->mode[d].woff;
      int m = 0;
      for (int w = 0; w < p->N; ++w)
        if (w != d) a.fac[m++] = b.fac[w];
      a.out = A.M;
      a.cta_part = p->cta_part;  // modes run one after another: the workspace is reused
      a.cta_meta = p->cta_meta;
      a.err = p->dev_err;
      a.nnz = p->nnz;
      a.I = I;
      a.R = p->R;
      a.nin = p->N - 1;
      a.nu = p->nu;
      // same virtual block counts as the single-tensor sweep (identical sums)
      b.nb_gram[d] = work_blocks(I, GRAM_TILE_ROWS, A.gram_blocks);
      b.gram_rpb[d] = ceil_div<int64_t>(I, b.nb_gram[d]);
      b.nb_solve[d] = work_blocks(I, 4 * (ALS_THREADS / 32), A.gram_blocks);
      b.nb_scale[d] = work_blocks(I, ALS_THREADS / p->R, A.gram_blocks);
      if (p->nnz > 0)
        for (int z = 0; z < p->kappa; ++z) mtt[d][b.kclass].push_back(make_int2(t, z));
      if (p->nnz == 0 || p->mode[d].empty_rows > 0) {
        const int64_t chunks = ceil_div<int64_t>(I * p->R, ZERO_CHUNK);
        for (int64_t c = 0; c < chunks; ++c) zero[d].push_back(make_int2(t, (int)c));
      }
      tens[d].push_back(make_int2(t, 0));
      for (int v = 0; v < b.nb_solve[d]; ++v) solve[d].push_back(make_int2(t, v));
      for (int v = 0; v < b.nb_scale[d]; ++v) scale[d].push_back(make_int2(t, v));
      for (int v = 0; v < b.nb_gram[d]; ++v) gram[d].push_back(make_int2(t, v));
      if (d == p->N - 1) fit[d].push_back(make_int2(t, 0));
      B->mtt_smem[b.kclass] = std::max(B->mtt_smem[b.kclass],
                                       mttkrp_smem_bytes(p->R, record_int4s(p->N), p->nu));
    }
    // an empty tensor has no partition items: its row masks are all clear,
    // so the zero-fill items cover its whole output
  }
  for (int d = 0; d < SPM_MAX_MODES && st == SPM_OK; ++d) {
    auto& I = B->items[d];
    I.n_zero = (int)zero[d].size();
    I.n_tens = (int)tens[d].size();
    I.n_solve = (int)solve[d].size();
    I.n_scale = (int)scale[d].size();
    I.n_gram = (int)gram[d].size();
    I.n_fit = (int)fit[d].size();
    for (int kc = 0; kc < KC_NONE; ++kc) {
      I.n_mtt[kc] = (int)mtt[d][kc].size();
      if (st == SPM_OK) st = upload(B, &I.mtt[kc], mtt[d][kc], s);
    }
    if (st == SPM_OK) st = upload(B, &I.zero, zero[d], s);
    if (st == SPM_OK) st = upload(B, &I.tens, tens[d], s);
    if (st == SPM_OK) st = upload(B, &I.solve, solve[d], s);
    if (st == SPM_OK) st = upload(B, &I.scale, scale[d], s);
    if (st == SPM_OK) st = upload(B, &I.gram, gram[d], s);
    if (st == SPM_OK) st = upload(B, &I.fit, fit[d], s);
  }
  if (st == SPM_OK) st = upload(B, &B->bt, B->host, s);
  if (st == SPM_OK) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(int) * SPM_MAX_MODES * KC_NONE) != cudaSuccess) st = SPM_ERR_OOM;
    else {
      B->allocs.push_back(q);
      B->queue = static_cast<int*>(q);
    }
  }
  B->grid = std::max(1, sm_count());
  // kernel attributes once, so that a sweep only launches (graph capture)
  for (int kc = 0; kc < KC_NONE && st == SPM_OK; ++kc)
    if (B->mtt_smem[kc] > 0)
      st = bf16 ? launch_batch_mttkrp_bf16(kc, nullptr, nullptr, 0, nullptr, 0, 0, B->mtt_smem[kc], s)
                : launch_batch_mttkrp_f32(kc, nullptr, nullptr, 0, nullptr, 0, 0, B->mtt_smem[kc], s);
  // initial Grams of every factor
  for (int w = 0; w < B->maxN && st == SPM_OK; ++w) st = batch_gram(B, w, s);
  if (st == SPM_OK && cudaStreamSynchronize(s) != cudaSuccess) st = SPM_ERR_CUDA;
  if (st != SPM_OK) {
    (void)cudaGetLastError();
    free_batch(B);
    return st;
  }
  *out = B;
  return SPM_OK;
}

spm_status spm_batch_sweep(spm_batch_t B, void* stream) {
  if (!B) return SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int d = 0; d < B->maxN; ++d) {
    auto& I = B->items[d];
    if (I.n_zero > 0) batch_zero_kernel<<<I.n_zero, 256, 0, s>>>(B->bt, I.zero, d);
    int* q = B->queue + d * KC_NONE;
    SPM_CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(int) * KC_NONE, s));
    for (int kc = 0; kc < KC_NONE; ++kc) {
      const int n = I.n_mtt[kc];
      if (n == 0) continue;
      const int grid = std::min(B->grid, n);
      SPM_TRY(B->bf16 ? launch_batch_mttkrp_bf16(kc, B->bt, I.mtt[kc], n, q + kc, d, grid,
                                                 B->mtt_smem[kc], s)
                      : launch_batch_mttkrp_f32(kc, B->bt, I.mtt[kc], n, q + kc, d, grid,
                                                B->mtt_smem[kc], s));
    }
    for (int kc = 0; kc < KC_NONE; ++kc) {
      const int n = I.n_mtt[kc];
      if (n == 0) continue;
      batch_fixup_kernel<<<(int)ceil_div<int64_t>((int64_t)n * 32, 256), 256, 0, s>>>(
          B->bt, I.mtt[kc], n, d);
    }
    batch_system_kernel<<<I.n_tens, ALS_THREADS, 0, s>>>(B->bt, I.tens, d);
    batch_solve_kernel<<<I.n_solve, ALS_THREADS, 0, s>>>(B->bt, I.solve, d);
    batch_lambda_kernel<<<I.n_tens, 256, 0, s>>>(B->bt, I.tens, d);
    if (B->bf16) batch_scale_kernel<__nv_bfloat16><<<I.n_scale, ALS_THREADS, 0, s>>>(B->bt, I.scale, d);
    else batch_scale_kernel<float><<<I.n_scale, ALS_THREADS, 0, s>>>(B->bt, I.scale, d);
    SPM_TRY(batch_gram(B, d, s));
    if (I.n_fit > 0) batch_fit_kernel<<<I.n_fit, ALS_THREADS, 0, s>>>(B->bt, I.fit, d);
    SPM_CUDA_TRY(cudaGetLastError());
  }
  return SPM_OK;
}

spm_status spm_batch_status(spm_batch_t B, int* active, int* sweeps, void* stream) {
  if (!B || !active) return SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SPM_CUDA_TRY(cudaMemcpyAsync(B->host.data(), B->bt, sizeof(BatchTensor) * B->n,
                               cudaMemcpyDeviceToHost, s));
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  for (int t = 0; t < B->n; ++t) {
    active[t] = B->host[t].active;
    if (sweeps) sweeps[t] = B->host[t].sweeps;
  }
  return SPM_OK;
}

void spm_batch_destroy(spm_batch_t B) { free_batch(B); }

}  // extern "C"
