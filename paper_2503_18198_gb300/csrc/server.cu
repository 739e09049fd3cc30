// server.cu -- continuous batching of CP-ALS jobs on one GPU.
//
// Jobs (a COO tensor, a rank, initial factors, a stopping rule) are queued by
// spm_server_submit and served by spm_server_step, which the caller runs in
// a loop:
//   1. one batched sweep (batch.cu) of every running job is launched on the
//      sweep stream;
//   2. while it runs, queued jobs are admitted in arrival order as long as
//      the running-job limit and the device-memory budget allow: the plan
//      (mode copies, partitions) is built and the factors are set up on the
//      build stream, so plan building overlaps the sweep;
//   3. after the sweep, jobs whose fit changed by less than their tolerance
//      (or that reached their sweep limit) leave the batch, their plans are
//      freed and their results wait for spm_server_result; admitted jobs join
//      the batch for the next sweep.
// A job's arithmetic is that of cpd_als_step on its own plan (same partition
// count, same summation order), so its result does not depend on which other
// jobs shared its sweeps.
#include <algorithm>
#include <chrono>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "batch.cuh"

namespace spm {
namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

__global__ void cast_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                                 int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

struct Job {
  int64_t id = 0;
  int state = SPM_JOB_QUEUED;
  spm_status status = SPM_OK;
  int N = 0, R = 0;
  int64_t dims[SPM_MAX_MODES] = {};
  int64_t nnz = 0;
  const int32_t* idx[SPM_MAX_MODES] = {};
  const float* vals = nullptr;
  const float* init[SPM_MAX_MODES] = {};
  double tol = 0.0;
  int max_sweeps = 1;
  uint32_t plan_flags = 0;
  size_t resident = 0, transient = 0;  // estimate
  size_t held = 0;                     // bytes charged to the budget
  spmttkrp_plan_s* plan = nullptr;
  void* fac[SPM_MAX_MODES] = {};
  double* lamfit = nullptr;  // [R] weights, then the fit
  int sweeps = 0;
  double fit = 0.0;
  int start_sweeps = 0;          // > 0 for a job resumed from a snapshot
  double start_prev_fit = -1.0e300;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

}  // namespace
}  // namespace spm

struct spm_server_s {
  size_t budget = 0;
  size_t used = 0;
  int max_active = 0;
  uint32_t flags = 0;   // factor type
  int64_t nnz_per_partition = 0;
  cudaStream_t s_sweep = nullptr;
  cudaStream_t s_build = nullptr;
  spm_batch_s* B = nullptr;
  std::deque<spm::Job*> queue;
  std::vector<spm::Job*> running;  // same order as the batch members
  std::unordered_map<int64_t, spm::Job*> jobs;
  int64_t next_id = 1;
};

namespace spm {
namespace {

void release_plan(spm_server_s* S, Job* j) {
  if (j->plan) {
    S->used -= std::min(S->used, j->plan->bytes);
    j->held -= std::min(j->held, j->plan->bytes);
    spmttkrp_plan_destroy(j->plan);
    j->plan = nullptr;
  }
}

void release_all(spm_server_s* S, Job* j) {
  release_plan(S, j);
  for (int w = 0; w < SPM_MAX_MODES; ++w)
    if (j->fac[w]) {
      cudaFree(j->fac[w]);
      j->fac[w] = nullptr;
    }
  if (j->lamfit) {
    cudaFree(j->lamfit);
    j->lamfit = nullptr;
  }
  S->used -= std::min(S->used, j->held);
  j->held = 0;
}

size_t factor_bytes(const spm_server_s* S, const Job* j) {
  const size_t sf = (S->flags & SPM_FACTOR_MASK) == SPM_FACTOR_BF16 ? 2 : 4;
  size_t b = sizeof(double) * (j->R + 1);
  for (int w = 0; w < j->N; ++w) b += sf * (size_t)j->dims[w] * j->R;
  return b;
}

// Build the plan and the factors of j on the build stream.
spm_status admit(spm_server_s* S, Job* j) {
  cudaStream_t s = S->s_build;
  spmttkrp_plan_t p = nullptr;
  SPM_TRY(spmttkrp_plan(&p, j->N, j->dims, j->nnz, j->idx, j->vals, j->R, j->plan_flags, s));
  j->plan = p;
  S->used += p->bytes;
  j->held += p->bytes;
  const bool bf16 = (S->flags & SPM_FACTOR_MASK) == SPM_FACTOR_BF16;
  for (int w = 0; w < j->N; ++w) {
    const int64_t n = j->dims[w] * j->R;
    const size_t bytes = (bf16 ? 2 : 4) * (size_t)n;
    if (cudaMalloc(&j->fac[w], bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      return SPM_ERR_OOM;
    }
    S->used += bytes;
    j->held += bytes;
    if (bf16)
      cast_bf16_kernel<<<(int)std::min<int64_t>(ceil_div<int64_t>(n, 256), 4096), 256, 0, s>>>(
          j->init[w], static_cast<__nv_bfloat16*>(j->fac[w]), n);
    else
      SPM_CUDA_TRY(cudaMemcpyAsync(j->fac[w], j->init[w], bytes, cudaMemcpyDeviceToDevice, s));
  }
  if (cudaMalloc((void**)&j->lamfit, sizeof(double) * (j->R + 1)) != cudaSuccess) {
    (void)cudaGetLastError();
    return SPM_ERR_OOM;
  }
  S->used += sizeof(double) * (j->R + 1);
  j->held += sizeof(double) * (j->R + 1);
  SPM_CUDA_TRY(cudaGetLastError());
  // the caller's inputs are no longer needed once these copies are done
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  return SPM_OK;
}

void fail(spm_server_s* S, Job* j, spm_status st) {
  j->state = SPM_JOB_FAILED;
  j->status = st;
  j->t_done = now_ms();
  release_all(S, j);
}

}  // namespace
}  // namespace spm

using namespace spm;

extern "C" {

spm_status spm_server_create(spm_server_t* out, size_t hbm_budget, int max_active, uint32_t flags,
                             int64_t nnz_per_partition) {
  if (!out) return SPM_ERR_INVALID_ARG;
  *out = nullptr;
  if (hbm_budget == 0 || max_active < 1 || nnz_per_partition < 0 ||
      (flags & ~SPM_FACTOR_MASK) != 0)
    return SPM_ERR_INVALID_ARG;
  spm_server_s* S = new (std::nothrow) spm_server_s();
  if (!S) return SPM_ERR_OOM;
  S->budget = hbm_budget;
  S->max_active = max_active;
  S->flags = flags;
  S->nnz_per_partition = nnz_per_partition;
  S->B = new (std::nothrow) spm_batch_s();
  if (!S->B || cudaStreamCreateWithFlags(&S->s_sweep, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->s_build, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    spm_server_destroy(S);
    return SPM_ERR_CUDA;
  }
  cudaGetDevice(&S->B->device);
  *out = S;
  return SPM_OK;
}

spm_status spm_server_submit(spm_server_t S, const spm_job_desc* d, int64_t* job) {
  if (!S || !d || !job) return SPM_ERR_INVALID_ARG;
  const int N = d->nmodes;
  if (N < 2 || N > SPM_MAX_MODES || !d->dims || d->nnz < 0 || !d->init || d->max_sweeps < 1 ||
      !(d->tol >= 0.0))
    return SPM_ERR_INVALID_ARG;
  if (batch_kclass(N, d->rank) == KC_NONE) return SPM_ERR_UNSUPPORTED;
  if (d->nnz > 0 && (!d->idx || !d->vals)) return SPM_ERR_INVALID_ARG;
  Job* j = new (std::nothrow) Job();
  if (!j) return SPM_ERR_OOM;
  j->id = S->next_id++;
  j->N = N;
  j->R = d->rank;
  j->nnz = d->nnz;
  j->vals = d->vals;
  for (int w = 0; w < N; ++w) {
    j->dims[w] = d->dims[w];
    j->idx[w] = d->nnz > 0 ? d->idx[w] : nullptr;
    j->init[w] = d->init[w];
    if (d->dims[w] < 1 || d->dims[w] >= ((int64_t)1 << 31) || !d->init[w] ||
        (reinterpret_cast<uintptr_t>(d->init[w]) & 15u)) {
      delete j;
      return SPM_ERR_INVALID_ARG;
    }
  }
  j->tol = d->tol;
  j->max_sweeps = d->max_sweeps;
  int kappa = default_kappa();
  if (S->nnz_per_partition > 0)
    kappa = (int)std::max<int64_t>(
        1, std::min<int64_t>(0xFFFF, ceil_div<int64_t>(std::max<int64_t>(1, d->nnz),
                                                       S->nnz_per_partition)));
  j->plan_flags = (S->flags & SPM_FACTOR_MASK) | SPM_KAPPA(kappa);
  plan_bytes_estimate(N, j->dims, j->nnz, j->R, kappa, true, false, &j->resident, &j->transient);
  j->t_submit = now_ms();
  S->queue.push_back(j);
  S->jobs[j->id] = j;
  *job = j->id;
  return SPM_OK;
}

spm_status spm_server_step(spm_server_t S, int* running, int* queued) {
  NvtxScope nv("spm_server_step");
  if (!S) return SPM_ERR_INVALID_ARG;
  spm_batch_s* B = S->B;
  // 1. one sweep of every running job (asynchronous)
  spm_status sweep_st = SPM_OK;
  if (!S->running.empty()) sweep_st = batch_sweep(B, S->s_sweep);
  // 2. admission, overlapping the sweep
  std::vector<Job*> admitted;
  while (!S->queue.empty() &&
         (int)(S->running.size() + admitted.size()) < S->max_active) {
    // once the sweep is over, further builds would only keep it waiting:
    // the rest join at a later step
    if (!admitted.empty() && !S->running.empty() && cudaStreamQuery(S->s_sweep) == cudaSuccess)
      break;
    Job* j = S->queue.front();
    const size_t need = j->resident + factor_bytes(S, j);
    if (need + j->transient > S->budget) {  // can never fit
      S->queue.pop_front();
      fail(S, j, SPM_ERR_OOM);
      continue;
    }
    if (S->used + need + j->transient > S->budget) break;  // wait for memory
    S->queue.pop_front();
    j->t_admit = now_ms();
    const spm_status st = admit(S, j);
    if (st != SPM_OK) {
      fail(S, j, st);
      continue;
    }
    admitted.push_back(j);
  }
  // 3. retire finished jobs
  SPM_CUDA_TRY(cudaStreamSynchronize(S->s_sweep));
  SPM_TRY(sweep_st);
  if (!S->running.empty()) SPM_TRY(batch_pull(B, S->s_sweep));
  for (int t = (int)S->running.size() - 1; t >= 0; --t) {
    Job* j = S->running[t];
    const BatchTensor& b = B->host[t];
    int err = 0;
    SPM_CUDA_TRY(cudaMemcpy(&err, j->plan->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!err && b.active) continue;
    j->sweeps = b.sweeps;
    SPM_CUDA_TRY(cudaMemcpy(&j->fit, j->lamfit + j->R, sizeof(double), cudaMemcpyDeviceToHost));
    batch_remove(B, t);
    S->running.erase(S->running.begin() + t);
    if (err) {
      fail(S, j, (err & DEV_ERR_NUMERIC) ? SPM_ERR_NUMERIC
                 : (err & DEV_ERR_TIMEOUT) ? SPM_ERR_TIMEOUT : SPM_ERR_CUDA);
      continue;
    }
    j->state = SPM_JOB_DONE;
    j->t_done = now_ms();
    release_plan(S, j);  // the results stay until spm_server_result
  }
  // 4. admitted jobs join the batch
  for (Job* j : admitted) {
    const spm_status st = batch_add(B, j->plan, j->fac, j->lamfit, j->lamfit + j->R, j->tol,
                                    j->max_sweeps, S->s_sweep, j->start_sweeps, j->start_prev_fit);
    if (st != SPM_OK) {
      fail(S, j, st);
      continue;
    }
    j->state = SPM_JOB_RUNNING;
    S->running.push_back(j);
  }
  if (running) *running = (int)S->running.size();
  if (queued) *queued = (int)S->queue.size();
  return SPM_OK;
}

spm_status spm_server_resume(spm_server_t S, const spm_job_desc* d, int sweeps_done,
                             double prev_fit, int64_t* job) {
  if (!S || !d || sweeps_done < 0 || sweeps_done >= d->max_sweeps) return SPM_ERR_INVALID_ARG;
  SPM_TRY(spm_server_submit(S, d, job));
  Job* j = S->jobs[*job];
  j->start_sweeps = sweeps_done;
  j->start_prev_fit = prev_fit;
  return SPM_OK;
}

spm_status spm_server_snapshot(spm_server_t S, int64_t job, void* const* factors, double* lambda,
                               int* sweeps, double* prev_fit, void* stream) {
  if (!S || !sweeps || !prev_fit) return SPM_ERR_INVALID_ARG;
  auto it = S->jobs.find(job);
  if (it == S->jobs.end() || it->second->state != SPM_JOB_RUNNING) return SPM_ERR_INVALID_ARG;
  Job* j = it->second;
  int t = 0;
  while (t < (int)S->running.size() && S->running[t] != j) ++t;
  if (t == (int)S->running.size()) return SPM_ERR_INVALID_ARG;
  // the host descriptors are current between steps (pulled after each sweep)
  const BatchTensor& b = S->B->host[t];
  *sweeps = b.sweeps;
  *prev_fit = b.prev_fit;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t sf = (S->flags & SPM_FACTOR_MASK) == SPM_FACTOR_BF16 ? 2 : 4;
  if (factors)
    for (int w = 0; w < j->N; ++w)
      if (factors[w])
        SPM_CUDA_TRY(cudaMemcpyAsync(factors[w], j->fac[w], sf * (size_t)j->dims[w] * j->R,
                                     cudaMemcpyDeviceToDevice, s));
  if (lambda)
    SPM_CUDA_TRY(cudaMemcpyAsync(lambda, j->lamfit, sizeof(double) * j->R,
                                 cudaMemcpyDeviceToDevice, s));
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  return SPM_OK;
}

spm_status spm_server_job(spm_server_t S, int64_t job, spm_job_info* info) {
  if (!S || !info) return SPM_ERR_INVALID_ARG;
  auto it = S->jobs.find(job);
  if (it == S->jobs.end()) return SPM_ERR_INVALID_ARG;
  const Job* j = it->second;
  info->state = j->state;
  info->status = j->status;
  info->sweeps = j->sweeps;
  info->fit = j->fit;
  info->bytes = j->held;
  info->est_bytes = j->resident + factor_bytes(S, j);
  const bool admitted = j->t_admit > 0.0;
  const bool finished = j->state == SPM_JOB_DONE || j->state == SPM_JOB_FAILED;
  info->queued_ms = admitted ? j->t_admit - j->t_submit : 0.0;
  info->total_ms = finished ? j->t_done - j->t_submit : 0.0;
  return SPM_OK;
}

spm_status spm_server_result(spm_server_t S, int64_t job, void* const* factors, double* lambda,
                             void* stream) {
  if (!S) return SPM_ERR_INVALID_ARG;
  auto it = S->jobs.find(job);
  if (it == S->jobs.end()) return SPM_ERR_INVALID_ARG;
  Job* j = it->second;
  if (j->state != SPM_JOB_DONE) return j->state == SPM_JOB_FAILED ? j->status : SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t sf = (S->flags & SPM_FACTOR_MASK) == SPM_FACTOR_BF16 ? 2 : 4;
  if (factors)
    for (int w = 0; w < j->N; ++w)
      if (factors[w])
        SPM_CUDA_TRY(cudaMemcpyAsync(factors[w], j->fac[w], sf * (size_t)j->dims[w] * j->R,
                                     cudaMemcpyDeviceToDevice, s));
  if (lambda)
    SPM_CUDA_TRY(cudaMemcpyAsync(lambda, j->lamfit, sizeof(double) * j->R,
                                 cudaMemcpyDeviceToDevice, s));
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  release_all(S, j);
  S->jobs.erase(it);
  delete j;
  return SPM_OK;
}

spm_status spm_server_usage(spm_server_t S, size_t* used, size_t* budget) {
  if (!S) return SPM_ERR_INVALID_ARG;
  if (used) *used = S->used;
  if (budget) *budget = S->budget;
  return SPM_OK;
}

void spm_server_destroy(spm_server_t S) {
  if (!S) return;
  if (S->s_sweep) cudaStreamSynchronize(S->s_sweep);
  if (S->s_build) cudaStreamSynchronize(S->s_build);
  for (auto& kv : S->jobs) {
    release_all(S, kv.second);
    delete kv.second;
  }
  if (S->B) batch_free(S->B);
  if (S->s_sweep) cudaStreamDestroy(S->s_sweep);
  if (S->s_build) cudaStreamDestroy(S->s_build);
  (void)cudaGetLastError();
  delete S;
}

}  // extern "C"
