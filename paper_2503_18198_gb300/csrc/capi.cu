// capi.cu -- the extern "C" entry points declared in include/spmttkrp.h.
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>

#include "plan.cuh"

namespace spm {

spm_status plan_alloc(spmttkrp_plan_s* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (p->nallocs >= (int)(sizeof(p->allocs) / sizeof(p->allocs[0]))) return SPM_ERR_OOM;
  if (alloc_fault_due()) return SPM_ERR_OOM;  // injected by spm_inject_alloc_failure
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *ptr = nullptr;
    return e == cudaErrorMemoryAllocation ? SPM_ERR_OOM : SPM_ERR_CUDA;
  }
  p->alloc_bytes[p->nallocs] = bytes;
  p->allocs[p->nallocs++] = *ptr;
  p->bytes += bytes;
  return SPM_OK;
}

spm_status plan_realloc(spmttkrp_plan_s* p, void** ptr, size_t bytes) {
  int i = 0;
  while (i < p->nallocs && p->allocs[i] != *ptr) ++i;
  if (i == p->nallocs) return SPM_ERR_INVALID_ARG;
  if (bytes == 0) bytes = 16;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SPM_ERR_OOM : SPM_ERR_CUDA;
  }
  cudaFree(*ptr);
  p->bytes = p->bytes - p->alloc_bytes[i] + bytes;
  p->allocs[i] = q;
  p->alloc_bytes[i] = bytes;
  *ptr = q;
  return SPM_OK;
}

void plan_free(spmttkrp_plan_s* p, void** ptr) {
  int i = 0;
  while (i < p->nallocs && p->allocs[i] != *ptr) ++i;
  if (i == p->nallocs) return;
  cudaFree(*ptr);
  p->bytes -= p->alloc_bytes[i];
  for (int j = i + 1; j < p->nallocs; ++j) {
    p->allocs[j - 1] = p->allocs[j];
    p->alloc_bytes[j - 1] = p->alloc_bytes[j];
  }
  --p->nallocs;
  *ptr = nullptr;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return -1;
  }
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return -1;
  }
  return n;
}

int default_kappa() {
  const int n = sm_count();
  return n < 1 ? n : SPM_PARTITIONS_PER_SM * n;
}

namespace {

void free_plan(spmttkrp_plan_s* p) {
  if (!p) return;
  for (cudaEvent_t e : p->ev)
    if (e) cudaEventDestroy(e);
  if (p->copy_in) cudaStreamDestroy(p->copy_in);
  if (p->copy_out) cudaStreamDestroy(p->copy_out);
  if (p->als.ev_fork) cudaEventDestroy(p->als.ev_fork);
  if (p->als.ev_join) cudaEventDestroy(p->als.ev_join);
  if (p->als.side) cudaStreamDestroy(p->als.side);
  for (int i = 0; i < p->nallocs; ++i) cudaFree(p->allocs[i]);
  (void)cudaGetLastError();
  delete p;
}

// Lean copy: input position of each copy position = perm0[src[k]].
__global__ void lean_perm_kernel(const int32_t* __restrict__ perm0, const int32_t* __restrict__ src,
                                 int64_t n, int64_t* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = perm0[src[k]];
}

__global__ void perm_to_i64_kernel(const int32_t* __restrict__ in, int64_t n,
                                   int64_t* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = in[k];
}

}  // namespace
}  // namespace spm

using namespace spm;

extern "C" {

const char* spm_status_string(spm_status s) {
  switch (s) {
    case SPM_OK: return "ok";
    case SPM_ERR_INVALID_ARG: return "invalid argument";
    case SPM_ERR_INDEX_OUT_OF_RANGE: return "index out of range";
    case SPM_ERR_OOM: return "out of device memory";
    case SPM_ERR_CUDA: return "CUDA runtime error";
    case SPM_ERR_NUMERIC: return "numerical failure (system not positive definite or NaN)";
    case SPM_ERR_TIMEOUT: return "bounded device wait timed out";
    case SPM_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

int spm_device_sm_count(void) { return sm_count(); }

spm_status spmttkrp_plan(spmttkrp_plan_t* out, int nmodes, const int64_t* dims, int64_t nnz,
                         const int32_t* const* idx, const float* vals, int rank,
                         uint32_t flags, void* stream) {
  NvtxScope nv("spmttkrp_plan");
  if (!out) return SPM_ERR_INVALID_ARG;
  *out = nullptr;
  if (nmodes < 2 || nmodes > SPM_MAX_MODES || !dims || nnz < 0 ||
      nnz >= ((int64_t)1 << 31) - ((int64_t)1 << 20) || rank < 1 || rank > SPM_MAX_RANK)
    return SPM_ERR_INVALID_ARG;
  for (int w = 0; w < nmodes; ++w)
    if (dims[w] < 1 || dims[w] >= ((int64_t)1 << 31)) return SPM_ERR_INVALID_ARG;
  if (nnz > 0) {
    if (!idx || !vals) return SPM_ERR_INVALID_ARG;
    for (int w = 0; w < nmodes; ++w)
      if (!idx[w]) return SPM_ERR_INVALID_ARG;
  }
  const uint32_t known =
      SPM_FACTOR_MASK | SPM_POLICY_MASK | SPM_PLAN_LEAN | SPM_PLAN_FIBRE | (0xFFFFu << 16);
  if (flags & ~known) return SPM_ERR_INVALID_ARG;
  const int policy = (int)((flags & SPM_POLICY_MASK) >> 4);
  if (policy > 3) return SPM_ERR_INVALID_ARG;
  const bool lean = (flags & SPM_PLAN_LEAN) != 0;
  const bool fibre = (flags & SPM_PLAN_FIBRE) != 0;
  // the fibre layout: three modes, unit-per-slot kernel ranks, copies in the
  // P1 order (Scheme 1 reorders them), one record layout at a time
  if (fibre && (nmodes != 3 || fibre_slots(rank) == 0 || lean ||
                (policy != (int)(SPM_POLICY_BALANCED >> 4) &&
                 policy != (int)(SPM_POLICY_SCHEME2 >> 4))))
    return SPM_ERR_UNSUPPORTED;
  // a lean plan keeps every copy in the P1 order (Scheme 1 reorders copies)
  if (lean && policy != (int)(SPM_POLICY_BALANCED >> 4) && policy != (int)(SPM_POLICY_SCHEME2 >> 4))
    return SPM_ERR_UNSUPPORTED;
  if (lean && nmodes > 5) return SPM_ERR_UNSUPPORTED;
  int kappa = (int)SPM_KAPPA_OF(flags);
  if (kappa == 0) kappa = default_kappa();
  if (kappa < 1) return SPM_ERR_CUDA;

  spmttkrp_plan_s* p = new (std::nothrow) spmttkrp_plan_s();
  if (!p) return SPM_ERR_OOM;
  cudaGetDevice(&p->device);
  p->N = nmodes;
  p->R = rank;
  for (int w = 0; w < nmodes; ++w) p->dims[w] = dims[w];
  p->nnz = nnz;
  p->flags = flags;
  p->bf16 = (flags & SPM_FACTOR_MASK) == SPM_FACTOR_BF16;
  p->lean = lean;
  p->fibre = fibre;
  p->kappa = kappa;
  p->kappa_cap = kappa;
  // a fibre plan's warps take fibre_slots(R) units side by side, all 32 warps
  // of a block once each
  p->nu = fibre ? 32 * fibre_slots(rank) : SPM_UNITS_PER_PARTITION(rank);
  p->policy = policy;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  spm_status st = plan_alloc(p, (void**)&p->dev_err, sizeof(int));
  if (st == SPM_OK) st = plan_alloc(p, (void**)&p->normX2, sizeof(double));
  if (st == SPM_OK) st = plan_alloc(p, (void**)&p->cta_part, sizeof(float) * 2 * (size_t)kappa * rank);
  if (st == SPM_OK) st = plan_alloc(p, (void**)&p->cta_meta, sizeof(int) * 4 * (size_t)kappa);
  if (st == SPM_OK && cudaMemsetAsync(p->dev_err, 0, sizeof(int), s) != cudaSuccess) st = SPM_ERR_CUDA;
  if (st == SPM_OK) st = build_copies(p, idx, vals, s);
  if (st != SPM_OK) {
    cudaStreamSynchronize(s);
    (void)cudaGetLastError();
    free_plan(p);
    return st;
  }
  *out = p;
  return SPM_OK;
}

spm_status spmttkrp_plan_bytes(spmttkrp_plan_t plan, size_t* bytes) {
  if (!plan || !bytes) return SPM_ERR_INVALID_ARG;
  *bytes = plan->bytes;
  return SPM_OK;
}

spm_status spmttkrp_plan_permutation(spmttkrp_plan_t plan, int mode, int64_t* perm,
                                     void* stream) {
  if (!plan || mode < 0 || mode >= plan->N || (!perm && plan->nnz > 0)) return SPM_ERR_INVALID_ARG;
  if (plan->nnz == 0) return SPM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = plan->nnz;
  const int blocks = (int)std::min<int64_t>(ceil_div<int64_t>(n, 256), 152 * 16);
  if (plan->mode[mode].src)
    lean_perm_kernel<<<blocks, 256, 0, s>>>(plan->mode[0].perm, plan->mode[mode].src, n, perm);
  else
    perm_to_i64_kernel<<<blocks, 256, 0, s>>>(plan->mode[mode].perm, n, perm);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

spm_status spmttkrp_plan_partition(spmttkrp_plan_t plan, int mode, int64_t* off, int* kappa_out,
                                   void* stream) {
  if (!plan || mode < 0 || mode >= plan->N || !off) return SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SPM_CUDA_TRY(cudaMemcpyAsync(off, plan->mode[mode].off, sizeof(int64_t) * (plan->kappa + 1),
                               cudaMemcpyDeviceToDevice, s));
  if (kappa_out) *kappa_out = plan->kappa;
  return SPM_OK;
}

spm_status spmttkrp_plan_work_units(spmttkrp_plan_t plan, int mode, int64_t* off, void* stream) {
  if (!plan || mode < 0 || mode >= plan->N || !off) return SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SPM_CUDA_TRY(cudaMemcpyAsync(off, plan->mode[mode].woff,
                               sizeof(int64_t) * ((size_t)plan->kappa * plan->nu + 1),
                               cudaMemcpyDeviceToDevice, s));
  return SPM_OK;
}

spm_status spmttkrp_plan_scheme(spmttkrp_plan_t plan, int mode, int* scheme) {
  if (!plan || mode < 0 || mode >= plan->N || !scheme) return SPM_ERR_INVALID_ARG;
  *scheme = plan->mode[mode].scheme;
  return SPM_OK;
}

spm_status spmttkrp_plan_bytes_estimate(int nmodes, const int64_t* dims, int64_t nnz, int rank,
                                        uint32_t flags, size_t* resident, size_t* transient) {
  if (nmodes < 2 || nmodes > SPM_MAX_MODES || !dims || nnz < 0 || rank < 1 ||
      rank > SPM_MAX_RANK || !resident)
    return SPM_ERR_INVALID_ARG;
  int kappa = (int)SPM_KAPPA_OF(flags);
  if (kappa == 0) kappa = default_kappa();
  if (kappa < 1) return SPM_ERR_CUDA;  // SPM_KAPPA(0) needs a device to count its SMs
  const bool fibre = (flags & SPM_PLAN_FIBRE) != 0;
  if (fibre && (nmodes != 3 || fibre_slots(rank) == 0)) return SPM_ERR_UNSUPPORTED;
  size_t tr = 0;
  plan_bytes_estimate(nmodes, dims, nnz, rank, kappa, true, (flags & SPM_PLAN_LEAN) != 0, resident,
                      &tr, fibre, (int)((flags & SPM_POLICY_MASK) >> 4));
  if (transient) *transient = tr;
  return SPM_OK;
}

spm_status spmttkrp_plan_fibre_count(spmttkrp_plan_t plan, int mode, int64_t* nfib) {
  if (!plan || !nfib || mode < 0 || mode >= plan->N) return SPM_ERR_INVALID_ARG;
  if (!plan->fibre) return SPM_ERR_UNSUPPORTED;
  *nfib = plan->mode[mode].nfib;
  return SPM_OK;
}

spm_status spmttkrp_plan_repartition(spmttkrp_plan_t plan, int kappa, void* stream) {
  if (!plan) return SPM_ERR_INVALID_ARG;
  if (kappa == 0) kappa = default_kappa();
  return plan_repartition(plan, kappa, static_cast<cudaStream_t>(stream));
}

spm_status spmttkrp_plan_autotune(spmttkrp_plan_t plan, const void* const* factors,
                                  const int* kappas, int nkappas, int reps, int* chosen,
                                  float* ms, void* stream) {
  if (!plan || !factors || reps < 1 || (kappas && nkappas < 1) || !chosen) return SPM_ERR_INVALID_ARG;
  if (plan->fibre ||
      (plan->policy != (int)(SPM_POLICY_BALANCED >> 4) && plan->policy != (int)(SPM_POLICY_SCHEME2 >> 4)))
    return SPM_ERR_UNSUPPORTED;
  const int sms = sm_count();
  if (sms < 1) return SPM_ERR_CUDA;
  const int dflt[2] = {sms, 2 * sms};
  if (!kappas) {
    kappas = dflt;
    nkappas = 2;
  }
  for (int c = 0; c < nkappas; ++c)
    if (kappas[c] < 1 || kappas[c] > 0xFFFF) return SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SPM_TRY(ensure_als_state(plan));  // its M buffer (I_max x R) takes the outputs
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    (void)cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return SPM_ERR_CUDA;
  }
  spm_status st = SPM_OK;
  int best = -1;
  float best_ms = 0.f;
  for (int c = 0; c < nkappas && st == SPM_OK; ++c) {
    st = plan_repartition(plan, kappas[c], s);
    float t_min = 0.f;
    for (int r = 0; r <= reps && st == SPM_OK; ++r) {  // r == 0 warms up
      cudaEventRecord(e0, s);
      for (int d = 0; d < plan->N && st == SPM_OK; ++d)
        st = run_mttkrp(plan, d, factors, plan->als.M, s);
      cudaEventRecord(e1, s);
      if (st == SPM_OK && cudaEventSynchronize(e1) != cudaSuccess) st = SPM_ERR_CUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r == 1 || (r > 1 && t < t_min)) t_min = t;
    }
    if (st != SPM_OK) break;
    if (ms) ms[c] = t_min;
    if (best < 0 || t_min < best_ms) {
      best = c;
      best_ms = t_min;
    }
  }
  if (st == SPM_OK) {
    st = plan_repartition(plan, kappas[best], s);
    *chosen = kappas[best];
  }
  if (st == SPM_OK && cudaStreamSynchronize(s) != cudaSuccess) st = SPM_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  (void)cudaGetLastError();
  return st;
}

void spmttkrp_plan_destroy(spmttkrp_plan_t plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  free_plan(plan);
}

spm_status spmttkrp_run(spmttkrp_plan_t plan, int mode, const void* const* factors, float* out,
                        void* stream) {
  NvtxScope nv("spmttkrp_run");
  if (!plan) return SPM_ERR_INVALID_ARG;
  return run_mttkrp(plan, mode, factors, out, static_cast<cudaStream_t>(stream));
}

spm_status cpd_als_step(spmttkrp_plan_t plan, void* const* factors, double* lambda, double* fit,
                        void* stream) {
  NvtxScope nv("cpd_als_step");
  if (!plan || !factors || !lambda) return SPM_ERR_INVALID_ARG;
  return als_sweep(plan, factors, lambda, fit, static_cast<cudaStream_t>(stream));
}

spm_status cpd_als_reset(spmttkrp_plan_t plan) {
  if (!plan) return SPM_ERR_INVALID_ARG;
  plan->als.ready = false;
  return SPM_OK;
}

spm_status spmttkrp_run_all_host(spmttkrp_plan_t p, const void* const* host_factors,
                                 float* const* host_out, void* stream) {
  NvtxScope nv("spmttkrp_run_all_host");
  if (!p || !host_factors || !host_out) return SPM_ERR_INVALID_ARG;
  const int N = p->N, R = p->R;
  for (int w = 0; w < N; ++w)
    if (!host_factors[w] || !host_out[w]) return SPM_ERR_INVALID_ARG;
  const size_t sf = p->bf16 ? 2 : 4;
  if (!p->h_fac[0]) {  // first call: staging buffers, side streams, events
    for (int w = 0; w < N; ++w) {
      SPM_TRY(plan_alloc(p, &p->h_fac[w], sf * (size_t)p->dims[w] * R));
      SPM_TRY(plan_alloc(p, (void**)&p->h_out[w], sizeof(float) * (size_t)p->dims[w] * R));
    }
    SPM_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_in, cudaStreamNonBlocking));
    SPM_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_out, cudaStreamNonBlocking));
    for (cudaEvent_t& e : p->ev) SPM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t* ev_in = p->ev;                   // [N] factor w on the device
  cudaEvent_t* ev_done = p->ev + SPM_MAX_MODES;  // [N] output d computed
  cudaEvent_t ev_start = p->ev[2 * SPM_MAX_MODES];
  cudaEvent_t ev_outs = p->ev[2 * SPM_MAX_MODES + 1];
  // copies start after the caller's earlier work on `stream`
  SPM_CUDA_TRY(cudaEventRecord(ev_start, s));
  SPM_CUDA_TRY(cudaStreamWaitEvent(p->copy_in, ev_start, 0));
  SPM_CUDA_TRY(cudaStreamWaitEvent(p->copy_out, ev_start, 0));
  // factors 1..N-1 first (mode 0 needs exactly those), factor 0 last
  for (int k = 1; k <= N; ++k) {
    const int w = k % N;
    SPM_CUDA_TRY(cudaMemcpyAsync(p->h_fac[w], host_factors[w], sf * (size_t)p->dims[w] * R,
                                 cudaMemcpyHostToDevice, p->copy_in));
    SPM_CUDA_TRY(cudaEventRecord(ev_in[w], p->copy_in));
  }
  for (int d = 0; d < N; ++d) {
    for (int w = 0; w < N; ++w)
      if (w != d) SPM_CUDA_TRY(cudaStreamWaitEvent(s, ev_in[w], 0));
    SPM_TRY(run_mttkrp(p, d, p->h_fac, p->h_out[d], s));
    SPM_CUDA_TRY(cudaEventRecord(ev_done[d], s));
    // output d goes back while mode d + 1 computes
    SPM_CUDA_TRY(cudaStreamWaitEvent(p->copy_out, ev_done[d], 0));
    SPM_CUDA_TRY(cudaMemcpyAsync(host_out[d], p->h_out[d], sizeof(float) * (size_t)p->dims[d] * R,
                                 cudaMemcpyDeviceToHost, p->copy_out));
  }
  // work queued on `stream` after this call sees every copy done
  SPM_CUDA_TRY(cudaEventRecord(ev_outs, p->copy_out));
  SPM_CUDA_TRY(cudaStreamWaitEvent(s, ev_outs, 0));
  return SPM_OK;
}

spm_status spmttkrp_plan_status(spmttkrp_plan_t plan, void* stream) {
  if (!plan) return SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h = 0;
  SPM_CUDA_TRY(cudaMemcpyAsync(&h, plan->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  SPM_CUDA_TRY(cudaMemsetAsync(plan->dev_err, 0, sizeof(int), s));
  if (h & DEV_ERR_NUMERIC) return SPM_ERR_NUMERIC;
  if (h & DEV_ERR_TIMEOUT) return SPM_ERR_TIMEOUT;
  return SPM_OK;
}

}  // extern "C"
