// diag.cu -- self-test of the bounded device-side wait, and the host-side
// allocation fault injection used by the failure-detection tests.
#include <atomic>

#include "plan.cuh"

namespace spm {
namespace {

// One mbarrier that nothing ever arrives on: the bounded wait gives up after
// `limit` polls and the block records a timeout, as the MTTKRP kernel's ring
// waits do when a copy never lands.
__global__ void wait_timeout_kernel(uint32_t limit, int* __restrict__ err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0u, limit);
  if (!ok && threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
  __syncthreads();
  if (threadIdx.x == 0) mbar_inval(&bar);
}

std::atomic<int> g_fail_alloc{-1};

}  // namespace

bool alloc_fault_due() {
  int k = g_fail_alloc.load();
  while (k >= 0) {
    if (g_fail_alloc.compare_exchange_weak(k, k - 1)) return k == 0;
  }
  return false;
}

}  // namespace spm

extern "C" {

spm_status spm_selftest_wait_timeout(uint32_t limit, void* stream) {
  if (limit == 0) return SPM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* d_err = nullptr;
  SPM_CUDA_TRY(cudaMallocAsync((void**)&d_err, sizeof(int), s));
  SPM_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  spm::wait_timeout_kernel<<<1, 64, 0, s>>>(limit, d_err);
  SPM_CUDA_TRY(cudaGetLastError());
  int h = 0;
  SPM_CUDA_TRY(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPM_CUDA_TRY(cudaFreeAsync(d_err, s));
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  return (h & spm::DEV_ERR_TIMEOUT) ? SPM_ERR_TIMEOUT : SPM_OK;
}

spm_status spm_selftest_mttkrp_timeout(spmttkrp_plan_t plan, int mode,
                                       const void* const* factors, float* out, void* stream) {
  if (!plan) return SPM_ERR_INVALID_ARG;
  // Every warp's first wait on a record copy gives up without polling; the
  // copies already issued still land (the drain waits for them), and the
  // blocks skip their merge and stores.
  plan->wait_limit = ~0u;
  const spm_status st = spm::run_mttkrp(plan, mode, factors, out, static_cast<cudaStream_t>(stream));
  plan->wait_limit = 0;
  if (st != SPM_OK) return st;
  return spmttkrp_plan_status(plan, stream);
}

void spm_inject_alloc_failure(int k) { spm::g_fail_alloc.store(k < 0 ? -1 : k); }

}  // extern "C"
