// noalloc.cu -- spMTTKRP along one mode with no device allocation at all.
//
// For callers that cannot allocate device memory while they work: a serving
// loop that runs inside a memory pool sized once at start-up, code that runs
// where a cudaMalloc would synchronise the device or is simply not allowed,
// or an embedding that hands the library only its inputs and outputs.  The
// one scratch buffer the MTTKRP launch sequence needs (work-unit offsets and
// the per-partition boundary partials) lives in a file-scope __device__
// array of fixed size, which every GPU that loads this library holds until
// the process exits.
#include <mutex>

#include "mttkrp_kernel.cuh"

namespace spm {

using MttkrpKernelFn = void (*)(const MttkrpArgs);
MttkrpKernelFn pick_mttkrp(bool bf16, int nin, int R);
spm_status launch_mttkrp_fixup(const float* cta_part, const int* cta_meta, int kappa, int R,
                               float* out, cudaStream_t s);

namespace {

// The shared scratch: [error word][work-unit offsets][boundary partials]
// [partition meta].
static __device__ __align__(256) unsigned char g_noalloc_scratch[SPM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once
// per device; in host code the symbol itself is only a host-side handle).
spm_status scratch_address(unsigned char** out) {
  int dev = 0;
  SPM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return SPM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      (void)cudaGetLastError();
      return SPM_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return SPM_OK;
}

// Work unit j of P starts at floor(j * nnz / P) (equal nonzero counts).
__global__ void equal_units_kernel(int64_t nnz, int64_t P, int64_t* __restrict__ woff) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= P;
       j += (int64_t)gridDim.x * blockDim.x)
    woff[j] = (j * nnz) / P;
}

struct RecordCheck {
  int32_t lim[SPM_MAX_MODES];  // dims in record word order (output mode first)
  int nwords;                  // index words per record (N)
  int ri;                      // 16-byte words per record
};

// The caller's records before the MTTKRP reads them: every index inside its
// mode's range (else DEV_ERR_INDEX) and output-mode indices non-decreasing
// (else DEV_ERR_ORDER).  The MTTKRP blocks read the flags first and store
// nothing when one is set, so bad records cannot send a gather or a store
// outside the caller's buffers.
__global__ void check_records_kernel(const int4* __restrict__ rec, int64_t nnz, RecordCheck c,
                                     int* __restrict__ err) {
  int bad = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int* w = reinterpret_cast<const int*>(rec + k * c.ri);
    for (int j = 0; j < c.nwords; ++j) {
      const int v = __ldg(w + j);
      if (v < 0 || v >= c.lim[j]) bad |= DEV_ERR_INDEX;
    }
    if (k > 0 && __ldg(reinterpret_cast<const int*>(rec + (k - 1) * c.ri)) > __ldg(w))
      bad |= DEV_ERR_ORDER;
  }
  bad = __reduce_or_sync(SPM_FULL_MASK, bad);
  if (bad && (threadIdx.x & 31) == 0) atomicOr(err, bad);
}

}  // namespace
}  // namespace spm

using namespace spm;

extern "C" spm_status spmttkrp_run_noalloc(int nmodes, const int64_t* dims, int64_t nnz, int mode,
                                           int rank, const void* records,
                                           const void* const* factors, uint32_t flags,
                                           float* out, void* stream) {
  if (nmodes < 2 || nmodes > SPM_MAX_MODES || !dims || nnz < 0 || mode < 0 || mode >= nmodes ||
      rank < 1 || rank > SPM_MAX_RANK || !factors || !out)
    return SPM_ERR_INVALID_ARG;
  if (nnz > 0 && !records) return SPM_ERR_INVALID_ARG;
  for (int w = 0; w < nmodes; ++w)
    if (dims[w] < 1 || dims[w] >= ((int64_t)1 << 31)) return SPM_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)(SPM_FACTOR_MASK | (0xFFFFu << 16))) return SPM_ERR_INVALID_ARG;
  const bool bf16 = (flags & SPM_FACTOR_MASK) == SPM_FACTOR_BF16;
  for (int w = 0; w < nmodes; ++w)
    if (w != mode && (!factors[w] || (reinterpret_cast<uintptr_t>(factors[w]) & 15u)))
      return SPM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(out) & 15u) ||
      (records && (reinterpret_cast<uintptr_t>(records) & 15u)))
    return SPM_ERR_INVALID_ARG;
  int kappa = (int)SPM_KAPPA_OF(flags);
  if (kappa == 0) kappa = default_kappa();
  if (kappa < 1) return SPM_ERR_CUDA;
  const int nu = SPM_UNITS_PER_PARTITION(rank);
  const int64_t P = (int64_t)kappa * nu;

  // scratch layout and size check (nothing here is allocated)
  const size_t woff_bytes = ((size_t)(P + 1) * sizeof(int64_t) + 255) & ~(size_t)255;
  const size_t part_bytes = ((size_t)kappa * 2 * rank * sizeof(float) + 255) & ~(size_t)255;
  const size_t meta_bytes = ((size_t)kappa * 4 * sizeof(int) + 255) & ~(size_t)255;
  if (woff_bytes + part_bytes + meta_bytes + 256 > (size_t)SPM_NOALLOC_SCRATCH_BYTES)
    return SPM_ERR_UNSUPPORTED;
  unsigned char* scratch = nullptr;
  SPM_TRY(scratch_address(&scratch));
  // layout: [error word, 256 bytes][work-unit offsets][boundary partials][meta]
  int* err = reinterpret_cast<int*>(scratch);
  int64_t* woff = reinterpret_cast<int64_t*>(scratch + 256);
  float* cta_part = reinterpret_cast<float*>(scratch + 256 + woff_bytes);
  int* cta_meta = reinterpret_cast<int*>(scratch + 256 + woff_bytes + part_bytes);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t out_bytes = sizeof(float) * (size_t)dims[mode] * (size_t)rank;
  // the error word starts clear for every call (spmttkrp_noalloc_status
  // reports the latest call's); every other scratch byte the kernels read is
  // written first by this call
  SPM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  // rows without nonzeros must read zero; every other row is overwritten
  SPM_CUDA_TRY(cudaMemsetAsync(out, 0, out_bytes, s));
  if (nnz == 0) return SPM_OK;
  {
    RecordCheck chk{};
    chk.lim[0] = (int32_t)dims[mode];
    int j = 1;
    for (int w = 0; w < nmodes; ++w)
      if (w != mode) chk.lim[j++] = (int32_t)dims[w];
    chk.nwords = nmodes;
    chk.ri = record_int4s(nmodes);
    const int blocks = (int)std::min<int64_t>(ceil_div<int64_t>(nnz, 256), 152 * 8);
    check_records_kernel<<<blocks, 256, 0, s>>>(static_cast<const int4*>(records), nnz, chk, err);
    SPM_CUDA_TRY(cudaGetLastError());
  }
  equal_units_kernel<<<(int)std::min<int64_t>(ceil_div<int64_t>(P + 1, 256), 1024), 256, 0, s>>>(
      nnz, P, woff);
  SPM_CUDA_TRY(cudaGetLastError());

  MttkrpArgs a{};
  a.rec = static_cast<const int4*>(records);
  a.woff = woff;
  int m = 0;
  for (int w = 0; w < nmodes; ++w)
    if (w != mode) a.fac[m++] = factors[w];
  a.out = out;
  a.cta_part = cta_part;
  a.cta_meta = cta_meta;
  a.nnz = nnz;
  a.I = dims[mode];
  a.R = rank;
  a.nin = nmodes - 1;
  a.nu = nu;
  a.err = err;    // read back by spmttkrp_noalloc_status
  a.guard = err;  // set by the record check: the blocks store nothing
  MttkrpKernelFn fn = pick_mttkrp(bf16, nmodes - 1, rank);
  const size_t smem = mttkrp_smem_bytes(rank, record_int4s(nmodes), nu, bf16 ? 2 : 4);
  SPM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<kappa, MT_THREADS, smem, s>>>(a);
  SPM_CUDA_TRY(cudaGetLastError());
  return launch_mttkrp_fixup(cta_part, cta_meta, kappa, rank, out, s);
}

extern "C" spm_status spmttkrp_noalloc_status(void* stream) {
  unsigned char* scratch = nullptr;
  SPM_TRY(scratch_address(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h = 0;
  SPM_CUDA_TRY(cudaMemcpyAsync(&h, scratch, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  if (h & DEV_ERR_INDEX) return SPM_ERR_INDEX_OUT_OF_RANGE;
  if (h & DEV_ERR_ORDER) return SPM_ERR_INVALID_ARG;
  if (h & DEV_ERR_TIMEOUT) return SPM_ERR_TIMEOUT;
  return SPM_OK;
}
