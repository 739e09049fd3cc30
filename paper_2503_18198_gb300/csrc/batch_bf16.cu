// Batched persistent spMTTKRP launch, BF16 factors (all (N, R) classes).
#include <algorithm>

#include "batch_kernels.cuh"

namespace spm {

namespace {

template <int KC>
spm_status launch_class(const BatchTensor* bt, const int2* items, int nitems, int* queue, int mode,
                        int grid, size_t smem, cudaStream_t s) {
  auto fn = &mttkrp_batch_kernel<__nv_bfloat16, KC>;
  if (grid == 0) {
    // configuration only (at batch creation, outside any stream capture)
    SPM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int carve = (int)std::min<size_t>(100, (smem + 4096) * 100 / (228 * 1024) + 1);
    SPM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    return SPM_OK;
  }
  fn<<<grid, MT_THREADS, smem, s>>>(bt, items, nitems, queue, mode);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

}  // namespace

spm_status launch_batch_mttkrp_bf16(int kc, const BatchTensor* bt, const int2* items, int nitems,
                                 int* queue, int mode, int grid, size_t smem, cudaStream_t s) {
  switch (kc) {
    case KC_N3_R8: return launch_class<KC_N3_R8>(bt, items, nitems, queue, mode, grid, smem, s);
    case KC_N3_R16: return launch_class<KC_N3_R16>(bt, items, nitems, queue, mode, grid, smem, s);
    case KC_N3_R32: return launch_class<KC_N3_R32>(bt, items, nitems, queue, mode, grid, smem, s);
    case KC_N3_R64: return launch_class<KC_N3_R64>(bt, items, nitems, queue, mode, grid, smem, s);
    case KC_N4_R8: return launch_class<KC_N4_R8>(bt, items, nitems, queue, mode, grid, smem, s);
    case KC_N4_R16: return launch_class<KC_N4_R16>(bt, items, nitems, queue, mode, grid, smem, s);
    case KC_N4_R32: return launch_class<KC_N4_R32>(bt, items, nitems, queue, mode, grid, smem, s);
    case KC_N4_R64: return launch_class<KC_N4_R64>(bt, items, nitems, queue, mode, grid, smem, s);
    default: return SPM_ERR_UNSUPPORTED;
  }
}

}  // namespace spm
