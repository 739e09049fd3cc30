// Launch of the fibre-layout spMTTKRP (mttkrp_fibre.cuh) for one mode.
#include "mttkrp_fibre.cuh"

namespace spm {

using FibreKernelFn = void (*)(const FibreArgs);

static FibreKernelFn pick_fibre(bool bf16, int R) {
  switch (R) {
    case 16: return bf16 ? &mttkrp_fibre_kernel<__nv_bfloat16, 16> : &mttkrp_fibre_kernel<float, 16>;
    case 32: return bf16 ? &mttkrp_fibre_kernel<__nv_bfloat16, 32> : &mttkrp_fibre_kernel<float, 32>;
    case 64: return bf16 ? &mttkrp_fibre_kernel<__nv_bfloat16, 64> : &mttkrp_fibre_kernel<float, 64>;
    default: return nullptr;
  }
}

// The MTTKRP kernel launch of a fibre-layout copy (output clearing and the
// partition fix-up are launched by the caller, as for record copies).
spm_status launch_mttkrp_fibre(spmttkrp_plan_s* p, int mode, const void* const* factors,
                               float* out, cudaStream_t s) {
  const spm_mode_copy& c = p->mode[mode];
  FibreArgs a{};
  a.stream = c.fstream;
  a.units = c.funits;
  a.woff = c.woff;
  int m = 0;
  const void* fac[2] = {nullptr, nullptr};
  for (int w = 0; w < p->N; ++w)
    if (w != mode) fac[m++] = factors[w];
  a.fac_a = fac[0];
  a.fac_b = fac[1];
  a.out = out;
  a.cta_part = p->cta_part;
  a.cta_meta = p->cta_meta;
  a.err = p->dev_err;
  a.wait_limit = p->wait_limit;
  a.nnz = p->nnz;
  a.nu = p->nu;
  FibreKernelFn fn = pick_fibre(p->bf16, p->R);
  if (!fn || p->nu != 32 * fibre_slots(p->R)) return SPM_ERR_UNSUPPORTED;
  const size_t smem = fibre_smem_bytes(p->R, p->nu);
  SPM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int carve = (int)std::min<size_t>(100, (smem + 8192) * 100 / (228 * 1024) + 1);
  SPM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
  fn<<<p->kappa, MT_THREADS, smem, s>>>(a);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

}  // namespace spm
