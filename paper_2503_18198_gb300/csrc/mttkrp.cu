// mttkrp.cu -- launch sequence of one spMTTKRP along mode d (Algorithm 1's
// body for one mode): [clear output if Scheme 1] -> mttkrp kernel over the
// kappa partitions -> fix-up of rows that straddle partitions (Scheme 2).
#include <algorithm>

#include "mttkrp_kernel.cuh"

namespace spm {

using MttkrpKernelFn = void (*)(const MttkrpArgs);
MttkrpKernelFn pick_mttkrp_f32_a(int nin, int R);
MttkrpKernelFn pick_mttkrp_f32_b(int nin, int R);
MttkrpKernelFn pick_mttkrp_bf16_a(int nin, int R);
MttkrpKernelFn pick_mttkrp_bf16_b(int nin, int R);
MttkrpKernelFn pick_mttkrp_f32_c(int R);
MttkrpKernelFn pick_mttkrp_bf16_c(int R);
MttkrpKernelFn pick_mttkrp_f32_lean(int nin, int R);
MttkrpKernelFn pick_mttkrp_bf16_lean(int nin, int R);

spm_status launch_mttkrp_fibre(spmttkrp_plan_s* p, int mode, const void* const* factors,
                               float* out, cudaStream_t s);  // mttkrp_fibre.cu

MttkrpKernelFn pick_mttkrp(bool bf16, int nin, int R) {
  if (nin == 4) return bf16 ? pick_mttkrp_bf16_c(R) : pick_mttkrp_f32_c(R);
  if (bf16) return nin <= 2 ? pick_mttkrp_bf16_a(nin, R) : pick_mttkrp_bf16_b(nin, R);
  return nin <= 2 ? pick_mttkrp_f32_a(nin, R) : pick_mttkrp_f32_b(nin, R);
}

namespace {

// Rows without nonzeros (bit clear in `mask`) are written as zeros.
__global__ void zero_empty_rows_kernel(const uint32_t* __restrict__ mask, int64_t I, int R,
                                       float* __restrict__ out) {
  zero_empty_rows_body(mask, I, R, out, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                       (I + 31) / 32, (int64_t)gridDim.x * blockDim.x);
}

// One warp per partition z (see mttkrp_fixup_body).
__global__ void __launch_bounds__(256)
    mttkrp_fixup_kernel(const float* __restrict__ cta_part, const int* __restrict__ cta_meta,
                        int kappa, int R, float* __restrict__ out) {
  const int z = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (z < kappa) mttkrp_fixup_body(cta_part, cta_meta, kappa, R, out, z, threadIdx.x & 31);
}

}  // namespace

// Launch the partition fix-up on given boundary partials (used by callers
// that keep those partials outside a plan).
spm_status launch_mttkrp_fixup(const float* cta_part, const int* cta_meta, int kappa, int R,
                               float* out, cudaStream_t s) {
  if (kappa <= 1) return SPM_OK;
  const int threads = 256;
  const int blocks = (int)ceil_div<int64_t>((int64_t)kappa * 32, threads);
  mttkrp_fixup_kernel<<<blocks, threads, 0, s>>>(cta_part, cta_meta, kappa, R, out);
  SPM_CUDA_TRY(cudaGetLastError());
  return SPM_OK;
}

spm_status run_mttkrp(spmttkrp_plan_s* p, int mode, const void* const* factors, float* out,
                      cudaStream_t s) {
  if (!p || mode < 0 || mode >= p->N || !factors || !out) return SPM_ERR_INVALID_ARG;
  const int R = p->R;
  const spm_mode_copy& c = p->mode[mode];
  MttkrpArgs a{};
  const bool lean = c.src != nullptr;  // lean copy: records gathered from copy 0
  a.rec = lean ? p->mode[0].rec : c.rec;
  a.src = c.src;
  a.fmode = mode;
  a.woff = c.woff;
  int m = 0;
  for (int w = 0; w < p->N; ++w) {
    if (w == mode) continue;
    if (!factors[w] || (reinterpret_cast<uintptr_t>(factors[w]) & 15u)) return SPM_ERR_INVALID_ARG;
    a.fac[m++] = factors[w];
  }
  if (reinterpret_cast<uintptr_t>(out) & 15u) return SPM_ERR_INVALID_ARG;
  a.out = out;
  a.cta_part = p->cta_part;
  a.cta_meta = p->cta_meta;
  a.nnz = p->nnz;
  a.I = p->dims[mode];
  a.R = R;
  a.nin = p->N - 1;
  a.nu = p->nu;
  a.err = p->dev_err;
  a.wait_limit = p->wait_limit;
  const size_t out_bytes = sizeof(float) * (size_t)a.I * (size_t)R;
  if (p->nnz == 0) {
    SPM_CUDA_TRY(cudaMemsetAsync(out, 0, out_bytes, s));
    return SPM_OK;
  }
  if (c.scheme == 1) {
    SPM_CUDA_TRY(cudaMemsetAsync(out, 0, out_bytes, s));
  } else if (c.empty_rows > 0) {
    const int64_t words = (a.I + 31) / 32;
    const int blocks = (int)std::min<int64_t>(ceil_div<int64_t>(words, 256), 152 * 8);
    zero_empty_rows_kernel<<<blocks, 256, 0, s>>>(c.rowmask, a.I, R, out);
    SPM_CUDA_TRY(cudaGetLastError());
  }
  if (c.fstream) {
    SPM_TRY(launch_mttkrp_fibre(p, mode, factors, out, s));
  } else {
    MttkrpKernelFn fn = lean ? (p->bf16 ? pick_mttkrp_bf16_lean(p->N - 1, R)
                                        : pick_mttkrp_f32_lean(p->N - 1, R))
                             : pick_mttkrp(p->bf16, p->N - 1, R);
    if (!fn) return SPM_ERR_UNSUPPORTED;
    const size_t smem = mttkrp_smem_bytes(R, record_int4s(p->N), p->nu, p->bf16 ? 2 : 4);
    SPM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // Smallest shared-memory carve-out that fits: the rest of the unified
    // array is L1 for the gathered factor rows.
    const int carve = (int)std::min<size_t>(100, (smem + 4096) * 100 / (228 * 1024) + 1);
    SPM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    fn<<<p->kappa, MT_THREADS, smem, s>>>(a);
    SPM_CUDA_TRY(cudaGetLastError());
  }
  if (c.scheme != 1 && p->kappa > 1) {
    const int threads = 256;
    const int blocks = (int)ceil_div<int64_t>((int64_t)p->kappa * 32, threads);
    mttkrp_fixup_kernel<<<blocks, threads, 0, s>>>(p->cta_part, p->cta_meta, p->kappa, R, out);
    SPM_CUDA_TRY(cudaGetLastError());
  }
  return SPM_OK;
}

}  // namespace spm
