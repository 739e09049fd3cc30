// BF16-factor MTTKRP instantiations (FP32 accumulation), 2 and 3 modes.
#include "mttkrp_inst.cuh"

namespace spm {
MttkrpKernelFn pick_mttkrp_bf16_a(int nin, int R) {
  return nin == 1 ? pick_mttkrp_t<__nv_bfloat16, 1>(R) : pick_mttkrp_t<__nv_bfloat16, 2>(R);
}
}  // namespace spm
