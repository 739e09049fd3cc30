// BF16-factor MTTKRP instantiations, 4 modes and the generic >= 6 modes.
#include "mttkrp_inst.cuh"

namespace spm {
MttkrpKernelFn pick_mttkrp_bf16_b(int nin, int R) {
  return nin == 3 ? pick_mttkrp_t<__nv_bfloat16, 3>(R) : pick_mttkrp_generic_t<__nv_bfloat16>(R);
}
}  // namespace spm
