// FP32-factor MTTKRP instantiations, 2 and 3 modes.
#include "mttkrp_inst.cuh"

namespace spm {
MttkrpKernelFn pick_mttkrp_f32_a(int nin, int R) {
  return nin == 1 ? pick_mttkrp_t<float, 1>(R) : pick_mttkrp_t<float, 2>(R);
}
}  // namespace spm
