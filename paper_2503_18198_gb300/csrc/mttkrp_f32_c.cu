// FP32-factor MTTKRP instantiations, 5 modes (vector path).
#include "mttkrp_inst.cuh"

namespace spm {
MttkrpKernelFn pick_mttkrp_f32_c(int R) { return pick_mttkrp_t<float, 4>(R); }
}  // namespace spm
