// BF16-factor MTTKRP instantiations, 5 modes (vector path).
#include "mttkrp_inst.cuh"

namespace spm {
MttkrpKernelFn pick_mttkrp_bf16_c(int R) { return pick_mttkrp_t<__nv_bfloat16, 4>(R); }
}  // namespace spm
