// BF16-factor MTTKRP instantiations for memory-lean copies (2 to 5 modes).
#include "mttkrp_inst.cuh"

namespace spm {
MttkrpKernelFn pick_mttkrp_bf16_lean(int nin, int R) {
  switch (nin) {
    case 1: return pick_mttkrp_t<__nv_bfloat16, 1, true>(R);
    case 2: return pick_mttkrp_t<__nv_bfloat16, 2, true>(R);
    case 3: return pick_mttkrp_t<__nv_bfloat16, 3, true>(R);
    case 4: return pick_mttkrp_t<__nv_bfloat16, 4, true>(R);
    default: return nullptr;
  }
}
}  // namespace spm
