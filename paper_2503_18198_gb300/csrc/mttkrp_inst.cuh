// mttkrp_inst.cuh -- kernel selection for one factor storage type and a set
// of input-mode counts.  Included by several translation units so that the
// instantiations compile in parallel.
#pragma once

#include "mttkrp_kernel.cuh"

namespace spm {

using MttkrpKernelFn = void (*)(const MttkrpArgs);

#ifndef SPM_MT_NARROW
#define SPM_MT_NARROW 0
#endif

// Fast shapes: the rank is VEC * LPN * CPL with one 16-byte load per lane
// and chunk.  Anything else uses the scalar variant (one nonzero per step).
template <typename FT, int NIN, bool LEAN = false>
MttkrpKernelFn pick_mttkrp_t(int R) {
  constexpr int RI = record_int4s(NIN > 0 ? NIN + 1 : SPM_MAX_MODES);
  constexpr int VEC = 16 / (int)sizeof(FT);
  if constexpr (sizeof(FT) == 2 && NIN == 2) {  // 3-mode BF16 with R <= 32: 8-byte lane loads
    if (R % 4 == 0 && R <= 32) {
      switch (R / 4) {
        case 1: return &mttkrp_kernel<RI, NIN, FT, 4, 1, 1, LEAN>;
        case 2: return &mttkrp_kernel<RI, NIN, FT, 4, 2, 1, LEAN>;
        case 4: return &mttkrp_kernel<RI, NIN, FT, 4, 4, 1, LEAN>;
        case 8: return &mttkrp_kernel<RI, NIN, FT, 4, 8, 1, LEAN>;
        default: break;
      }
    }
  }
#if SPM_MT_NARROW
  // FP32 rows of 32 or 64 ranks on half as many lanes, two 16-byte chunks
  // per lane: twice the nonzeros per warp step
  if constexpr (sizeof(FT) == 4 && NIN > 0) {
    if (R == 8 * VEC) return &mttkrp_kernel<RI, NIN, FT, VEC, 4, 2, LEAN>;
    if (R == 16 * VEC) return &mttkrp_kernel<RI, NIN, FT, VEC, 8, 2, LEAN>;
  }
#endif
  if (R % VEC == 0) {
    switch (R / VEC) {
      case 1: return &mttkrp_kernel<RI, NIN, FT, VEC, 1, 1, LEAN>;
      case 2: return &mttkrp_kernel<RI, NIN, FT, VEC, 2, 1, LEAN>;
      case 4: return &mttkrp_kernel<RI, NIN, FT, VEC, 4, 1, LEAN>;
      case 8: return &mttkrp_kernel<RI, NIN, FT, VEC, 8, 1, LEAN>;
      case 16: return &mttkrp_kernel<RI, NIN, FT, VEC, 16, 1, LEAN>;
      case 32: return &mttkrp_kernel<RI, NIN, FT, VEC, 32, 1, LEAN>;
      case 64: return &mttkrp_kernel<RI, NIN, FT, VEC, 32, 2, LEAN>;
      default: break;
    }
  }
  return &mttkrp_kernel<RI, NIN, FT, 1, 32, 8, LEAN>;
}

// The generic-N variant (six or more modes) only has the scalar shape.
template <typename FT>
MttkrpKernelFn pick_mttkrp_generic_t(int) {
  return &mttkrp_kernel<2, 0, FT, 1, 32, 8>;
}

}  // namespace spm
