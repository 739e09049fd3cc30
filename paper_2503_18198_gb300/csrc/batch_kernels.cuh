// batch_kernels.cuh -- CP-ALS sweeps over many independent tensors with one
// launch per step for all of them.
//
// Every tensor keeps its own plan (mode copies, partitions, ALS workspace), so
// its arithmetic and summation order are exactly those of a single-tensor
// sweep: a tensor's result does not depend on which other tensors share the
// batch.  What changes is the launch structure:
//  * spMTTKRP: one persistent launch per mode; blocks take (tensor,
//    partition) items from a global work queue and run the partition body of
//    the single-tensor kernel on them (the per-job work queue);
//  * fix-up, empty-row zeroing and the ALS passes: one launch per step whose
//    blocks map to (tensor, virtual block) items.
// Converged tensors (fit change below the tolerance, or the sweep limit) are
// marked inactive on the device and skipped, so a CUDA graph of one sweep can
// be replayed without host round trips.
#pragma once

#include "als_tc.cuh"
#include "mttkrp_kernel.cuh"

namespace spm {

struct BatchTensor {
  MttkrpArgs margs[SPM_MAX_MODES];  // per output mode (out = the ALS M buffer)
  void* fac[SPM_MAX_MODES];
  int64_t dims[SPM_MAX_MODES];
  uint32_t* rowmask[SPM_MAX_MODES];
  const uint32_t* live[SPM_MAX_MODES];  // rowmask when the mode has empty rows, else null
  int nb_gram[SPM_MAX_MODES];   // virtual blocks of the row passes per mode
  int nb_solve[SPM_MAX_MODES];
  int nb_scale[SPM_MAX_MODES];
  int64_t gram_rpb[SPM_MAX_MODES];  // rows per Gram block
  int N, R, kappa, kclass;
  // ALS state of the tensor's plan
  double* gram;
  double* gram_part;
  double* chol;
  float* winv;
  double* colsq_part;
  float* colmax_part;
  unsigned char* wdig;  // W digit tiles (tensor-core solve ranks), else null
  double* inner_part;
  double* lambda_ws;
  float* M;
  float* Z;
  const double* normX2;
  int* err;
  double* lambda_out;  // caller's lambda slice
  double* fit_out;     // caller's fit slot
  // convergence state (device-updated)
  int active;
  int sweeps;
  int max_sweeps;
  double tol;
  double prev_fit;
};

// (N, R) classes of the batched MTTKRP dispatcher.
enum : int { KC_N3_R8, KC_N3_R16, KC_N3_R32, KC_N3_R64, KC_N4_R8, KC_N4_R16, KC_N4_R32, KC_N4_R64, KC_NONE };

inline int batch_kclass(int N, int R) {
  const int base = N == 3 ? 0 : (N == 4 ? 4 : -1);
  if (base < 0) return KC_NONE;
  switch (R) {
    case 8: return base + 0;
    case 16: return base + 1;
    case 32: return base + 2;
    case 64: return base + 3;
    default: return KC_NONE;
  }
}

// Template parameters of class KC with factor type FT (16-byte lanes: VEC = 4
// FP32 or 8 BF16 values, LPN = R / VEC lanes per nonzero).
template <int KC>
struct BatchClass {
  static constexpr int N = KC < KC_N4_R8 ? 3 : 4;
  static constexpr int R = 8 << (KC % 4);
  static constexpr int RI = N <= 3 ? 1 : 2;  // 16-byte words per record
};

// Persistent spMTTKRP over the (tensor, partition) items of one mode and one
// (N, R) class: blocks take items from a work queue in order.  One kernel per
// class keeps each instantiation's register allocation that of the
// single-tensor kernel.
template <typename FT, int KC>
__global__ void __launch_bounds__(MT_THREADS, 1)
    mttkrp_batch_kernel(const BatchTensor* __restrict__ bt, const int2* __restrict__ items,
                        int nitems, int* __restrict__ queue, int mode) {
  using C = BatchClass<KC>;
  // the lane layout the single-tensor kernel picks for this (type, rank)
  constexpr int V = (sizeof(FT) == 2 && C::N == 3 && C::R <= 32) ? 4 : 16 / (int)sizeof(FT);
  __shared__ int item;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(queue, 1);
    __syncthreads();
    const int i = item;
    __syncthreads();
    if (i >= nitems) return;
    const int2 tz = items[i];
    const BatchTensor& b = bt[tz.x];
    if (b.active) mttkrp_partition<C::RI, C::N - 1, FT, V, C::R / V, 1>(b.margs[mode], tz.y);
    __syncthreads();
    // a bounded wait that gave up may leave a copy in flight into this
    // block's ring: take no further partition into it
    if (b.active && (*(volatile const int*)b.err & DEV_ERR_TIMEOUT)) return;
  }
}

}  // namespace spm
