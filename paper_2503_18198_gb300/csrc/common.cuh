// common.cuh -- internal helpers of the sm_103a sparse MTTKRP library.
// Used only by the library's own .cu files.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spmttkrp.h"

#define SPM_FULL_MASK 0xffffffffu

// Return SPM_ERR_CUDA from the enclosing function when a runtime call fails.
#define SPM_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t spm_e_ = (expr);                            \
    if (spm_e_ != cudaSuccess) {                            \
      (void)cudaGetLastError();                             \
      return spm_e_ == cudaErrorMemoryAllocation ? SPM_ERR_OOM : SPM_ERR_CUDA; \
    }                                                       \
  } while (0)

#define SPM_TRY(expr)                    \
  do {                                   \
    spm_status spm_s_ = (expr);          \
    if (spm_s_ != SPM_OK) return spm_s_; \
  } while (0)

#include <nvtx3/nvToolsExt.h>

namespace spm {

// Words per nonzero record of a mode copy: c_d, the N-1 input-mode indices in
// ascending mode order, the value bits, zero padding to a multiple of 4 words
// (16 bytes) so that a record is fetched with 128-bit loads.
__host__ __device__ constexpr int record_int4s(int nmodes) {
  return (nmodes + 1 + 3) / 4;
}

// Device-side error flags (or-ed into one int in plan memory).
enum : int {
  DEV_ERR_INDEX = 1,
  DEV_ERR_NUMERIC = 2,
  DEV_ERR_TIMEOUT = 4,
  DEV_ERR_ORDER = 8,  // caller-held records not sorted by the output-mode index
};

// 128-bit streaming load that does not allocate in L1: the tensor copy is
// read exactly once per MTTKRP and must not evict factor rows.
__device__ __forceinline__ int4 ld_stream_v4(const int4* p) {
  int4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

// 128-bit read-only load of factor data (cached in L1 and L2).
__device__ __forceinline__ float4 ld_factor_v4(const void* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}


__device__ __forceinline__ void bf16x8_to_f32(const float4 raw, float* out) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 f = __bfloat1622float2(h[i]);
    out[2 * i] = f.x;
    out[2 * i + 1] = f.y;
  }
}

// ---- shared-memory barriers and 1-D bulk copies (TMA engine, sm_90+) ----

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Invalidate a barrier with no pending operation so its word can be
// initialised again (persistent blocks that run several partitions).
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Make barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Global -> shared bulk copy completing on `bar` (addresses and size 16-byte
// multiples).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

#ifndef SPM_MBAR_SUSPEND_NS
#define SPM_MBAR_SUSPEND_NS 0
#endif

// One poll of a barrier phase.  With a non-zero suspend hint the waiting
// thread sleeps (up to the hint) until the phase completes instead of
// spinning through issue slots.
// L2 eviction-priority policies (createpolicy): the streamed tensor copy is
// read once (evict first), the gathered factor rows are reused (evict last).
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// Bulk copy with an L2 cache policy for the source lines.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// 128-bit read-only load with an L2 cache policy.
// Read-only 16-byte load with an L2 policy, schedulable like a plain load.
__device__ __forceinline__ uint4 ld_nc_v4_pol(const void* p, uint64_t policy) {
  uint4 r;
  asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p), "l"(policy));
  return r;
}

// Packed FP32 pairs (sm_100 and later): each lane of the pair is rounded
// exactly as the scalar mul.rn / fma.rn.
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// 16 bytes of a read-only row as two FP32 pairs, ready for the f32x2 ops
__device__ __forceinline__ ulonglong2 ld_nc_v2_u64(const void* p) {
  ulonglong2 r;
  asm("ld.global.nc.v2.u64 {%0,%1}, [%2];" : "=l"(r.x), "=l"(r.y) : "l"(p));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

__device__ __forceinline__ uint4 ld_nc_v4_hint(const void* p, uint64_t policy) {
  uint4 r;
  asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p), "l"(policy));
  return r;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
#if SPM_MBAR_SUSPEND_NS > 0
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"((uint32_t)SPM_MBAR_SUSPEND_NS)
      : "memory");
#else
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
#endif
  return ok != 0;
}

// Bounded wait on a phase of `bar`.  Returns false (and the caller records a
// timeout) if the phase has not completed after `limit` polls; every poll
// itself suspends for a hardware-chosen interval, so the bound is seconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t limit = (1u << 24)) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// NVTX range for the duration of a host scope (shown by profilers that
// record NVTX; free otherwise).
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};

template <typename T>
__host__ __device__ inline T ceil_div(T a, T b) {
  return (a + b - 1) / b;
}

}  // namespace spm
