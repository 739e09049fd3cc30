// plan.cuh -- the plan object and the internal entry points between the
// library's translation units.
#pragma once

#include "common.cuh"

// Work unit of a fibre-layout copy: its range of stream entries (from its
// first nonzero to its last, headers between them included) and the fibre
// header of its first nonzero, which may lie before the range.
struct FibreUnit {
  int64_t sbeg, send;  // stream entries [sbeg, send); empty unit: sbeg == send
  int cd_first;        // output row of the unit's first nonzero
  int ca_first;        // first input-mode index of that nonzero's fibre
  int cd_last;         // output row of the nonzero before the unit's end (-1: none)
  int pad;
};

struct spm_mode_copy {
  int4* rec = nullptr;       // records, record_int4s(N) int4 per nonzero (null: lean or fibre copy)
  int2* fstream = nullptr;   // fibre copy: header entries {c_a | 2^31, c_d} each followed by
                             // the fibre's nonzero entries {c_b, value bits}; 2 entries of padding
  FibreUnit* funits = nullptr;  // fibre copy: [kappa * nu] work units
  int64_t nfib = 0;          // fibre copy: number of fibres (headers)
  int32_t* perm = nullptr;   // input position of each copy position (null: lean copy)
  int32_t* src = nullptr;    // lean copy: position in copy 0 of each copy position
  int64_t* off = nullptr;    // device int64[kappa+1] partition offsets
  int64_t* woff = nullptr;   // device int64[kappa*nu+1] work-unit offsets
  uint32_t* rowmask = nullptr;  // bit i set: output row i has a nonzero
  int64_t empty_rows = 0;    // rows without nonzeros
  int scheme = 0;            // 0 cost-balanced, 1 or 2 (Sec. III-B)
};

// Bytes of the W digit tiles of the tensor-core row solve for rank R: the
// BF16 digit stack (7 digits x R x R) and R column exponents; ranks 16, 32
// and 64 only.
inline constexpr size_t als_wdig_bytes(int R) {
  return (R == 16 || R == 32 || R == 64) ? (size_t)7 * 2 * R * R + 4 * (size_t)R : 0;
}

struct spm_als_state {
  bool ready = false;                 // Gram cache valid for `fac_ptr`
  const void* fac_ptr[SPM_MAX_MODES] = {};
  double* gram = nullptr;             // [N][R*R] Grams of the stored factors
  double* gram_part = nullptr;        // [gram_blocks][R*R] block partials
  int gram_blocks = 0;
  double* chol = nullptr;             // R*R: Cholesky factor of V (lower)
  float* winv = nullptr;              // 2*R*R: V^{-1} as hi/lo float pairs
  double* colsq_part = nullptr;       // [gram_blocks][R] column sums of Z^2
  float* colmax_part = nullptr;       // [gram_blocks][R] column maxima of |Z|
  unsigned char* wdig = nullptr;      // W = V^{-1} as BF16 digit tiles (tensor-core solve)
  double* inner_part = nullptr;       // [gram_blocks][R] sums of M .* Y
  double* lambda_ws = nullptr;        // R
  float* M = nullptr;                 // Imax*R MTTKRP output
  float* Z = nullptr;                 // Imax*R unnormalised update
  // the normal-equation systems of mode d depend only on the other modes'
  // Grams, so they are formed on a side stream while the MTTKRP of mode d runs
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

struct spmttkrp_plan_s {
  int device = 0;
  int N = 0;
  int R = 0;
  int64_t dims[SPM_MAX_MODES] = {};
  int64_t nnz = 0;
  uint32_t flags = 0;
  bool bf16 = false;
  bool lean = false;  // SPM_PLAN_LEAN: copies 1..N-1 are positions into copy 0
  bool fibre = false; // SPM_PLAN_FIBRE: every copy in the fibre layout (3 modes)
  int kappa = 0;
  int kappa_cap = 0;  // partitions the off/woff/cta arrays are sized for
  int nu = 0;      // work units per partition
  int policy = 0;  // SPM_POLICY_* >> 4
  spm_mode_copy mode[SPM_MAX_MODES];
  // MTTKRP workspace: per-partition boundary-row partial sums.
  float* cta_part = nullptr;   // [kappa][2][R]
  int* cta_meta = nullptr;     // [kappa][4]
  // Device scalars.
  int* dev_err = nullptr;      // sticky error flags (spm::DEV_ERR_*)
  double* normX2 = nullptr;    // |X|_F^2 (duplicates summed)
  double* norm_part = nullptr; // partials for normX2
  spm_als_state als;
  // host-buffer entry point: device staging of factors and outputs, and the
  // side streams / events that overlap its copies with the modes' kernels
  void* h_fac[SPM_MAX_MODES] = {};
  float* h_out[SPM_MAX_MODES] = {};
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t ev[2 * SPM_MAX_MODES + 2] = {};
  size_t bytes = 0;
  // record-copy wait bound of the MTTKRP kernel (0 = default; failure tests
  // set ~0u so the first wait gives up at once)
  uint32_t wait_limit = 0;
  // allocation bookkeeping
  void* allocs[64] = {};
  size_t alloc_bytes[64] = {};
  int nallocs = 0;
};

namespace spm {

// Allocation owned by the plan (recorded for destroy and for plan_bytes).
spm_status plan_alloc(spmttkrp_plan_s* p, void** ptr, size_t bytes);

// Replace an allocation made by plan_alloc with a new one of `bytes`
// (contents not kept).
spm_status plan_realloc(spmttkrp_plan_s* p, void** ptr, size_t bytes);

// Release one allocation made by plan_alloc (after a device synchronisation
// of the caller's stream, or stream-ordered work that no longer reads it).
void plan_free(spmttkrp_plan_s* p, void** ptr);

// Slots (work units a warp takes side by side) of the fibre-layout kernel for
// rank R: each lane holds SPM_FB_VEC ranks of a unit's rows (4: one 16-byte
// FP32 or 8-byte BF16 load per row; 8: two 16-byte FP32 loads or one 16-byte
// BF16 load), R / SPM_FB_VEC lanes per unit; 0 when the rank has no fibre
// kernel.  With 8 the per-step control work is shared by twice the slots but
// a batch more often holds a row change; 4 measured faster.
#ifndef SPM_FB_VEC
#define SPM_FB_VEC 4
#endif
inline int fibre_slots(int R) {
  return (R == 16 || R == 32 || R == 64) ? 32 * SPM_FB_VEC / R : 0;
}

// Device bytes a plan holds (resident: copies, partitions, workspace, and
// with `als` the CP-ALS state) and the most its build adds for a while
// (transient scratch), for the given shape.
void plan_bytes_estimate(int N, const int64_t* dims, int64_t nnz, int R, int kappa, bool als,
                         bool lean, size_t* resident, size_t* transient, bool fibre = false,
                         int policy = 0);

// P2 again for a new partition count (cost-balanced and Scheme 2 policies).
spm_status plan_repartition(spmttkrp_plan_s* p, int kappa, cudaStream_t s);

// P1 + P2: build every mode copy and its partition (plan.cu).
spm_status build_copies(spmttkrp_plan_s* p, const int32_t* const* idx,
                        const float* vals, cudaStream_t s);

// P3 + P4: one MTTKRP launch sequence for mode d (mttkrp.cu).
spm_status run_mttkrp(spmttkrp_plan_s* p, int mode, const void* const* factors,
                      float* out, cudaStream_t s);

// P6: one CP-ALS sweep (als.cu).
spm_status als_sweep(spmttkrp_plan_s* p, void* const* factors, double* lambda,
                     double* fit, cudaStream_t s);

// G = Y^T Y (FP64, R x R) of a stored factor with the plan's block split (als.cu).
// With `mask`, rows whose bit is clear are known to be zero and are skipped.
spm_status gram(spmttkrp_plan_s* p, const void* Y, int64_t I, double* G, cudaStream_t s,
                const uint32_t* mask = nullptr);

// Allocate the plan's CP-ALS workspace on first use (als.cu).
spm_status ensure_als_state(spmttkrp_plan_s* p);

int sm_count();

// True when an allocation failure injected by spm_inject_alloc_failure is
// due now (diag.cu).
bool alloc_fault_due();

// Partition count of a plan made with SPM_KAPPA(0): SPM_PARTITIONS_PER_SM
// per SM (-1 when the device cannot be queried).
int default_kappa();

}  // namespace spm
