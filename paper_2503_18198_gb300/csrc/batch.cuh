// batch.cuh -- the batch object (host side): a changing set of tensors whose
// CP-ALS sweeps share launches (kernels in batch_kernels.cuh).  Used by the
// batch C ABI (batch.cu) and by the serving loop (server.cu).
#pragma once

#include <vector>

#include "batch_kernels.cuh"

struct spm_batch_s {
  int device = 0;
  int bf16 = -1;  // factor storage type of the members, -1 while empty
  std::vector<spmttkrp_plan_s*> plans;
  std::vector<spm::BatchTensor> host;  // descriptors; the device copy is newer after sweeps
  bool dirty = true;                   // host list changed since the last upload
  // Work-item tables of one mode, as offsets into `items`.
  struct ModeItems {
    int mtt_off[spm::KC_NONE] = {};
    int n_mtt[spm::KC_NONE] = {};  // (tensor, partition) per (N, R) class
    int zero_off = 0, n_zero = 0;  // (tensor, element chunk)
    int tens_off = 0, n_tens = 0;  // (tensor, 0): tensors that have this mode
    int solve_off = 0, n_solve = 0;  // (tensor, virtual block), CUDA-core solve ranks
    int tcs_off[3] = {}, n_tcs[3] = {};  // the same for the tensor-core solve, R = 16, 32, 64
    int scale_off = 0, n_scale = 0;  // CUDA-core normalisation (ranks without the tensor-core pass)
    int tcg_off[2] = {}, n_tcg[2] = {};  // tensor-core normalisation + Gram, R = 16, 32
    int gram_off = 0, n_gram = 0;    // CUDA-core Gram partials
    int fit_off = 0, n_fit = 0;  // tensors whose last mode is this one
  } mi[SPM_MAX_MODES];
  int maxN = 0;
  int maxR = 1;  // largest rank of the members (grid of the system launch)
  // device memory of the batch itself
  spm::BatchTensor* bt = nullptr;
  size_t bt_cap = 0;
  int2* items = nullptr;
  size_t items_cap = 0;
  int* queue = nullptr;  // work-queue counters, one per (mode, class)
  int grid = 0;          // persistent blocks of an MTTKRP launch
  size_t mtt_smem[spm::KC_NONE] = {};
  size_t smem_set[spm::KC_NONE] = {};  // dynamic shared memory the attribute allows
  std::vector<int2> stage;
  // side stream on which each mode's systems are formed beside its MTTKRP
  // (created when the first member is added, outside any stream capture)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace spm {

// Add a tensor (its plan, device factors, and where its weights and fit go).
// Computes the Grams of its factors on `s` (after pulling the members' state
// if the device copy is current); the device tables are rebuilt by the next
// batch_commit.  Factors must stay allocated while it is a member.
// A resumed tensor starts with `start_sweeps` sweeps done and `prev_fit` as
// the fit of its last sweep.
spm_status batch_add(spm_batch_s* B, spmttkrp_plan_s* p, void* const* factors, double* lambda,
                     double* fit, double tol, int max_sweeps, cudaStream_t s,
                     int start_sweeps = 0, double prev_fit = -1.0e300);

// Drop member t from the host list (call batch_pull first so that the
// convergence state of the others is current).
void batch_remove(spm_batch_s* B, int t);

// Synchronise `s` and copy the device descriptors (convergence state) back.
spm_status batch_pull(spm_batch_s* B, cudaStream_t s);

// Rebuild and upload the descriptors and work-item tables if the member list
// changed (stream-ordered on `s`; may allocate, so not under graph capture).
spm_status batch_commit(spm_batch_s* B, cudaStream_t s);

// The spMTTKRP of mode d for every member (zero-fill, persistent launches per
// class, fix-up), output in each member's ALS M buffer.
spm_status batch_mttkrp(spm_batch_s* B, int d, cudaStream_t s);

// One CP-ALS sweep of every active member (launches only once committed).
spm_status batch_sweep(spm_batch_s* B, cudaStream_t s);

void batch_free(spm_batch_s* B);

}  // namespace spm
