/*
 * spmttkrp.h -- C ABI of the GB300 (sm_103a) sparse MTTKRP / CPD-ALS library.
 *
 * The library computes, for an N-mode sparse tensor X in COO form and dense
 * factor matrices Y_0..Y_{N-1} (I_w x R), the sparse MTTKRP along any mode d
 *
 *     M_d(i, r) = sum over nonzeros x with c_d(x) = i of
 *                 val(x) * prod_{w != d} Y_w(c_w(x), r)
 *
 * (Eq. 1 of "Accelerating Sparse MTTKRP for Small Tensor Decomposition on
 * GPU", written elementwise in its Sec. II-A6 and generalised to N modes in
 * its Algorithm 2), and CP-ALS sweeps built on it (Sec. II-A5).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers marked "device" are CUDA device pointers of the current device;
 *   pointers marked "host" are ordinary host memory.
 * - Matrices are row-major with leading dimension R (element (i, r) at
 *   i*R + r).  Indices are int32, values FP32.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Every call is stream-ordered and returns without waiting for
 *   the GPU, except spmttkrp_plan, which synchronises `stream` once to read
 *   its validation flag.
 * - Errors are returned as spm_status; nothing is thrown across the ABI and
 *   no call aborts the process.  Device-side checks set flags that the host
 *   reads; no kernel traps.  A failing call leaves caller-owned outputs in an
 *   unspecified state.
 * - The library never calls into any CPU fallback: every step runs in its own
 *   CUDA kernels.  Loading it on a machine without a CUDA device is fine;
 *   calls then return SPM_ERR_CUDA.
 */
#ifndef SPMTTKRP_H_
#define SPMTTKRP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spmttkrp_plan_s *spmttkrp_plan_t;

typedef enum {
  SPM_OK = 0,
  SPM_ERR_INVALID_ARG = 1,        /* bad count, pointer, mode, rank or flag   */
  SPM_ERR_INDEX_OUT_OF_RANGE = 2, /* some idx[w][k] < 0 or >= dims[w]         */
  SPM_ERR_OOM = 3,                /* a device allocation failed               */
  SPM_ERR_CUDA = 4,               /* a CUDA runtime call failed               */
  SPM_ERR_NUMERIC = 5,            /* ALS system not positive definite / NaN   */
  SPM_ERR_TIMEOUT = 6,            /* a bounded device-side wait gave up       */
  SPM_ERR_UNSUPPORTED = 7         /* valid request outside what is built      */
} spm_status;

/* ---- plan flags ---------------------------------------------------------- */
/* Storage type of the factor matrices passed to spmttkrp_run/cpd_als_step.
 * BF16 halves the bytes gathered per nonzero; accumulation stays FP32. */
#define SPM_FACTOR_FP32 0x0u
#define SPM_FACTOR_BF16 0x1u
#define SPM_FACTOR_MASK 0x1u

/* Partitioning policy of the nonzeros of each mode copy across the kappa
 * thread-block partitions (Sec. III-B) and, inside each partition, into
 * NU = SPM_UNITS_PER_PARTITION(R) work units that the block's warps take in
 * turn:
 *  BALANCED (default) the copy (in key order) is cut into kappa * NU
 *           contiguous work units of equal cost, where a
 *           nonzero costs 1, plus SPM_ROW_COST if it is the first nonzero of
 *           its output row (a row change is what the kernel pays for beyond
 *           streaming).  Unit j starts at the smallest copy position k
 *           with C(k) * P >= j * C(nnz), C(k) = k + SPM_ROW_COST * (rows that
 *           start before k), P = kappa * NU.  Partition z is units
 *           z*NU .. (z+1)*NU-1.  This keeps the
 *           equal-nnz shape of Scheme 2 while accounting for the sparsity of
 *           the output mode (row boundaries).
 *  SCHEME2  equal distribution of nonzeros (Sec. III-B2): partition z holds
 *           copy positions [floor(z*nnz/kappa), floor((z+1)*nnz/kappa)).
 *  SCHEME1  equal distribution of output indices (Sec. III-B1): rows with at
 *           least one nonzero are ordered by degree (descending, ties by
 *           index) and dealt cyclically to the partitions; the copy is then
 *           ordered by partition, so no row spans two partitions.
 *  ADAPTIVE the paper's rule per mode: SCHEME1 when I_d >= kappa, else
 *           SCHEME2 (Sec. III-B).
 * With SCHEME1/SCHEME2 each partition is split into work units of equal
 * nonzero count: unit w of partition z starts at
 * off[z] + floor((off[z+1] - off[z]) * w / NU).
 * Rows that straddle units or partitions are combined deterministically. */
#define SPM_POLICY_BALANCED (0u << 4)
#define SPM_POLICY_SCHEME2 (1u << 4)
#define SPM_POLICY_SCHEME1 (2u << 4)
#define SPM_POLICY_ADAPTIVE (3u << 4)
#define SPM_POLICY_MASK (0xFu << 4)

/* work units per partition for rank R: 4096 / R clamped to [16, 128] */
#define SPM_UNITS_PER_PARTITION(R) \
  ((4096 / (R)) < 16 ? 16 : ((4096 / (R)) > 128 ? 128 : (4096 / (R))))
#define SPM_ROW_COST 16 /* extra cost of a row start, in nonzeros */

/* Memory-lean plan: only the mode-0 copy holds records; every other mode
 * keeps its order as 32-bit positions into that copy (4 bytes per nonzero
 * instead of a 16- or 32-byte record), and its MTTKRP gathers the records in
 * that order.  Results are bitwise those of the full plan (same nonzero
 * order, same arithmetic).  BALANCED and SCHEME2 policies only; not for
 * batches (SPM_ERR_UNSUPPORTED).  The paper keeps one copy per mode
 * (Sec. III-C); this trades gather traffic for memory when N copies do not
 * fit. */
#define SPM_PLAN_LEAN (1u << 8)

/* Fibre layout of the mode copies (3-mode tensors, ranks 16, 32 and 64, FP32
 * or BF16 factors, BALANCED or SCHEME2 policies; otherwise
 * SPM_ERR_UNSUPPORTED).  Each copy, still in the key order above, is grouped
 * into fibres -- maximal runs of nonzeros sharing (c_d, c_a), a being the
 * first input mode -- and stored as one stream of 8-byte entries: a header
 * {c_a | 2^31, c_d} for each fibre followed by an entry {c_b, value bits} for
 * each of its nonzeros (CSF-style, cf. the compressed formats that Sec. II
 * contrasts with the per-mode COO copies of Sec. III-C).  The MTTKRP gathers
 * the row Y_a(c_a) once per fibre instead of once per nonzero, and the copy
 * takes 8 bytes per nonzero plus 8 per fibre instead of 16 per nonzero.
 * Permutations, partitions and work units are those of the record layout
 * (same P1 order, same P2 rule); work units per partition are 32 x 128 / R
 * (the record layout's count at R = 32 and 64, twice it at R = 16).
 * Results agree with the record layout within FP32 summation order.  Not
 * for batches, servers, repartitioning or the partition autotuner
 * (SPM_ERR_UNSUPPORTED). */
#define SPM_PLAN_FIBRE (1u << 9)

/* Number of partitions kappa.  0 (default) = SPM_PARTITIONS_PER_SM times the
 * device's SM count.  The paper assigns one partition per streaming
 * multiprocessor (Sec. III-B); on GB300 two resident waves of partition
 * blocks per SM balance the per-partition time variance (the block
 * scheduler gives a free SM the next partition).  Any value 1..65535 may be
 * forced, e.g. SPM_KAPPA(sm count) for the paper's one-per-SM layout. */
#define SPM_PARTITIONS_PER_SM 2
#define SPM_KAPPA(k) (((uint32_t)(k) & 0xFFFFu) << 16)
#define SPM_KAPPA_OF(flags) (((uint32_t)(flags) >> 16) & 0xFFFFu)

/* Limits of the library. */
#define SPM_MAX_MODES 7
#define SPM_MAX_RANK 256

/* ---- plan ---------------------------------------------------------------- */

/* Build the mode-specific tensor copies and their partitions
 * (Sec. III-C: one COO copy per output mode; Sec. III-B: the partitions).
 *
 *  out      host; receives the plan handle (NULL on failure).
 *  nmodes   N, 2 <= N <= SPM_MAX_MODES.
 *  dims     host int64[N]; 1 <= dims[w] < 2^31.
 *  nnz      number of nonzeros, 0 <= nnz < 2^31 - 2^20.
 *  idx      host array of N device pointers, idx[w] = int32[nnz] mode-w
 *           coordinates.  Duplicate coordinates are allowed and are summed
 *           (MTTKRP is linear in the values).
 *  vals     device float[nnz].
 *  rank     R, 1 <= R <= SPM_MAX_RANK; factors passed later must have R
 *           columns.
 *  flags    SPM_FACTOR_*, SPM_POLICY_*, SPM_KAPPA(k), or-ed.
 *  stream   cudaStream_t as void*.
 *
 * For every mode d the copy holds the nonzeros ordered by the key
 * (c_d, then c_w for w != d in ascending w, then input position); with
 * SCHEME1 the copy is further ordered by partition id first (stable).
 * All indices are checked on the device: any index outside [0, dims[w])
 * yields SPM_ERR_INDEX_OUT_OF_RANGE and no plan.
 * Ownership: the plan copies everything it needs, so idx/vals may be freed
 * once this call returns.  The plan owns all its device memory until
 * spmttkrp_plan_destroy. */
spm_status spmttkrp_plan(spmttkrp_plan_t *out, int nmodes,
                         const int64_t *dims, int64_t nnz,
                         const int32_t *const *idx, const float *vals,
                         int rank, uint32_t flags, void *stream);

/* Device bytes held by the plan (all copies, permutations, partitions and
 * its workspace) -- the "total memory consumption" of Sec. V-C and the
 * admission figure of a serving loop.  `bytes` is host. */
spm_status spmttkrp_plan_bytes(spmttkrp_plan_t plan, size_t *bytes);

/* Input positions of the nonzeros of the mode-`mode` copy, in copy order
 * (the permutation pi_d of Sec. III-B2's ordering).  perm: device
 * int64[nnz]. */
spm_status spmttkrp_plan_permutation(spmttkrp_plan_t plan, int mode,
                                     int64_t *perm, void *stream);

/* Partition offsets of the mode-`mode` copy: off[z]..off[z+1] are the copy
 * positions of partition B_{d,z} (Algorithm 1), z = 0..kappa-1.
 * off: device int64[kappa+1].  *kappa_out (host, may be NULL) = kappa. */
spm_status spmttkrp_plan_partition(spmttkrp_plan_t plan, int mode,
                                   int64_t *off, int *kappa_out,
                                   void *stream);

/* Number of fibres (distinct (c_d, c_a) pairs, a the first input mode) of the
 * mode-`mode` copy of a plan made with SPM_PLAN_FIBRE (host int64 *nfib);
 * SPM_ERR_UNSUPPORTED for other plans. */
spm_status spmttkrp_plan_fibre_count(spmttkrp_plan_t plan, int mode, int64_t *nfib);

/* Policy used for mode `mode` after ADAPTIVE is resolved: 1 = Scheme 1,
 * 2 = Scheme 2 (Sec. III-B), 0 = cost-balanced.  `scheme` is host. */
spm_status spmttkrp_plan_scheme(spmttkrp_plan_t plan, int mode, int *scheme);

/* Work-unit offsets of the mode-`mode` copy: off[j]..off[j+1] are the copy
 * positions of work unit j, j = 0..kappa*NU-1 with NU =
 * SPM_UNITS_PER_PARTITION(rank) (see the policy flags above).
 * off: device int64[kappa*NU+1]. */
spm_status spmttkrp_plan_work_units(spmttkrp_plan_t plan, int mode, int64_t *off,
                                    void *stream);

/* Release the plan and all its device memory (stream-ordered frees after a
 * device synchronisation).  NULL is ignored. */
void spmttkrp_plan_destroy(spmttkrp_plan_t plan);

/* ---- MTTKRP -------------------------------------------------------------- */

/* M_mode = X_(mode) (Khatri-Rao product of the other factors), Eq. 1 /
 * Algorithm 1 for one mode.
 *
 *  factors  host array of N device pointers, factors[w] = I_w x R row-major,
 *           float or bf16 as the plan's SPM_FACTOR_* flag says; factors[mode]
 *           is not read and may be NULL.  Each must be 16-byte aligned.
 *  out      device float[I_mode * R], overwritten (rows without nonzeros are
 *           written as zero).  Must not alias a factor.
 *  stream   cudaStream_t as void*.
 *
 * Accumulation is FP32; the summation order is fixed by the plan, so repeated
 * calls give bitwise identical results.  Calls on one plan that overlap on
 * the GPU (different streams, no ordering) race on the plan's workspace. */
spm_status spmttkrp_run(spmttkrp_plan_t plan, int mode,
                        const void *const *factors, float *out, void *stream);

/* MTTKRP along one mode with no device allocation (the paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * while they run, e.g. a serving loop confined to a memory pool sized at
 * start-up, or code running where cudaMalloc would synchronise the device).
 *
 * The caller passes a mode copy it holds itself instead of a plan:
 *  nmodes, dims, rank  as for spmttkrp_plan; mode = the output mode d.
 *  records  device, nnz records of 16 * ceil((nmodes+1)/4) bytes each:
 *           int32 words [c_d, c_w for w != d in ascending w, value bits
 *           (FP32), zero padding], sorted by c_d (records of one output row
 *           contiguous, rows ascending).  16-byte aligned.
 *  factors  host array of nmodes device pointers as for spmttkrp_run.
 *  flags    SPM_FACTOR_* and SPM_KAPPA(k); work units are equal nonzero
 *           splits (no plan, so no cost-balanced partition).
 *  out      device float[dims[mode] * rank], overwritten.
 * The records are checked on the device first (one extra read of them): an
 * index outside its mode's range or a record whose c_d is smaller than the
 * one before it makes the call store nothing but the cleared `out`, so bad
 * records cannot send a gather or a store outside the caller's buffers.
 * The call returns before the GPU has run (it does not synchronise), so such
 * a device-side finding -- and a record-copy wait that gave up
 * (SPM_ERR_TIMEOUT, output incomplete) -- is reported by
 * spmttkrp_noalloc_status, not by this call's return value.
 * Its only scratch (work-unit offsets and partition boundary partials) is a
 * file-scope __device__ array of SPM_NOALLOC_SCRATCH_BYTES that every GPU
 * holds from library load to process exit; a request whose scratch would
 * exceed it (roughly kappa * (8*rank + 16) + 8 * kappa * units bytes)
 * returns SPM_ERR_UNSUPPORTED.  The call allocates nothing (no cudaMalloc,
 * no cudaFree, no allocating library routine); it clears `out` with
 * cudaMemsetAsync and writes every scratch byte it later reads, so nothing
 * carries over from the previous call.  All calls share the one array:
 * calls that overlap on the GPU (different streams without ordering, or
 * different host threads) race and give wrong results.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture. */
#define SPM_NOALLOC_SCRATCH_BYTES (1u << 20)
spm_status spmttkrp_run_noalloc(int nmodes, const int64_t *dims, int64_t nnz,
                                int mode, int rank, const void *records,
                                const void *const *factors, uint32_t flags,
                                float *out, void *stream);

/* Synchronise `stream` and report the device-side outcome of the latest
 * spmttkrp_run_noalloc call on the current device (the paper has no
 * counterpart): SPM_OK, SPM_ERR_INDEX_OUT_OF_RANGE (an index outside its
 * mode's range), SPM_ERR_INVALID_ARG (records not sorted by c_d) or
 * SPM_ERR_TIMEOUT (a record-copy wait gave up).  It reads the error word of
 * the same shared scratch array, so it allocates nothing either; a later
 * call on the device replaces the outcome it reports. */
spm_status spmttkrp_noalloc_status(void *stream);

/* ---- CPD-ALS --------------------------------------------------------------- */

/* spMTTKRP along every mode 0..N-1 from and to host memory:
 *  host_factors  host array of N host pointers to the factors (I_w x R,
 *                FP32 or BF16 per the plan, row-major);
 *  host_out      host array of N host pointers to the outputs (I_d x R FP32).
 * The factors are copied to device staging buffers owned by the plan
 * (allocated on the first call), factors 1..N-1 first so that mode 0 starts
 * while factor 0 is still in flight; each output is copied back on a side
 * stream while the next mode computes.  Launch-only: the call returns once
 * everything is queued, and work queued on `stream` afterwards (or a
 * synchronisation of it) sees all copies complete.  With pinned host memory
 * the copies are asynchronous and overlap; with pageable memory they are
 * correct but staged by the driver.  The host buffers must stay valid until
 * then.  The paper runs its kernel on device-resident data; this is the
 * host-facing form of the same computation. */
spm_status spmttkrp_run_all_host(spmttkrp_plan_t plan, const void *const *host_factors,
                                 float *const *host_out, void *stream);

/* One CP-ALS sweep over modes 0..N-1 in order (Sec. II-A5), Gauss-Seidel:
 * for each d,
 *   M      = spMTTKRP_d(factors)                     (the plan's kernels)
 *   V      = Hadamard over w != d of (Y_w^T Y_w)     (R x R, FP64)
 *   Z      = M V^{-1}, through the FP64 Cholesky factor of V
 *   lambda = column 2-norms of Z;  Y_d = Z diag(1/lambda) (columns with
 *            lambda_r = 0 are left as they are), stored as FP32 or BF16.
 * After the last mode the fit 1 - |X - Xhat|_F / |X|_F is evaluated from
 * |X|^2, lambda, the Grams and the last mode's M (Kolda & Bader).
 *
 *  factors  host array of N device pointers, updated in place.
 *  lambda   device double[R], receives the weights of the last mode.
 *  fit      device double[1] or NULL.
 *  stream   cudaStream_t as void*.
 *
 * The Gram of each factor is cached in the plan and refreshed after its
 * update; the cache is (re)built from `factors` on the first call and
 * whenever the factor pointers change.  A caller that writes the factors
 * itself between calls (a restart, a checkpoint restored into the same
 * buffers) calls cpd_als_reset first.  If V is not numerically positive
 * definite (or not finite) the sweep stops at that mode, the device-side
 * error flag makes the plan's later sweeps skip their work, and
 * spmttkrp_plan_status reports SPM_ERR_NUMERIC and clears the flag (the
 * check is device-side, so it is seen at the next synchronising call).
 * The CP-ALS state is the factors and lambda, both the caller's: a run
 * resumed from copies of them continues bitwise as the uninterrupted one.
 * Stream order: V and its inverse for mode d need no MTTKRP output, so they
 * are formed on a side stream owned by the plan, forked from `stream` with
 * an event and joined back into it before the solve of mode d; work queued
 * on `stream` after the call sees the whole sweep.  Calls on one plan from
 * different streams must not overlap (they share the plan's workspace). */
spm_status cpd_als_step(spmttkrp_plan_t plan, void *const *factors,
                        double *lambda, double *fit, void *stream);

/* Forget the cached Grams: the next cpd_als_step rebuilds them from its
 * factors.  Host only. */
spm_status cpd_als_reset(spmttkrp_plan_t plan);

/* Device bytes a plan of this shape holds once cpd_als_step has run on it
 * (*resident: mode copies, partitions, MTTKRP and CP-ALS workspace; equals
 * spmttkrp_plan_bytes of such a plan) and the most its build adds for a while
 * on top (*transient, may be NULL: the sort scratch).  Factors, lambda and
 * fit buffers are the caller's and not included.  Host only; with
 * SPM_KAPPA(0) in flags the partition count comes from the current device's
 * SM count (SPM_ERR_CUDA when there is no device), with an explicit kappa no
 * device is touched. */
spm_status spmttkrp_plan_bytes_estimate(int nmodes, const int64_t *dims, int64_t nnz,
                                        int rank, uint32_t flags, size_t *resident,
                                        size_t *transient);

/* Re-run P2 (Sec. III-B) for a new partition count kappa (0 = the default of SPM_KAPPA(0),
 * else 1..65535); the mode copies are kept.  Only for the BALANCED and
 * SCHEME2 policies (else SPM_ERR_UNSUPPORTED).  Growing kappa beyond the
 * largest value the plan has had synchronises `stream` and reallocates the
 * partition arrays.  Results of spmttkrp_run do not depend on kappa beyond
 * FP32 summation order.  Must not be called while a batch holds the plan. */
spm_status spmttkrp_plan_repartition(spmttkrp_plan_t plan, int kappa, void *stream);

/* Autotune the partition count of one plan: for each candidate kappa
 * (kappas[0..nkappas-1]; NULL = {SM count, 2 x SM count}) the plan is
 * repartitioned and spmttkrp_run of every mode is timed with CUDA events on
 * `stream` (best of `reps` after one warm-up, outputs written to the plan's
 * CP-ALS workspace, which is allocated if absent).  The plan is left at the
 * fastest candidate, *chosen receives it and ms[c] (host, may be NULL) each
 * candidate's time for all modes.  Factors as for spmttkrp_run (read only).
 * BALANCED and SCHEME2 policies only.  Synchronises `stream`.  The paper fixes
 * one partition per SM (Sec. III-B); which count is fastest on GB300 depends
 * on the tensor's skew, hence the measurement. */
spm_status spmttkrp_plan_autotune(spmttkrp_plan_t plan, const void *const *factors,
                                  const int *kappas, int nkappas, int reps, int *chosen,
                                  float *ms, void *stream);

/* ---- batched CP-ALS over many tensors ---------------------------------------- */

/* A batch runs CP-ALS sweeps (Sec. II-A5, as cpd_als_step) over many independent
 * tensors with one launch per step for all of them: the spMTTKRP of a mode is
 * one persistent launch whose blocks take (tensor, partition) items from a work
 * queue (Algorithm 1's partitions of every tensor), and the ALS passes are
 * launches whose blocks map to (tensor, block) items.  The paper runs one
 * tensor at a time; grouping the tensors only changes the launch structure:
 * each tensor keeps its plan, arithmetic and summation order, so its result is
 * bitwise the one cpd_als_step gives it alone, whatever else is in the batch.
 *
 *  plans     host array of ntensors plans, all with the same SPM_FACTOR_* type,
 *            N in {3, 4}, rank in {8, 16, 32, 64}, policy BALANCED or SCHEME2;
 *            otherwise SPM_ERR_UNSUPPORTED.  The plans must outlive the batch.
 *  factors   host array [ntensors * SPM_MAX_MODES]: factors[t*SPM_MAX_MODES+w]
 *            is tensor t's device factor w (as for cpd_als_step, 16-byte
 *            aligned); updated in place by every sweep.  Fixed for the batch's
 *            life.
 *  lambdas   device double[sum of ranks]: tensor t's weights start at the sum
 *            of the ranks of tensors 0..t-1.
 *  fits      device double[ntensors]: fit after each tensor's latest sweep.
 *  tol, max_sweeps  a tensor stops (is skipped by later sweeps) once
 *            |fit - previous fit| < tol or it has done max_sweeps sweeps; the
 *            decision is taken on the device.
 * Creation computes the Grams of all factors and synchronises `stream`. */
typedef struct spm_batch_s *spm_batch_t;
spm_status spm_batch_create(spm_batch_t *out, int ntensors,
                            const spmttkrp_plan_t *plans, void *const *factors,
                            double *lambdas, double *fits, double tol,
                            int max_sweeps, void *stream);

/* One sweep over every still-active tensor.  Launch-only (no host
 * synchronisation, no allocation): can be captured in a CUDA graph and
 * replayed.  Each mode's systems are formed on a side stream of the batch
 * (created when the first tensor is added), forked from and joined back
 * into `stream` with events, so a capture on `stream` records them too. */
spm_status spm_batch_sweep(spm_batch_t batch, void *stream);

/* Synchronise `stream`; active[t] (host) = 1 while tensor t still iterates,
 * sweeps[t] (host, may be NULL) = sweeps done. */
spm_status spm_batch_status(spm_batch_t batch, int *active, int *sweeps,
                            void *stream);

/* Release the batch (not the plans or the caller's buffers). */
void spm_batch_destroy(spm_batch_t batch);

/* Autotuner of the batched spMTTKRP: picks the nonzeros per partition.  For
 * each candidate c (c > 0: every tensor gets kappa = ceil(nnz / c) partitions,
 * at most 65535; c == 0: the plan default, SPM_KAPPA(0)) the plans are repartitioned
 * (spmttkrp_plan_repartition) and the batched spMTTKRP of all modes is timed
 * with CUDA events on `stream`, the best of `reps` runs after one warm-up.
 * The plans are left partitioned for the fastest candidate (*chosen);
 * ms[c] (host, may be NULL) receives each candidate's time.  Factors: as for
 * spm_batch_create (read only).  Synchronises `stream`.  Same plan
 * restrictions as spm_batch_create; no batch may hold the plans meanwhile. */
spm_status spm_batch_autotune(int ntensors, const spmttkrp_plan_t *plans,
                              void *const *factors, const int64_t *candidates,
                              int ncandidates, int reps, int64_t *chosen,
                              float *ms, void *stream);

/* ---- serving: continuous batching of CP-ALS jobs ------------------------------ */

/* A server runs CP-ALS jobs (Sec. II-A5 as cpd_als_step, until the fit changes
 * by less than the job's tolerance or its sweep limit) on the current device.
 * The caller drives it with spm_server_step in a loop: each step launches one
 * batched sweep of every running job (as spm_batch_sweep), admits queued jobs
 * in arrival order while the running-job limit and the device-memory budget
 * allow (building their plans on a second stream, overlapping the sweep),
 * then retires the jobs that stopped.  A job's result is bitwise the one
 * cpd_als_step gives on a plan with the same flags, whatever else runs.
 * The paper has no serving layer; this is the GPU-resident job loop around
 * its MTTKRP. */
typedef struct spm_server_s *spm_server_t;

enum { SPM_JOB_QUEUED = 0, SPM_JOB_RUNNING = 1, SPM_JOB_DONE = 2, SPM_JOB_FAILED = 3 };

typedef struct {
  int nmodes;                  /* 3 or 4                                     */
  const int64_t *dims;         /* host [nmodes]                              */
  int64_t nnz;
  const int32_t *const *idx;   /* host array of nmodes device pointers [nnz] */
  const float *vals;           /* device [nnz]                               */
  int rank;                    /* 8, 16, 32 or 64                            */
  const float *const *init;    /* host array of nmodes device pointers to the
                                  initial FP32 factors I_w x R (16-byte
                                  aligned; rounded to BF16 for BF16 servers) */
  double tol;                  /* stop when |fit change| < tol               */
  int max_sweeps;              /* ... or after this many sweeps (>= 1)       */
} spm_job_desc;

typedef struct {
  int state;                   /* SPM_JOB_*                                  */
  spm_status status;           /* why, when SPM_JOB_FAILED                   */
  int sweeps;                  /* sweeps run (when done)                     */
  double fit;                  /* final fit (when done)                      */
  size_t bytes;                /* device bytes the job holds now             */
  size_t est_bytes;            /* its admission estimate (plan + factors)    */
  double queued_ms;            /* submit -> admission (host clock)           */
  double total_ms;             /* submit -> retirement: time to solution     */
} spm_job_info;

/* hbm_budget: device bytes the server's jobs may hold at once (plans,
 * factors, and the transient sort scratch of a build); max_active: running
 * jobs at most; flags: SPM_FACTOR_FP32 or SPM_FACTOR_BF16;
 * nnz_per_partition: partitions per job = ceil(nnz / this), 1..65535
 * (0 = the plan default, SPM_KAPPA(0)). */
spm_status spm_server_create(spm_server_t *out, size_t hbm_budget, int max_active,
                             uint32_t flags, int64_t nnz_per_partition);

/* Queue a job; *job receives its id.  The inputs (idx, vals, init) must be
 * complete on the device (their producing stream synchronised) and stay valid
 * until the job has left SPM_JOB_QUEUED.  A job whose estimate exceeds the
 * budget fails with SPM_ERR_OOM at its turn. */
spm_status spm_server_submit(spm_server_t server, const spm_job_desc *desc, int64_t *job);

/* One step (sweep, admission, retirement); synchronises the server's streams.
 * *running / *queued (may be NULL) receive the counts after the step. */
spm_status spm_server_step(spm_server_t server, int *running, int *queued);

spm_status spm_server_job(spm_server_t server, int64_t job, spm_job_info *info);

/* Checkpoint of a running job between steps: its factors (stored type,
 * device, NULL entries skipped), weights (device double[R], may be NULL),
 * sweeps done and the fit of its last sweep (host).  Synchronises `stream`. */
spm_status spm_server_snapshot(spm_server_t server, int64_t job, void *const *factors,
                               double *lambda, int *sweeps, double *prev_fit, void *stream);

/* Queue a job resumed from a snapshot: desc->init holds the snapshot's
 * factors as FP32 (exact for BF16 ones), `sweeps_done` and `prev_fit` the
 * snapshot's counters (0 <= sweeps_done < desc->max_sweeps).  On a server
 * with the same flags and nnz_per_partition the job then finishes bitwise as
 * it would have without the interruption. */
spm_status spm_server_resume(spm_server_t server, const spm_job_desc *desc, int sweeps_done,
                             double prev_fit, int64_t *job);

/* Copy a finished job's factors (stored type, device, NULL entries skipped)
 * and weights (device double[R], may be NULL) out on `stream`, synchronise,
 * and release the job.  Returns the failure status for a failed job. */
spm_status spm_server_result(spm_server_t server, int64_t job, void *const *factors,
                             double *lambda, void *stream);

/* Device bytes held by the server's jobs now, and the budget. */
spm_status spm_server_usage(spm_server_t server, size_t *used, size_t *budget);

void spm_server_destroy(spm_server_t server);

/* ---- failure-detection hooks (tests) ----------------------------------------- */

/* Launch a kernel whose bounded wait on an mbarrier that nothing completes
 * gives up after `limit` polls (the same wait the MTTKRP kernel uses for its
 * record copies); returns SPM_ERR_TIMEOUT when the timeout was recorded, as
 * expected, with the CUDA context still usable.  Synchronises `stream`. */
spm_status spm_selftest_wait_timeout(uint32_t limit, void *stream);

/* Run the plan's spMTTKRP along `mode` (arguments as for spmttkrp_run) with
 * the record-copy waits of its kernel set to give up at once: every warp's
 * first wait times out, waits for the copies it already issued to land, and
 * its block stores nothing (no output row, no boundary partial).  Returns
 * what spmttkrp_plan_status then reports -- SPM_ERR_TIMEOUT, as expected --
 * with the CUDA context still usable and `out` written only inside its
 * I_mode x R rows (rows without nonzeros are zeroed, the others keep their
 * old contents).  Synchronises `stream`.  For the failure-detection tests. */
spm_status spm_selftest_mttkrp_timeout(spmttkrp_plan_t plan, int mode,
                                       const void *const *factors, float *out,
                                       void *stream);

/* The CP-ALS row passes of one mode on caller data, for precision tests of
 * the tensor-core arithmetic (Sec. II-A5's update; the splitting is stated in
 * the library's design notes).  Device pointers: M (I x R FP32, row-major),
 * V (R x R FP64, symmetric positive definite).  Runs the library's kernels:
 * W = V^{-1} by the FP64 Cholesky (one block per column) with W's BF16 digit
 * stack, Z = M W on the tensor cores (Z: I x R FP32), lambda = column 2-norms
 * of Z (R doubles), Y = Z / lambda (I x R FP32) and, for R = 16 or 32,
 * G = Y^T Y on the tensor cores from the stored Y (R x R FP64; untouched for
 * R = 64).  R must be 16, 32 or 64 and I >= 1 (else SPM_ERR_UNSUPPORTED /
 * SPM_ERR_INVALID_ARG); V not positive definite gives SPM_ERR_NUMERIC.
 * Allocates and frees its own scratch; synchronises `stream`. */
spm_status spm_selftest_tc_rowpass(int R, int64_t I, const float *M, const double *V,
                                   float *Z, float *Y, double *G, double *lambda,
                                   void *stream);

/* Fault injection on the host: the k-th device allocation made for a plan
 * from now on (k = 0: the next one) fails as if cudaMalloc had run out of
 * memory; k < 0 disables.  One-shot.  For tests of the error paths. */
void spm_inject_alloc_failure(int k);

/* Synchronise `stream` and return the plan's sticky device-side error
 * (SPM_OK, SPM_ERR_NUMERIC or SPM_ERR_TIMEOUT), then clear it. */
spm_status spmttkrp_plan_status(spmttkrp_plan_t plan, void *stream);

/* ---- misc ------------------------------------------------------------------ */

/* Static, never-NULL description of a status code. */
const char *spm_status_string(spm_status s);

/* Number of SMs of the current device (the default kappa), or -1. */
int spm_device_sm_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SPMTTKRP_H_ */
