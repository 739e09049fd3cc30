// mttkrp_kernel.cuh -- the sm_103a spMTTKRP kernel for one output mode.
//
// What it computes (Eq. 1, Sec. II-A6, Algorithm 2): for the mode-d copy,
//   M_d(c_d, r) = sum over nonzeros of val * prod_{w != d} Y_w(c_w, r).
//
// How (GB300 design, not the paper's block layout):
//  * One thread block per partition B_{d,z} (Algorithm 1's parallel loop),
//    1024 threads as in the paper's R x P = 32 x 32 block.  The partition is
//    cut by the plan into NU contiguous work units; the block's 32 warps take
//    units from a shared-memory counter, so a warp that drew cheap units
//    takes more (dynamic balance inside the block, fixed merge order).
//  * A warp streams its unit of the copy through a 3-stage ring of small
//    shared-memory tiles filled by 1-D bulk copies (cp.async.bulk on the TMA
//    engine, completion on an mbarrier).  Tiles are small so that most of
//    the SM's unified L1/shared array stays L1 cache for factor rows.
//  * A warp works on G consecutive nonzeros per step: each "slot" of LPN
//    lanes takes one nonzero, each lane VEC ranks per 16-byte load, so a
//    factor row is fetched as whole 128-byte lines.  U steps of records and
//    gathers are issued before any of them is used, to keep loads in flight.
//  * A tile whose first and last records are on the current output row lies
//    entirely on it (rows are sorted), and is accumulated with no per-step
//    row bookkeeping -- the common case on heavy rows.  Otherwise each step
//    checks its rows with a warp vote; on a row change the slots' sums are
//    combined with a segmented shuffle scan and finished rows are stored
//    once.  Partial rows never round-trip through global memory (the paper's
//    point about intermediate values, Sec. I).
//  * Rows cut by a unit boundary are merged by the block with a segmented
//    scan over the units' boundary partials in shared memory (the paper's
//    Local_Update); rows cut by a partition boundary (equal-nnz or balanced
//    policies) leave one partial per block in a small workspace that a fix-up
//    kernel adds in partition order (the paper's Global_Update, made
//    deterministic).
//  * Rows with no nonzero are zeroed by a separate pass over a plan-time
//    bitmap of non-empty rows.
#pragma once

#include <type_traits>

#include "plan.cuh"

namespace spm {

#ifndef SPM_L2_HINTS
#define SPM_L2_HINTS 0  // 1: records evict-first, factor rows evict-last in L2
#endif
#ifndef SPM_MT_WARPS
#define SPM_MT_WARPS 32
#endif
constexpr int MT_WARPS = SPM_MT_WARPS;
constexpr int MT_THREADS = MT_WARPS * 32;
#ifndef SPM_MT_STAGES
#define SPM_MT_STAGES 3
#endif
#ifndef SPM_MT_TILE
#define SPM_MT_TILE 64
#endif
constexpr int MT_STAGES = SPM_MT_STAGES;
constexpr int MT_TILE_RECS = SPM_MT_TILE;  // 16-byte records per stage tile (per warp);
                                           // a tile of 32-byte records holds half as many

struct MttkrpArgs {
  const int4* rec;        // copy records (lean copy: the mode-0 copy's)
  const int32_t* src;     // lean copy: position in the mode-0 copy of each copy position
  int fmode;              // lean copy: the output mode (its index is word fmode of a record)
  const int64_t* woff;    // work-unit offsets [kappa * nu + 1]
  const void* fac[SPM_MAX_MODES - 1];  // input factors in record order
  float* out;             // I_d x R
  float* cta_part;        // [kappa][2][R] boundary partials
  int* cta_meta;          // [kappa][4] (first row, last row, flags, 0)
  int* err;               // sticky device error flags
  const int* guard;       // if non-null and non-zero when the block starts, the block
                          // writes no output (a failed input check of the same call)
  uint32_t wait_limit;    // polls of a record-copy wait before it gives up:
                          // 0 = the default bound, ~0u = none at all (failure tests)
  int64_t nnz;
  int64_t I;              // rows of the output
  int R;                  // rank (runtime; equals the template rank when exact)
  int nin;                // number of input modes (N - 1)
  int nu;                 // work units per partition
};

// cta_meta flags
enum : int {
  META_PART0 = 1,        // cta_part[z][0] holds the first row's partial
  META_PART1 = 2,        // cta_part[z][1] holds the last row's partial
  META_SHARED_PREV = 4,  // first row continues from the previous partition
  META_SHARED_NEXT = 8,  // last row continues into the next partition
  META_EMPTY = 16,
};

#ifndef SPM_MT_F32X2
#define SPM_MT_F32X2 1  // 1: packed FP32-pair arithmetic in the full-step path
#endif
#ifndef SPM_MT_PAIRS
#define SPM_MT_PAIRS 1  // 1: FP32 rows and accumulators kept as FP32 pairs through the full-step path
#endif
#ifndef SPM_MT_PAIRS_BF16
#define SPM_MT_PAIRS_BF16 1  // 1: the same for BF16 factors (raw words widened to FP32 pairs)
#endif
#ifndef SPM_MT_U16
#define SPM_MT_U16 1  // gather batch when a step's rows take 16 registers per lane
#endif
#ifndef SPM_MT_REUSE
#define SPM_MT_REUSE 0  // 1: a slot keeps its first input mode's row and skips a repeated gather
#endif
// Shared memory of one block: per-warp rings of record tiles and their
// barriers, and two boundary partials (+ row ids) per work unit.  A stage
// tile has the same bytes for either record size; the factor type does not
// enter.
inline size_t mttkrp_smem_bytes(int R, int RI, int nu, int fsize) {
  (void)RI;
  (void)fsize;
  return (size_t)MT_WARPS * MT_STAGES * MT_TILE_RECS * 16 +
         (size_t)MT_WARPS * MT_STAGES * sizeof(uint64_t) + (size_t)2 * nu * R * sizeof(float) +
         (size_t)2 * nu * sizeof(int);
}

// Raw 32-bit words of one lane's slice of a factor row, and their conversion.
template <typename FT, int VEC>
struct Slice;

template <>
struct Slice<float, 4> {
  static constexpr int RAWN = 4;
  static __device__ __forceinline__ void load(const void* base, int64_t row, int R, int r0,
                                              uint32_t* raw) {
#if SPM_L2_HINTS
    const uint4 x = ld_nc_v4_hint(static_cast<const float*>(base) + row * R + r0, l2_policy_evict_last());
#else
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(static_cast<const float*>(base) +
                                                         row * R + r0));
#endif
    raw[0] = x.x; raw[1] = x.y; raw[2] = x.z; raw[3] = x.w;
  }
  static __device__ __forceinline__ void cvt(const uint32_t* raw, float* f) {
#pragma unroll
    for (int i = 0; i < 4; ++i) f[i] = __uint_as_float(raw[i]);
  }
};

template <>
struct Slice<__nv_bfloat16, 8> {
  static constexpr int RAWN = 4;
  static __device__ __forceinline__ void load(const void* base, int64_t row, int R, int r0,
                                              uint32_t* raw) {
#if SPM_L2_HINTS
    const uint4 x = ld_nc_v4_hint(static_cast<const __nv_bfloat16*>(base) + row * R + r0,
                                  l2_policy_evict_last());
#else
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(
        static_cast<const __nv_bfloat16*>(base) + row * R + r0));
#endif
    raw[0] = x.x; raw[1] = x.y; raw[2] = x.z; raw[3] = x.w;
  }
  static __device__ __forceinline__ void cvt(const uint32_t* raw, float* f) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[2 * i] = __uint_as_float(raw[i] << 16);
      f[2 * i + 1] = __uint_as_float(raw[i] & 0xFFFF0000u);
    }
  }
};

// BF16 rows of R <= 32 in 3-mode tensors: 8-byte loads (4 values per lane),
// so that a warp step holds as many nonzeros as the FP32 layout of the same
// rank (measured faster for 3 modes, slower for 5).
template <>
struct Slice<__nv_bfloat16, 4> {
  static constexpr int RAWN = 2;
  static __device__ __forceinline__ void load(const void* base, int64_t row, int R, int r0,
                                              uint32_t* raw) {
    const uint2 x = __ldg(reinterpret_cast<const uint2*>(
        static_cast<const __nv_bfloat16*>(base) + row * R + r0));
    raw[0] = x.x; raw[1] = x.y;
  }
  static __device__ __forceinline__ void cvt(const uint32_t* raw, float* f) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      f[2 * i] = __uint_as_float(raw[i] << 16);
      f[2 * i + 1] = __uint_as_float(raw[i] & 0xFFFF0000u);
    }
  }
};

template <>
struct Slice<float, 1> {
  static constexpr int RAWN = 1;
  static __device__ __forceinline__ void load(const void* base, int64_t row, int R, int r0,
                                              uint32_t* raw) {
    raw[0] = r0 < R ? __float_as_uint(__ldg(static_cast<const float*>(base) + row * R + r0)) : 0u;
  }
  static __device__ __forceinline__ void cvt(const uint32_t* raw, float* f) {
    f[0] = __uint_as_float(raw[0]);
  }
};

template <>
struct Slice<__nv_bfloat16, 1> {
  static constexpr int RAWN = 1;
  static __device__ __forceinline__ void load(const void* base, int64_t row, int R, int r0,
                                              uint32_t* raw) {
    raw[0] = r0 < R ? (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(base) + row * R + r0)
                    : 0u;
  }
  static __device__ __forceinline__ void cvt(const uint32_t* raw, float* f) {
    f[0] = __uint_as_float(raw[0] << 16);
  }
};

// Store one lane's VEC consecutive FP32 values (r0 .. r0+VEC-1) of a row.
template <int VEC>
__device__ __forceinline__ void store_vec(float* row_ptr, int R, int r0, const float* v) {
  if constexpr (VEC % 4 == 0) {
#pragma unroll
    for (int q = 0; q < VEC / 4; ++q)
      *reinterpret_cast<float4*>(row_ptr + r0 + 4 * q) =
          make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e)
      if (r0 + e < R) row_ptr[r0 + e] = v[e];
  }
}

// NIN > 0: exactly NIN input modes.  NIN == 0: runtime a.nin (six or more
// modes); the first two input modes are batched, further ones are fetched
// when the step is computed.
//
// mttkrp_partition processes partition z of one mode copy with the whole
// thread block (every thread must call it); it is the body of the
// single-tensor kernel and of the batched persistent kernel.
// Words of a mode-0 record rearranged into the mode-d order: word d moves to
// the front, words 0..d-1 one place back (the other modes stay ascending).
template <int W>
__device__ __forceinline__ void rotate_to_front(int (&w)[W], int d) {
  int cd = w[0];
#pragma unroll
  for (int j = 1; j < W; ++j)
    if (j == d) cd = w[j];
#pragma unroll
  for (int j = W - 1; j >= 1; --j)
    if (j <= d) w[j] = w[j - 1];
  w[0] = cd;
}

template <int RI, int NIN, typename FT, int VEC, int LPN, int CPL, bool LEAN = false>
__device__ __forceinline__ void mttkrp_partition(const MttkrpArgs& a, const int z) {
  using S = Slice<FT, VEC>;
  constexpr int RAWN = S::RAWN;
  constexpr int G = 32 / LPN;
  constexpr int W = 4 * RI;
  constexpr int NPIPE = NIN > 0 ? NIN : 2;  // batched input modes
  constexpr int TILE = MT_TILE_RECS / RI;
  constexpr int tile_bytes = TILE * 16 * RI;
  static_assert(TILE % G == 0, "tile geometry");
  constexpr int PIPE_REGS = CPL * RAWN * NPIPE;
#ifdef SPM_MT_BATCH
  constexpr int U = NIN == 0 ? 1 : SPM_MT_BATCH;
#else
  // 8-byte lanes (BF16, R <= 32) convert to as many floats as 16-byte FP32
  // lanes: the same two-step batch keeps them within 64 registers
  constexpr int U = NIN == 0 ? 1
                  : (VEC * (int)sizeof(FT) == 8 ? 2
                     : (PIPE_REGS <= 4 ? 4 : (PIPE_REGS <= 8 ? 2 : SPM_MT_U16)));
#endif
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int next_unit;
  __shared__ int aborted;  // some warp gave up on a record copy: no merge, no stores

  const int R = a.R;
  const int NU = a.nu;
  const int nin = NIN > 0 ? NIN : a.nin;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / LPN, sub = lane % LPN;
  const int64_t* uoff = a.woff + (int64_t)z * NU;
  const int64_t K0 = uoff[0], K1 = uoff[NU];

  unsigned char* stages = smem + (size_t)warp * MT_STAGES * tile_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)MT_WARPS * MT_STAGES * tile_bytes) +
                   warp * MT_STAGES;
  float* part = reinterpret_cast<float*>(smem + (size_t)MT_WARPS * MT_STAGES * tile_bytes +
                                         (size_t)MT_WARPS * MT_STAGES * sizeof(uint64_t));
  int* prow = reinterpret_cast<int*>(part + (size_t)2 * NU * R);  // [2 * NU]

  auto row_at = [&](int64_t k) -> int {
    if constexpr (LEAN)
      return __ldg(reinterpret_cast<const int*>(a.rec) + (int64_t)__ldg(a.src + k) * (4 * RI) +
                   a.fmode);
    else
      return __ldg(&a.rec[k * RI].x);
  };
  auto rank0 = [&](int c) -> int { return (c * LPN + sub) * VEC; };
  // Vector path with the rank fixed at compile time (R == VEC * LPN * CPL):
  // full steps are processed without per-step predication, gathers address
  // rows with a constant stride from per-lane base pointers.
  constexpr int LANE_BYTES = VEC * (int)sizeof(FT);
  constexpr bool FAST = NIN > 0 && (LANE_BYTES == 16 || LANE_BYTES == 8);
  using LdT = typename std::conditional<LANE_BYTES == 16, uint4, uint2>::type;
  // FP32 factors: a lane's 16-byte slice is loaded as two FP32 pairs and the
  // running sums are kept as pairs, so the packed arithmetic needs no moves.
  // BF16 factors: each raw word (two BF16 ranks) widens to one FP32 pair.
  constexpr bool P32 = std::is_same<FT, float>::value;
  constexpr bool PAIRS = FAST && ((P32 && SPM_MT_PAIRS && LANE_BYTES == 16) ||
                                  (!P32 && SPM_MT_PAIRS_BF16));
  constexpr int RT = VEC * LPN * CPL;
  constexpr int NINF = NIN > 0 ? NIN : 1;
  const LdT* facb[NINF];
#pragma unroll
  for (int m = 0; m < NINF; ++m)
    facb[m] = reinterpret_cast<const LdT*>(static_cast<const FT*>(a.fac[m]) + sub * VEC);

  if (lane == 0) {
#pragma unroll
    for (int st = 0; st < MT_STAGES; ++st) mbar_init(&bars[st], 1);
    fence_mbar_init();
  }
  if (threadIdx.x == 0) {
    next_unit = MT_WARPS;
    aborted = (a.guard && *(volatile const int*)a.guard) ? 1 : 0;
  }
  __syncthreads();
  const uint32_t wait_polls = a.wait_limit == 0u ? (1u << 24) : (a.wait_limit == ~0u ? 0u : a.wait_limit);

  int seq_issued = 0;    // ring sequence: tiles issued by this warp so far
  bool timeout = false;
  const bool skip = aborted != 0;  // guard set: no unit is taken, no copy issued

  auto slot_reduce = [&](float (&x)[CPL][VEC]) {
#pragma unroll
    for (int o = LPN; o < 32; o <<= 1)
#pragma unroll
      for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int e = 0; e < VEC; ++e) x[c][e] += __shfl_xor_sync(SPM_FULL_MASK, x[c][e], o);
  };

  for (int u = warp; u < NU && !timeout && !skip;) {
    const int64_t k0 = uoff[u], k1 = uoff[u + 1];
    const int lenw = (int)(k1 - k0);
    float* pf = part + (size_t)(2 * u) * R;
    float* pl = pf + R;
    if (lenw > 0) {
      const int ntiles = (lenw + TILE - 1) / TILE;
      const int seq0 = seq_issued;  // ring sequence number of this unit's tile 0
      auto issue = [&](int t) {     // lane 0 only
        const int64_t kb = k0 + (int64_t)t * TILE;
        const int64_t cnt = (k1 - kb) < TILE ? (k1 - kb) : TILE;
        const int q = seq0 + t;
        uint64_t* bar = &bars[q % MT_STAGES];
        if constexpr (LEAN) {
          // the tile's positions into the mode-0 copy, from the 16-byte
          // boundary at or below kb (the position array is padded at its end)
          const int64_t al = kb & ~(int64_t)3;
          const uint32_t lbytes = (uint32_t)((((kb - al) + cnt) * 4 + 15) & ~(int64_t)15);
          mbar_arrive_expect_tx(bar, lbytes);
          bulk_g2s(stages + (q % MT_STAGES) * tile_bytes, a.src + al, lbytes, bar);
          return;
        }
        const uint32_t bytes = (uint32_t)(cnt * 16 * RI);
        mbar_arrive_expect_tx(bar, bytes);
#if SPM_L2_HINTS
        bulk_g2s_hint(stages + (q % MT_STAGES) * tile_bytes, a.rec + kb * RI, bytes, bar,
                      l2_policy_evict_first());
#else
        bulk_g2s(stages + (q % MT_STAGES) * tile_bytes, a.rec + kb * RI, bytes, bar);
#endif
      };
      int issued = ntiles < MT_STAGES ? ntiles : MT_STAGES;
      if (lane == 0)
        for (int t = 0; t < issued; ++t) issue(t);

      const int first_row = row_at(k0);
      int cur = first_row;
      float acc[CPL][VEC];
#pragma unroll
      for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[c][e] = 0.f;

      // finished row from this slot's lanes; the unit's first row goes to the
      // block's boundary partials
      auto put_row = [&](int row, const float (&x)[CPL][VEC]) {
        float* dst = row == first_row ? pf : a.out + (int64_t)row * R;
#pragma unroll
        for (int c = 0; c < CPL; ++c) store_vec<VEC>(dst, R, rank0(c), x[c]);
      };

      // Fold one step's contributions v (rows `row`, empty slots already on
      // the last row) into the running row state.
      auto step_rows = [&](int row, float (&v)[CPL][VEC]) {
        if (__all_sync(SPM_FULL_MASK, row == cur)) {
#pragma unroll
          for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[c][e] += v[c][e];
          return;
        }
        // Row change inside this step: carry = total of `cur` so far.
        slot_reduce(acc);
        const int next_row = __shfl_down_sync(SPM_FULL_MASK, row, LPN);
        const bool tail = (slot == G - 1) || next_row != row;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {  // segmented inclusive scan over slots
          const int ru = __shfl_up_sync(SPM_FULL_MASK, row, o * LPN);
#pragma unroll
          for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
              const float t = __shfl_up_sync(SPM_FULL_MASK, v[c][e], o * LPN);
              if (slot >= o && ru == row) v[c][e] += t;
            }
        }
        if (row == cur) {
#pragma unroll
          for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < VEC; ++e) v[c][e] += acc[c][e];
        }
        const int row0 = __shfl_sync(SPM_FULL_MASK, row, 0);
        const int rowl = __shfl_sync(SPM_FULL_MASK, row, 31);
        if (row0 != cur && slot == 0) put_row(cur, acc);  // cur ended with the last step
        if (tail && row != rowl) put_row(row, v);
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc[c][e] = (slot == G - 1) ? v[c][e] : 0.f;
        cur = rowl;
      };

      for (int t = 0; t < ntiles; ++t) {
        if (t > 0) {
          __syncwarp();  // every lane is done with tile t-1: refill its stage
          if (issued < ntiles) {
            if (lane == 0) {
              fence_proxy_async_smem();
              issue(issued);
            }
            ++issued;
          }
        }
        {
          const int q = seq0 + t;
          const bool ok = mbar_wait_bounded(&bars[q % MT_STAGES], (uint32_t)((q / MT_STAGES) & 1),
                                            wait_polls);
          timeout = __any_sync(SPM_FULL_MASK, !ok);
        }
        if (timeout) {
          // let every copy this warp started (the one waited on included)
          // land before giving up, then make the whole block skip its
          // merge and stores: the units this warp held have no partials
          for (int q = seq0 + t; q < seq0 + issued; ++q)
            (void)mbar_wait_bounded(&bars[q % MT_STAGES], (uint32_t)((q / MT_STAGES) & 1), 1u << 20);
          if (lane == 0) {
            atomicOr(a.err, DEV_ERR_TIMEOUT);
            atomicExch(&aborted, 1);
          }
          break;
        }
        const unsigned char* stage_t = stages + ((seq0 + t) % MT_STAGES) * tile_bytes;
        const int4* recs = reinterpret_cast<const int4*>(stage_t);
        // lean copy: the stage holds positions into the mode-0 copy
        const int* srcs = reinterpret_cast<const int*>(stage_t) +
                          (LEAN ? (int)((k0 + (int64_t)t * TILE) & 3) : 0);
        auto load_rec = [&](int pos, int (&wv)[W]) {
          if constexpr (LEAN) {
            const int4* r = a.rec + (int64_t)srcs[pos] * RI;
#pragma unroll
            for (int qq = 0; qq < RI; ++qq) {
              const int4 v4 = __ldg(r + qq);
              wv[4 * qq] = v4.x; wv[4 * qq + 1] = v4.y; wv[4 * qq + 2] = v4.z; wv[4 * qq + 3] = v4.w;
            }
            rotate_to_front<W>(wv, a.fmode);
          } else {
#pragma unroll
            for (int qq = 0; qq < RI; ++qq) {
              const int4 v4 = recs[pos * RI + qq];
              wv[4 * qq] = v4.x; wv[4 * qq + 1] = v4.y; wv[4 * qq + 2] = v4.z; wv[4 * qq + 3] = v4.w;
            }
          }
        };
        auto tile_row = [&](int pos) -> int {
          if constexpr (LEAN)
            return __ldg(reinterpret_cast<const int*>(a.rec) + (int64_t)srcs[pos] * (4 * RI) +
                         a.fmode);
          else
            return recs[pos * RI].x;
        };
        const int n = (lenw - t * TILE) < TILE ? (lenw - t * TILE) : TILE;
        const int nst = (n + G - 1) / G;
        const bool pure = tile_row(0) == cur && tile_row(n - 1) == cur;
        int j_fast = 0;
        if constexpr (PAIRS) {
          // Full steps, U at a time.  Unless the tile lies on the current
          // row, each batch of U steps takes one vote, and a batch that
          // leaves the row passes its steps to step_rows.  Same roundings as
          // the scalar path: (val * y_a) * y_b ... then one fused multiply-add
          // into the running sum on the row, a product then an add in
          // step_rows.
          constexpr int H = VEC / 2;
          const int nb = ((n / G) / U) * U;
          uint64_t ap[CPL][H];
#pragma unroll
          for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < H; ++e) ap[c][e] = f2_pack(acc[c][2 * e], acc[c][2 * e + 1]);
          // FP32: the loaded pairs; BF16: raw words, widened when used
          using YT = typename std::conditional<P32, uint64_t, uint32_t>::type;
          auto pair = [](YT x) -> uint64_t {
            if constexpr (P32) return x;
            else return f2_pack(__uint_as_float((uint32_t)x << 16), __uint_as_float((uint32_t)x & 0xFFFF0000u));
          };
          for (int j = 0; j < nb; j += U) {
            int w[U][W];
            YT y[U][NINF][CPL][H];
#pragma unroll
            for (int uu = 0; uu < U; ++uu) load_rec((j + uu) * G + slot, w[uu]);
#pragma unroll
            for (int uu = 0; uu < U; ++uu)
#pragma unroll
              for (int m = 0; m < NINF; ++m)
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                  const LdT* src =
                      facb[m] + (size_t)(uint32_t)w[uu][1 + m] * (RT * sizeof(FT) / sizeof(LdT)) + c * LPN;
                  if constexpr (P32) {
                    const ulonglong2 x = ld_nc_v2_u64(src);
                    y[uu][m][c][0] = x.x;
                    y[uu][m][c][1] = x.y;
                  } else if constexpr (LANE_BYTES == 16) {
                    const uint4 x = __ldg(src);
                    y[uu][m][c][0] = x.x; y[uu][m][c][1] = x.y;
                    y[uu][m][c][2] = x.z; y[uu][m][c][3] = x.w;
                  } else {
                    const uint2 x = __ldg(src);
                    y[uu][m][c][0] = x.x; y[uu][m][c][1] = x.y;
                  }
                }
            bool same = pure;
            if (!pure) {
              bool ok = true;
#pragma unroll
              for (int uu = 0; uu < U; ++uu) ok = ok && w[uu][0] == cur;
              same = __all_sync(SPM_FULL_MASK, ok);
            }
            if (same) {
#pragma unroll
              for (int uu = 0; uu < U; ++uu) {
                const float val = __int_as_float(w[uu][NINF + 1]);
                const uint64_t vv = f2_pack(val, val);
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                  for (int e = 0; e < H; ++e) {
                    uint64_t g = f2_mul(vv, pair(y[uu][0][c][e]));
#pragma unroll
                    for (int m = 1; m + 1 < NINF; ++m) g = f2_mul(g, pair(y[uu][m][c][e]));
                    ap[c][e] = NINF > 1 ? f2_fma(g, pair(y[uu][NINF - 1][c][e]), ap[c][e])
                                        : f2_add(ap[c][e], g);
                  }
              }
            } else {
#pragma unroll
              for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < H; ++e) f2_unpack(ap[c][e], acc[c][2 * e], acc[c][2 * e + 1]);
#pragma unroll
              for (int uu = 0; uu < U; ++uu) {
                const float val = __int_as_float(w[uu][NINF + 1]);
                const uint64_t vv = f2_pack(val, val);
                float v[CPL][VEC];
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                  for (int e = 0; e < H; ++e) {
                    uint64_t g = f2_mul(vv, pair(y[uu][0][c][e]));
#pragma unroll
                    for (int m = 1; m + 1 < NINF; ++m) g = f2_mul(g, pair(y[uu][m][c][e]));
                    if (NINF > 1) g = f2_mul(g, pair(y[uu][NINF - 1][c][e]));
                    f2_unpack(g, v[c][2 * e], v[c][2 * e + 1]);
                  }
                step_rows(w[uu][0], v);
              }
#pragma unroll
              for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < H; ++e) ap[c][e] = f2_pack(acc[c][2 * e], acc[c][2 * e + 1]);
            }
          }
#pragma unroll
          for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < H; ++e) f2_unpack(ap[c][e], acc[c][2 * e], acc[c][2 * e + 1]);
          j_fast = nb;
        } else if constexpr (FAST) {
          // full steps (a record in every slot), U at a time
          const int nb = ((n / G) / U) * U;
#if SPM_MT_REUSE
          int last0 = -1;               // index of the first input mode's row held in y0prev
          uint32_t y0prev[CPL][RAWN];
#pragma unroll
          for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int i = 0; i < RAWN; ++i) y0prev[c][i] = 0u;
#endif
#if SPM_L2_HINTS
          const uint64_t pol_rows = l2_policy_evict_last();
#endif
          for (int j = 0; j < nb; j += U) {
            int w[U][W];
            uint32_t y[U][NINF][CPL][RAWN];
#pragma unroll
            for (int uu = 0; uu < U; ++uu) load_rec((j + uu) * G + slot, w[uu]);
#if SPM_MT_REUSE
            bool fresh0[U];
            {
              int prev = last0;
#pragma unroll
              for (int uu = 0; uu < U; ++uu) {
                fresh0[uu] = w[uu][1] != prev;
                prev = w[uu][1];
              }
            }
#endif
#pragma unroll
            for (int uu = 0; uu < U; ++uu)
#pragma unroll
              for (int m = 0; m < NINF; ++m)
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
#if SPM_MT_REUSE
                  if (m == 0 && !fresh0[uu]) continue;  // taken from the previous step below
#endif
                  const LdT* src = facb[m] +
                                   (size_t)(uint32_t)w[uu][1 + m] * (RT * sizeof(FT) / sizeof(LdT)) +
                                   c * LPN;
                  if constexpr (LANE_BYTES == 16) {
#if SPM_L2_HINTS
                    const uint4 x = ld_nc_v4_pol(src, pol_rows);
#else
                    const uint4 x = __ldg(src);
#endif
                    y[uu][m][c][0] = x.x; y[uu][m][c][1] = x.y;
                    y[uu][m][c][2] = x.z; y[uu][m][c][3] = x.w;
                  } else {
                    const uint2 x = __ldg(src);
                    y[uu][m][c][0] = x.x; y[uu][m][c][1] = x.y;
                  }
                }
#if SPM_MT_REUSE
#pragma unroll
            for (int uu = 0; uu < U; ++uu)
#pragma unroll
              for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int i = 0; i < RAWN; ++i) {
                  if (!fresh0[uu]) y[uu][0][c][i] = uu == 0 ? y0prev[c][i] : y[uu - 1][0][c][i];
                  if (uu == U - 1) y0prev[c][i] = y[uu][0][c][i];
                }
            last0 = w[U - 1][1];
#endif
            bool same = pure;
            if (!pure) {
              bool ok = true;
#pragma unroll
              for (int uu = 0; uu < U; ++uu) ok = ok && w[uu][0] == cur;
              same = __all_sync(SPM_FULL_MASK, ok);
            }
#pragma unroll
            for (int uu = 0; uu < U; ++uu) {
              const float val = __int_as_float(w[uu][NINF + 1]);
              float v[CPL][VEC];
#pragma unroll
              for (int c = 0; c < CPL; ++c) {
                float f[VEC], g[VEC];
                S::cvt(y[uu][0][c], f);
#if SPM_MT_F32X2
                // the same roundings as the scalar code, two ranks per instruction
                const uint64_t vv = f2_pack(val, val);
                uint64_t g2[VEC / 2];
#pragma unroll
                for (int e = 0; e < VEC / 2; ++e) g2[e] = f2_mul(vv, f2_pack(f[2 * e], f[2 * e + 1]));
#pragma unroll
                for (int m = 1; m + 1 < NINF; ++m) {
                  S::cvt(y[uu][m][c], f);
#pragma unroll
                  for (int e = 0; e < VEC / 2; ++e) g2[e] = f2_mul(g2[e], f2_pack(f[2 * e], f[2 * e + 1]));
                }
                if (NINF > 1) S::cvt(y[uu][NINF - 1][c], f);
#pragma unroll
                for (int e = 0; e < VEC / 2; ++e) {
                  const uint64_t fl = f2_pack(f[2 * e], f[2 * e + 1]);
                  if (same) {
                    uint64_t a2 = f2_pack(acc[c][2 * e], acc[c][2 * e + 1]);
                    a2 = NINF > 1 ? f2_fma(g2[e], fl, a2) : f2_mul(g2[e], f2_pack(1.f, 1.f));
                    if (NINF > 1) f2_unpack(a2, acc[c][2 * e], acc[c][2 * e + 1]);
                    else {
                      float g0, g1;
                      f2_unpack(g2[e], g0, g1);
                      acc[c][2 * e] += g0;
                      acc[c][2 * e + 1] += g1;
                    }
                  } else {
                    const uint64_t p2 = NINF > 1 ? f2_mul(g2[e], fl) : g2[e];
                    f2_unpack(p2, v[c][2 * e], v[c][2 * e + 1]);
                  }
                }
                (void)g;
#else
#pragma unroll
                for (int e = 0; e < VEC; ++e) g[e] = val * f[e];
#pragma unroll
                for (int m = 1; m + 1 < NINF; ++m) {
                  S::cvt(y[uu][m][c], f);
#pragma unroll
                  for (int e = 0; e < VEC; ++e) g[e] *= f[e];
                }
                if (NINF > 1) S::cvt(y[uu][NINF - 1][c], f);
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                  if (same) acc[c][e] = NINF > 1 ? fmaf(g[e], f[e], acc[c][e]) : acc[c][e] + g[e];
                  else v[c][e] = NINF > 1 ? g[e] * f[e] : g[e];
                }
#endif
              }
              if (!same) step_rows(w[uu][0], v);
            }
          }
          j_fast = nb;
        }
        for (int j = j_fast; j < nst; j += U) {
          int w[U][W];
          bool valid[U];
          uint32_t y[U][NPIPE][CPL][RAWN];
#pragma unroll
          for (int uu = 0; uu < U; ++uu) {
            const int pos = (j + uu) * G + slot;
            valid[uu] = (j + uu) < nst && pos < n;
#pragma unroll
            for (int qq = 0; qq < W; ++qq) w[uu][qq] = 0;
            if (valid[uu]) load_rec(pos, w[uu]);
          }
#pragma unroll
          for (int uu = 0; uu < U; ++uu)
#pragma unroll
            for (int m = 0; m < NPIPE; ++m) {
#pragma unroll
              for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int i = 0; i < RAWN; ++i) y[uu][m][c][i] = 0u;
              if (valid[uu] && m < nin) {
#pragma unroll
                for (int c = 0; c < CPL; ++c) S::load(a.fac[m], w[uu][1 + m], R, rank0(c), y[uu][m][c]);
              }
            }
#pragma unroll
          for (int uu = 0; uu < U; ++uu) {
            if (j + uu >= nst) break;
            float v[CPL][VEC];
            float val = 0.f;
            if (NIN > 0) {
              val = __int_as_float(w[uu][NIN > 0 ? NIN + 1 : 1]);
            } else {
#pragma unroll
              for (int qq = 1; qq < W; ++qq)
                if (qq == nin + 1) val = __int_as_float(w[uu][qq]);
            }
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
              float f[VEC];
              S::cvt(y[uu][0][c], f);
#pragma unroll
              for (int e = 0; e < VEC; ++e) v[c][e] = val * f[e];
#pragma unroll
              for (int m = 1; m < NPIPE; ++m)
                if (m < nin) {
                  S::cvt(y[uu][m][c], f);
#pragma unroll
                  for (int e = 0; e < VEC; ++e) v[c][e] *= f[e];
                }
              if (NIN == 0) {
                for (int m = NPIPE; m < nin; ++m) {
                  int idx = 0;
#pragma unroll
                  for (int qq = 1; qq < W; ++qq)
                    if (qq == 1 + m) idx = w[uu][qq];
                  uint32_t raw[RAWN];
                  if (valid[uu]) S::load(a.fac[m], idx, R, rank0(c), raw);
                  else raw[0] = 0u;
                  S::cvt(raw, f);
#pragma unroll
                  for (int e = 0; e < VEC; ++e) v[c][e] *= f[e];
                }
              }
            }
            if (pure) {
#pragma unroll
              for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < VEC; ++e) acc[c][e] += v[c][e];
            } else {
              int row = w[uu][0];
              if ((j + uu + 1) * G > n) {  // ragged step: empty slots join the last row
                const int nvalid = n - (j + uu) * G;
                const int lastv = __shfl_sync(SPM_FULL_MASK, row, (nvalid - 1) * LPN);
                if (!valid[uu]) row = lastv;
              }
              step_rows(row, v);
            }
          }
        }
      }
      // the unit's last row (== cur): its partial goes to the block merge
      slot_reduce(acc);
      const bool distinct_last = cur != first_row;
      if (slot == 0) {
        float* dst = distinct_last ? pl : pf;
#pragma unroll
        for (int c = 0; c < CPL; ++c) store_vec<VEC>(dst, R, rank0(c), acc[c]);
      }
      if (!distinct_last)
        for (int r = lane; r < R; r += 32) pl[r] = 0.f;
      if (lane == 0) {
        prow[2 * u] = first_row;
        prow[2 * u + 1] = distinct_last ? cur : -1;
      }
      seq_issued = seq0 + ntiles;
    } else {
      for (int r = lane; r < 2 * R; r += 32) pf[r] = 0.f;
      if (lane == 0) {
        prow[2 * u] = -1;
        prow[2 * u + 1] = -1;
      }
    }
    int nu_next = 0;
    if (lane == 0) nu_next = atomicAdd(&next_unit, 1);
    u = __shfl_sync(SPM_FULL_MASK, nu_next, 0);
  }
  if (lane == 0 && !timeout) {
#pragma unroll
    for (int st = 0; st < MT_STAGES; ++st) mbar_inval(&bars[st]);
  }
  __syncthreads();

  // ---- block merge of the unit-boundary partials ---------------------------
  // Entries e = 2u (first row of unit u) and 2u+1 (its distinct last row) in
  // copy order.  Missing entries take the row of the entry before them with a
  // zero value, so rows stay sorted and every run of equal rows is one group.
  // An inclusive segmented scan (Hillis-Steele, fixed order) leaves each
  // group's total on its last entry.
  int* meta = a.cta_meta + 4 * z;
  const int64_t len = K1 - K0;
  if (len == 0 || aborted) {
    if (threadIdx.x == 0) { meta[0] = -1; meta[1] = -1; meta[2] = META_EMPTY; meta[3] = 0; }
    return;
  }
  const int NE = 2 * NU;  // <= 256
  // rows of missing entries (value already zero): running maximum of the
  // entries so far, i.e. the row of the last real entry (-1 before any)
  if (warp == 0) {
    int m = -1;
    const int per = (NE + 31) / 32;
    const int e0 = lane * per;
    for (int e = e0; e < e0 + per && e < NE; ++e) m = max(m, prow[e]);
    int incl = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(SPM_FULL_MASK, incl, o);
      if (lane >= o) incl = max(incl, t);
    }
    int run = __shfl_up_sync(SPM_FULL_MASK, incl, 1);
    if (lane == 0) run = -1;
    for (int e = e0; e < e0 + per && e < NE; ++e) {
      run = max(run, prow[e]);
      prow[e] = run;
    }
  }
  __syncthreads();
  // inclusive segmented scan of the partials, rows as segment keys
  // NE * R <= 8192 for every rank (units per partition = clamp(4096/R, 16, 128))
  constexpr int MERGE_PER_THREAD = (8192 + MT_THREADS - 1) / MT_THREADS;
  for (int d = 1; d < NE; d <<= 1) {
    float tmp[MERGE_PER_THREAD];
    int cnt = 0;
    for (int x = threadIdx.x; x < NE * R && cnt < MERGE_PER_THREAD; x += MT_THREADS, ++cnt) {
      const int e = x / R;
      tmp[cnt] = (e >= d && prow[e - d] == prow[e]) ? part[x - d * R] : 0.f;
    }
    __syncthreads();
    cnt = 0;
    for (int x = threadIdx.x; x < NE * R && cnt < MERGE_PER_THREAD; x += MT_THREADS, ++cnt)
      part[x] += tmp[cnt];
    __syncthreads();
  }
  // each group's last entry holds the group total
  const int F = row_at(K0);
  const int L = row_at(K1 - 1);
  const bool shared_prev = K0 > 0 && row_at(K0 - 1) == F;
  const bool shared_next = K1 < a.nnz && row_at(K1) == L;
  float* part0 = a.cta_part + (int64_t)(2 * z) * R;
  float* part1 = part0 + R;
  for (int x = threadIdx.x; x < NE * R; x += MT_THREADS) {
    const int e = x / R, r = x % R;
    const int row = prow[e];
    if (row < 0 || (e + 1 < NE && prow[e + 1] == row)) continue;
    float* dst;
    if (row == F && shared_prev) dst = part0;
    else if (row == L && shared_next) dst = part1;
    else dst = a.out + (int64_t)row * R;
    dst[r] = part[x];
  }
  if (threadIdx.x == 0) {
    int flags = (shared_prev ? META_SHARED_PREV : 0) | (shared_next ? META_SHARED_NEXT : 0);
    if (shared_prev) flags |= META_PART0;
    if (shared_next && !(F == L && shared_prev)) flags |= META_PART1;
    meta[0] = F; meta[1] = L; meta[2] = flags; meta[3] = 0;
  }
}

// Partition fix-up for partition z, one warp (lane = its lane): if z holds
// the start of a row that continues into later partitions (its last-row
// partial), add the first-row partials of the following partitions in
// partition order and store the row.
__device__ __forceinline__ void mttkrp_fixup_body(const float* __restrict__ cta_part,
                                                  const int* __restrict__ cta_meta, int kappa,
                                                  int R, float* __restrict__ out, int z, int lane) {
  const int* m = cta_meta + 4 * z;
  if (!(m[2] & META_PART1)) return;
  const int row = m[1];
  float s[8];
  const float* p1 = cta_part + (int64_t)(2 * z + 1) * R;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int r = lane + 32 * j;
    s[j] = r < R ? p1[r] : 0.f;
  }
  // The partitions after z that continue `row`, in order; their metadata and
  // partials are loaded FQ at a time ahead of the (ordered) additions, so a
  // head row cut into many partitions does not pay one load latency each.
  constexpr int FQ = 4;
  bool more = true;
  for (int q0 = z + 1; q0 < kappa && more; q0 += FQ) {
    int4 mq[FQ];
    float pq[FQ][8];
#pragma unroll
    for (int k = 0; k < FQ; ++k) {
      const int q = q0 + k;
      mq[k] = q < kappa ? *reinterpret_cast<const int4*>(cta_meta + 4 * q) : make_int4(-1, -1, 0, 0);
      const float* p0 = cta_part + (int64_t)(2 * (q < kappa ? q : z)) * R;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int r = lane + 32 * j;
        pq[k][j] = r < R ? p0[r] : 0.f;
      }
    }
#pragma unroll
    for (int k = 0; k < FQ; ++k) {
      if (!more || q0 + k >= kappa) {
        more = false;
        continue;
      }
      const int fq = mq[k].z;
      if (fq & META_EMPTY) continue;
      if (mq[k].x != row) {
        more = false;
        continue;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int r = lane + 32 * j;
        if (r < R) s[j] += pq[k][j];
      }
      if (!(mq[k].y == row && (fq & META_SHARED_NEXT))) more = false;
    }
  }
  float* dst = out + (int64_t)row * R;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int r = lane + 32 * j;
    if (r < R) dst[r] = s[j];
  }
}

// Rows of an I x R output whose bit in `mask` is clear are zeroed, for the
// bitmap words [w0, w1) (word w covers rows 32w .. 32w+31), one word per
// thread stepping by wstep.  Full words cost one load; an empty row is
// cleared with 16-byte stores when R allows.
__device__ __forceinline__ void zero_empty_rows_body(const uint32_t* __restrict__ mask, int64_t I,
                                                     int R, float* __restrict__ out, int64_t w0,
                                                     int64_t w1, int64_t wstep) {
  for (int64_t w = w0; w < w1; w += wstep) {
    uint32_t clear = ~__ldg(&mask[w]);
    while (clear) {
      const int b = __ffs(clear) - 1;
      clear &= clear - 1;
      const int64_t row = w * 32 + b;
      if (row >= I) break;
      float* dst = out + row * R;
      if ((R & 3) == 0) {
        for (int c = 0; c < R; c += 4) *reinterpret_cast<float4*>(dst + c) = make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        for (int c = 0; c < R; ++c) dst[c] = 0.f;
      }
    }
  }
}

template <int RI, int NIN, typename FT, int VEC, int LPN, int CPL, bool LEAN = false>
__global__ void __launch_bounds__(MT_THREADS, 1) mttkrp_kernel(const MttkrpArgs a) {
  mttkrp_partition<RI, NIN, FT, VEC, LPN, CPL, LEAN>(a, blockIdx.x);
}

}  // namespace spm
