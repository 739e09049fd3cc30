// mttkrp_fibre.cuh -- spMTTKRP along one mode on a fibre-layout copy (3 modes).
//
// The copy is a stream of 8-byte entries: a header {c_a | 2^31, c_d} opens
// each fibre (a maximal run of nonzeros sharing (c_d, c_a)) and an entry
// {c_b, value} follows for each of its nonzeros: the first word is always
// the row to gather, its top bit choosing the factor.  Eq. 1 for mode d is then
//   M_d(c_d, :) += val * Y_b(c_b, :) .* Y_a(c_a, :)
// with Y_a(c_a) gathered once per fibre (at its header) and held in registers
// for the fibre's nonzeros.
//
// How (GB300 design):
//  * One thread block per partition; warp w of the block takes the
//    G = 32 * FB_VEC / R consecutive work units w*G .. w*G+G-1 of the
//    partition side by side, one per "slot" of R / FB_VEC lanes (FB_VEC = 4
//    ranks per lane: one 16-byte FP32 or 8-byte BF16 load per row).  A slot walks its unit's entries in
//    order, so fibre and row changes are the slot's own events: no segmented
//    scans across slots.
//  * Each entry costs exactly one row gather (Y_a at a header, Y_b at a
//    nonzero): about 1.4 rows per nonzero instead of 2.
//  * The warp streams its slots' entry ranges through a 3-stage ring of
//    shared-memory tiles filled by 1-D bulk copies (TMA engine) with
//    mbarrier completion; each slot's part of a stage is padded so that the
//    slots' 8-byte reads fall in different banks.  Waits are bounded: a
//    wait that gives up drains the warp's copies and the block stores
//    nothing (same protocol as the record kernel).
//  * A unit's first and last rows go to the block's boundary partials, rows
//    cut by partitions to the partition fix-up, exactly as for the record
//    layout (fixed summation order: repeated runs are bitwise identical).
#pragma once

#include <type_traits>

#include "mttkrp_kernel.cuh"

namespace spm {

struct FibreArgs {
  const int2* stream;        // entries of the mode copy
  const FibreUnit* units;    // [kappa * nu] work units
  const int64_t* woff;       // [kappa * nu + 1] work-unit nonzero offsets
  const void* fac_a;         // factor of the first input mode (gathered at headers)
  const void* fac_b;         // factor of the second input mode (gathered per nonzero)
  float* out;                // I_d x R
  float* cta_part;           // [kappa][2][R] boundary partials
  int* cta_meta;             // [kappa][4]
  int* err;                  // sticky device error flags
  uint32_t wait_limit;       // as MttkrpArgs::wait_limit
  int64_t nnz;
  int nu;                    // work units per partition (32 * G)
};

constexpr int FB_STAGES = 3;
constexpr int FB_ENTRIES = 128;  // entries of one warp's stage (all its slots)
constexpr int FB_VEC = SPM_FB_VEC;  // ranks per lane
#ifndef SPM_FB_BATCH
#define SPM_FB_BATCH (16 / SPM_FB_VEC)
#endif
constexpr int FB_BATCH = SPM_FB_BATCH;  // steps whose gathers are issued together

inline int fibre_stage_bytes(int R) {
  const int G = fibre_slots(R);
  return G * (FB_ENTRIES / G + 2) * 8;
}

inline size_t fibre_smem_bytes(int R, int nu) {
  return (size_t)MT_WARPS * FB_STAGES * fibre_stage_bytes(R) +
         (size_t)MT_WARPS * FB_STAGES * sizeof(uint64_t) + (size_t)2 * nu * R * sizeof(float) +
         (size_t)2 * nu * sizeof(int);
}

// One lane's FB_VEC ranks of a factor row, as FP32 pairs.
template <typename FT, int VEC>
struct FibreRow;

template <>
struct FibreRow<float, 4> {
  using Raw = ulonglong2;
  // lane base (the factor plus the lane's first rank) + row * row bytes
  static __device__ __forceinline__ Raw load(const char* lane_base, uint32_t row, int R) {
    return ld_nc_v2_u64(lane_base + (uint64_t)row * (uint32_t)(R * 4));
  }
  static __device__ __forceinline__ uint64_t pair(const Raw& x, int i) { return i == 0 ? x.x : x.y; }
};

struct U64x4 {
  ulonglong2 lo, hi;
};
template <>
struct FibreRow<float, 8> {
  using Raw = U64x4;
  static __device__ __forceinline__ Raw load(const char* lane_base, uint32_t row, int R) {
    const char* p = lane_base + (uint64_t)row * (uint32_t)(R * 4);
    return {ld_nc_v2_u64(p), ld_nc_v2_u64(p + 16)};
  }
  static __device__ __forceinline__ uint64_t pair(const Raw& x, int i) {
    return i == 0 ? x.lo.x : (i == 1 ? x.lo.y : (i == 2 ? x.hi.x : x.hi.y));
  }
};

__device__ __forceinline__ uint64_t bf16_word_pair(uint32_t w) {  // two BF16 ranks widened
  return f2_pack(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}

template <>
struct FibreRow<__nv_bfloat16, 4> {
  using Raw = uint2;
  static __device__ __forceinline__ Raw load(const char* lane_base, uint32_t row, int R) {
    return __ldg(reinterpret_cast<const uint2*>(lane_base + (uint64_t)row * (uint32_t)(R * 2)));
  }
  static __device__ __forceinline__ uint64_t pair(const Raw& x, int i) {
    return bf16_word_pair(i == 0 ? x.x : x.y);
  }
};

template <>
struct FibreRow<__nv_bfloat16, 8> {
  using Raw = uint4;
  static __device__ __forceinline__ Raw load(const char* lane_base, uint32_t row, int R) {
    return __ldg(reinterpret_cast<const uint4*>(lane_base + (uint64_t)row * (uint32_t)(R * 2)));
  }
  static __device__ __forceinline__ uint64_t pair(const Raw& x, int i) {
    return bf16_word_pair(i == 0 ? x.x : (i == 1 ? x.y : (i == 2 ? x.z : x.w)));
  }
};

// A lane's NP FP32 pairs (2 NP consecutive ranks) to dst, 16 bytes at a time.
template <int NP>
__device__ __forceinline__ void store_pairs(float* dst, const uint64_t (&p)[NP]) {
#pragma unroll
  for (int q = 0; q < NP / 2; ++q) {
    float o[4];
    f2_unpack(p[2 * q], o[0], o[1]);
    f2_unpack(p[2 * q + 1], o[2], o[3]);
    *reinterpret_cast<float4*>(dst + 4 * q) = make_float4(o[0], o[1], o[2], o[3]);
  }
}

template <typename FT, int R>
__device__ __forceinline__ void mttkrp_fibre_partition(const FibreArgs& a, const int z) {
  constexpr int VEC = FB_VEC;
  constexpr int NP = VEC / 2;           // FP32 pairs per lane
  using RW = FibreRow<FT, VEC>;
  using Raw = typename RW::Raw;
  constexpr int LPN = R / VEC;          // lanes per slot
  constexpr int G = 32 / LPN;           // slots (units) per warp
  constexpr int SUB = FB_ENTRIES / G;   // entries of one slot per stage
  constexpr int SUBW = SUB + 2;         // its buffer: one alignment entry, padding
  constexpr int STAGE_BYTES = G * SUBW * 8;
  constexpr int U = FB_BATCH;
  static_assert(SUB % U == 0, "batch must divide the slot tile");
  static_assert(STAGE_BYTES % 16 == 0 && (SUBW * 8) % 16 == 0, "bulk-copy alignment");

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int aborted;
  __shared__ int64_t ubeg[MT_WARPS][G], uend[MT_WARPS][G];

  const int NU = a.nu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / LPN, sub = lane % LPN;
  const int r0 = sub * VEC;
  const int ul = warp * G + slot;            // unit within the partition
  const int64_t ug = (int64_t)z * NU + ul;   // unit within the copy

  unsigned char* stages = smem + (size_t)warp * FB_STAGES * STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)MT_WARPS * FB_STAGES * STAGE_BYTES) +
                   warp * FB_STAGES;
  float* part = reinterpret_cast<float*>(smem + (size_t)MT_WARPS * FB_STAGES * STAGE_BYTES +
                                         (size_t)MT_WARPS * FB_STAGES * sizeof(uint64_t));
  int* prow = reinterpret_cast<int*>(part + (size_t)2 * NU * R);

  const FibreUnit un = a.units[ug];
  const int64_t s0 = un.sbeg, s1 = un.send;
  const int64_t n_s = s1 - s0;
  if (sub == 0) {
    ubeg[warp][slot] = s0;
    uend[warp][slot] = s1;
  }
  if (lane == 0) {
#pragma unroll
    for (int st = 0; st < FB_STAGES; ++st) mbar_init(&bars[st], 1);
    fence_mbar_init();
  }
  if (threadIdx.x == 0) aborted = 0;
  __syncthreads();
  const uint32_t wait_polls =
      a.wait_limit == 0u ? (1u << 24) : (a.wait_limit == ~0u ? 0u : a.wait_limit);

  const int ntiles = __reduce_max_sync(SPM_FULL_MASK, (int)((n_s + SUB - 1) / SUB));

  // lane 0: bulk copies of tile t of every slot's range into stage t % S
  auto issue = [&](int t) {
    uint64_t* bar = &bars[t % FB_STAGES];
    unsigned char* dst = stages + (t % FB_STAGES) * STAGE_BYTES;
    uint32_t total = 0;
#pragma unroll
    for (int s = 0; s < G; ++s) {
      const int64_t lo = ubeg[warp][s] + (int64_t)t * SUB;
      const int64_t cnt = uend[warp][s] - lo < SUB ? uend[warp][s] - lo : SUB;
      if (cnt > 0) total += (uint32_t)((((lo & 1) + cnt) * 8 + 15) & ~(int64_t)15);
    }
    mbar_arrive_expect_tx(bar, total);
#pragma unroll
    for (int s = 0; s < G; ++s) {
      const int64_t lo = ubeg[warp][s] + (int64_t)t * SUB;
      const int64_t cnt = uend[warp][s] - lo < SUB ? uend[warp][s] - lo : SUB;
      if (cnt > 0) {
        const int64_t al = lo & ~(int64_t)1;
        const uint32_t bytes = (uint32_t)((((lo - al) + cnt) * 8 + 15) & ~(int64_t)15);
        bulk_g2s(dst + s * SUBW * 8, a.stream + al, bytes, bar);
      }
    }
  };
  int issued = ntiles < FB_STAGES ? ntiles : FB_STAGES;
  if (lane == 0)
    for (int t = 0; t < issued; ++t) issue(t);

  // slot state: running row and its sum, the row of the current fibre; the
  // unit's first row, once complete, goes straight to its boundary partial
  const int first_row = un.cd_first;
  int cur_row = first_row;
  bool first_done = false;
  float* pfirst = part + (size_t)(2 * ul) * R + r0;
  float* plast = pfirst + R;
  uint64_t acc[NP], ya[NP];
#pragma unroll
  for (int e = 0; e < NP; ++e) acc[e] = ya[e] = 0ull;
  // the lane's slice of row 0 of each input factor
  const char* lane_a = static_cast<const char*>(a.fac_a) + (size_t)r0 * sizeof(FT);
  const char* lane_b = static_cast<const char*>(a.fac_b) + (size_t)r0 * sizeof(FT);
  if (n_s > 0) {
    const Raw y = RW::load(lane_a, (uint32_t)un.ca_first, R);
#pragma unroll
    for (int e = 0; e < NP; ++e) ya[e] = RW::pair(y, e);
  }
  bool timeout = false;

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
      const bool ok = mbar_wait_bounded(&bars[t % FB_STAGES], (uint32_t)((t / FB_STAGES) & 1), wait_polls);
      timeout = __any_sync(SPM_FULL_MASK, !ok);
    }
    if (timeout) {
      for (int q = t; q < issued; ++q)
        (void)mbar_wait_bounded(&bars[q % FB_STAGES], (uint32_t)((q / FB_STAGES) & 1), 1u << 20);
      if (lane == 0) {
        atomicOr(a.err, DEV_ERR_TIMEOUT);
        atomicExch(&aborted, 1);
      }
      break;
    }
    const int64_t lo = s0 + (int64_t)t * SUB;
    const int cnt = (int)(s1 - lo < SUB ? (s1 - lo > 0 ? s1 - lo : 0) : SUB);
    const int2* ent = reinterpret_cast<const int2*>(stages + (t % FB_STAGES) * STAGE_BYTES +
                                                    slot * SUBW * 8) + (int)(lo & 1);
    const int nst = __reduce_max_sync(SPM_FULL_MASK, cnt);
    const int cmin = __reduce_min_sync(SPM_FULL_MASK, cnt);
    // One batch of U steps: the gathers first (every step one row load:
    // Y_a(c_a) at a header, Y_b(c_b) at a nonzero), then the steps in order.
    // Most batches have every step valid and no change of output row in any
    // slot: they run branch-free (acc += (val * row) .* ya, a header adding 0
    // and making its row ya).  Otherwise each step checks its validity and a
    // row change (steps past the slot's entries load row 0 with value 0).
    auto batch = [&](const int j, auto full_c) {
      constexpr bool FULL = decltype(full_c)::value;
      Raw row[U];
      int w1[U];   // c_d at a header, the value bits at a nonzero
      bool hd[U];
      bool chg = false;
#pragma unroll
      for (int uu = 0; uu < U; ++uu) {
        const int2 e = ent[j + uu];
        int w0 = e.x;
        w1[uu] = e.y;
        if (!FULL) {
          const bool v = j + uu < cnt;
          w0 = v ? w0 : 0;
          w1[uu] = v ? w1[uu] : 0;
        }
        hd[uu] = w0 < 0;
        chg = chg || (hd[uu] && w1[uu] != cur_row);
        row[uu] = RW::load(hd[uu] ? lane_a : lane_b, (uint32_t)w0 & 0x7FFFFFFFu, R);
      }
      if (FULL && !__any_sync(SPM_FULL_MASK, chg)) {
#pragma unroll
        for (int uu = 0; uu < U; ++uu) {
          const float vf = hd[uu] ? 0.f : __int_as_float(w1[uu]);
          const uint64_t vv = f2_pack(vf, vf);
#pragma unroll
          for (int e = 0; e < NP; ++e) {
            const uint64_t y = RW::pair(row[uu], e);
            acc[e] = f2_fma(f2_mul(vv, y), ya[e], acc[e]);
            ya[e] = hd[uu] ? y : ya[e];
          }
        }
        return;
      }
#pragma unroll
      for (int uu = 0; uu < U; ++uu) {
        if (hd[uu] && w1[uu] != cur_row) {
          store_pairs<NP>(first_done ? a.out + (int64_t)cur_row * R + r0 : pfirst, acc);
          first_done = true;
#pragma unroll
          for (int e = 0; e < NP; ++e) acc[e] = 0ull;
          cur_row = w1[uu];
        }
        const float vf = hd[uu] ? 0.f : __int_as_float(w1[uu]);
        const uint64_t vv = f2_pack(vf, vf);
#pragma unroll
        for (int e = 0; e < NP; ++e) {
          const uint64_t y = RW::pair(row[uu], e);
          acc[e] = f2_fma(f2_mul(vv, y), ya[e], acc[e]);
          ya[e] = hd[uu] ? y : ya[e];
        }
      }
    };
    for (int j = 0; j < nst; j += U) {
      if (j + U <= cmin) batch(j, std::true_type{});
      else batch(j, std::false_type{});
    }
  }

  // the unit's boundary partials: its first row, and its last row if distinct
  if (!timeout) {
    // first row still open: it is the only row (or the unit is empty)
    uint64_t only[NP], last[NP];
#pragma unroll
    for (int e = 0; e < NP; ++e) {
      only[e] = n_s > 0 ? acc[e] : 0ull;
      last[e] = first_done ? acc[e] : 0ull;
    }
    if (!first_done) store_pairs<NP>(pfirst, only);
    store_pairs<NP>(plast, last);
    if (sub == 0) {
      prow[2 * ul] = n_s > 0 ? first_row : -1;
      prow[2 * ul + 1] = first_done ? cur_row : -1;
    }
  }
  if (lane == 0 && !timeout) {
#pragma unroll
    for (int st = 0; st < FB_STAGES; ++st) mbar_inval(&bars[st]);
  }
  __syncthreads();

  // ---- block merge of the unit-boundary partials (as the record kernel) ----
  int* meta = a.cta_meta + 4 * z;
  const int64_t K0 = a.woff[(int64_t)z * NU], K1 = a.woff[(int64_t)(z + 1) * NU];
  if (K1 == K0 || aborted) {
    if (threadIdx.x == 0) { meta[0] = -1; meta[1] = -1; meta[2] = META_EMPTY; meta[3] = 0; }
    return;
  }
  const int NE = 2 * NU;  // <= 512
  if (warp == 0) {
    int m = -1;
    const int per = (NE + 31) / 32;
    const int e0 = lane * per;
    for (int e = e0; e < e0 + per && e < NE; ++e) m = max(m, prow[e]);
    int incl = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int tt = __shfl_up_sync(SPM_FULL_MASK, incl, o);
      if (lane >= o) incl = max(incl, tt);
    }
    int run = __shfl_up_sync(SPM_FULL_MASK, incl, 1);
    if (lane == 0) run = -1;
    for (int e = e0; e < e0 + per && e < NE; ++e) {
      run = max(run, prow[e]);
      prow[e] = run;
    }
  }
  __syncthreads();
  constexpr int MERGE_PER_THREAD = (64 * 32 * FB_VEC + MT_THREADS - 1) / MT_THREADS;  // NE * R
  for (int d = 1; d < NE; d <<= 1) {
    float tmp[MERGE_PER_THREAD];
#pragma unroll
    for (int c = 0; c < MERGE_PER_THREAD; ++c) {
      const int x = threadIdx.x + c * MT_THREADS;
      const int e = x / R;
      tmp[c] = (x < NE * R && e >= d && prow[e - d] == prow[e]) ? part[x - d * R] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < MERGE_PER_THREAD; ++c) {
      const int x = threadIdx.x + c * MT_THREADS;
      if (x < NE * R) part[x] += tmp[c];
    }
    __syncthreads();
  }
  // rows at the partition's ends and beside them (from the unit table)
  const int F = a.units[(int64_t)z * NU].cd_first;
  const int L = a.units[(int64_t)z * NU + NU - 1].cd_last;
  const bool shared_prev = K0 > 0 && a.units[(int64_t)z * NU - 1].cd_last == F;
  const bool shared_next = K1 < a.nnz && a.units[(int64_t)(z + 1) * NU].cd_first == L;
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

template <typename FT, int R>
__global__ void __launch_bounds__(MT_THREADS, 1) mttkrp_fibre_kernel(const FibreArgs a) {
  mttkrp_fibre_partition<FT, R>(a, blockIdx.x);
}

}  // namespace spm
