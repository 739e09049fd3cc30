// als_tc.cuh -- the CP-ALS row passes on the tensor cores, with FP64-level
// accuracy from BF16 x BF16 -> FP32 MMAs (exact operand splitting).
//
// Row solve Z = M V^{-1}.  The R x R system comes from the FP64 Cholesky of
// the Hadamard product of the Grams (Sec. II-A5; system_body), W = V^{-1} in
// FP64.  Splitting:
//  * each row i of M (FP32) is scaled by 2^-e_i (e_i the exponent of its
//    largest magnitude) and cut into SM_DIG integer digits of 7 bits,
//    m_i = 2^e_i * sum_p k_p(i) 2^{-7(p+1)}, |k_p| <= 128;
//  * each column c of W likewise into SW_DIG digits with scale 2^f_c (done
//    once per mode by wdigits_body, not per block).
// A digit is an integer of at most 8 bits, exact in BF16; a product of two
// digits is at most 2^14, and a sum of at most SM_DIG * R such products stays
// below 2^24, so the MMA accumulates it exactly in FP32.  Products of the
// same total weight p + q = L share the scale 2^(e_i + f_c - 7(L+2)), so one
// TMEM accumulator per level L collects all of them exactly:
//   D_L = sum_{p + q = L} Kp(M) Kq(W),   Z = sum_L 2^(e_i + f_c - 7(L+2)) D_L.
// One MMA per digit p of M covers every level it feeds: its B operand is the
// stack of W's digit tiles q = 0 .. LMAX - p (N = (LMAX + 1 - p) R columns)
// and its accumulator starts at level p's columns.  Levels L <= LMAX are kept
// (the dropped ones weigh 2^-49 of level 0); levels LMAX .. 3 are summed in
// FP32 (their weight is at most 2^-21 of level 0), the rest in double-float
// with exact power-of-two scalings, then the sum is rounded once to FP32.
// The error against exact arithmetic is below 2^-34 of
// max_s |M(i,s)| * sum_s |W(s,c)| -- far under the FP32 rounding of Z.
//
// One CTA of 128 threads per virtual block: thread t owns row t of each
// 128-row tile (TMEM lane t); the tile of M comes in by one bulk copy, the
// digits are written to shared memory in the K-major layout of the MMA, one
// thread issues the MMAs and commits them to an mbarrier.  Rows without
// nonzeros (bit clear in `mask`) are not written, as in solve_body.
#pragma once

#include "als_kernels.cuh"
#include "tc_common.cuh"

namespace spm {

constexpr int TC_ROWS = 128;   // rows per tile (TMEM lanes)
constexpr int TC_THREADS = 128;
constexpr int SM_DIG = 5;      // digits of a row of M  (35 bits)
constexpr int SW_DIG = 7;      // digits of a column of W (49 bits)
constexpr int TC_LMAX = 6;     // highest digit level kept
static_assert(TC_LMAX + 1 == SW_DIG, "W's digit stack covers every kept level");

#ifndef SPM_ALS_TC
#define SPM_ALS_TC 1  // 0: every rank takes the CUDA-core (double-float) row solve
#endif
__host__ __device__ constexpr bool tc_solve_rank(int R) {
  return SPM_ALS_TC && (R == 16 || R == 32 || R == 64);
}

// Shapes of the solve's shared-memory tiles (bytes) for rank R.
template <int R>
struct TcSolveShape {
  static constexpr int KA = SM_DIG * R;        // K of the M-digit tile (digit p at K block p)
  static constexpr int NB = SW_DIG * R;        // rows of the W-digit stack (row q R + c)
  static constexpr int A_BYTES = TC_ROWS * KA * 2;
  static constexpr int B_BYTES = NB * R * 2;   // K = R
  static constexpr int WD_BYTES = B_BYTES + R * 4;  // + the column exponents f_c
  static constexpr int MT_BYTES = TC_ROWS * R * 4;  // one tile of M (FP32)
  static constexpr int ZS_STRIDE = R + 1;           // staged Z row (floats)
  static constexpr int NCOLS_USED = (TC_LMAX + 1) * R;
  static constexpr uint32_t NCOLS = NCOLS_USED <= 32 ? 32 : NCOLS_USED <= 64 ? 64
                                  : NCOLS_USED <= 128 ? 128 : NCOLS_USED <= 256 ? 256 : 512;
  // the staged Z tile reuses the digit tile once the MMAs have read it
  static_assert(TC_ROWS * ZS_STRIDE * 4 <= A_BYTES, "Z staging fits in the digit tile");
  static_assert(WD_BYTES % 16 == 0 && A_BYTES % 16 == 0, "bulk copy sizes");
  static constexpr size_t SMEM = (size_t)A_BYTES + WD_BYTES + 2 * MT_BYTES;
};

// Bytes of the per-mode W digit tile for rank R (0 when R takes no tensor-core solve).
__host__ __device__ constexpr int tc_wdig_bytes(int R) {
  return R == 16 ? TcSolveShape<16>::WD_BYTES
         : R == 32 ? TcSolveShape<32>::WD_BYTES
         : R == 64 ? TcSolveShape<64>::WD_BYTES : 0;
}

static_assert(tc_wdig_bytes(16) == als_wdig_bytes(16) && tc_wdig_bytes(32) == als_wdig_bytes(32) &&
                  tc_wdig_bytes(64) == als_wdig_bytes(64),
              "plan accounting of the W digit tiles");

// 2^k as a float for -126 <= k <= 127 (exact).
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// Exponent e with |x| < 2^e for the largest |x| seen (float bits; 0 for zero).
__device__ __forceinline__ int scale_expf(float amax) {
  if (!(amax > 0.f)) return 0;
  int e;
  (void)frexpf(amax, &e);  // amax = m 2^e, 0.5 <= m < 1
  return e;
}

__device__ __forceinline__ void df_add(df& a, float x) {  // a += x (error-free two-sum)
  const float s = __fadd_rn(a.hi, x);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, err);
}

// The W digit tile of one mode, from W = V^{-1} (FP64, R x R, row-major) in
// global memory.  Column c of W is scaled by 2^-f_c (|W(s,c)| < 2^f_c for all
// s), rounded to 49 fractional bits, and recoded from the least significant
// end into SW_DIG balanced 7-bit digits (|k_q| <= 64 below the leading digit,
// |k_0| <= 128): W(s,c) 2^-f_c ~ sum_q k_q 2^{-7(q+1)}.  Digit q of W(s,c)
// goes to row q R + c, column s of a K-major (K = R) BF16 tile; the R
// exponents f_c follow the tile.  Whole block; call after W is written.
__device__ __forceinline__ void wdigits_body(const double* __restrict__ W, int R,
                                             unsigned char* __restrict__ wdig) {
  __shared__ int fx[64];
  const int RR = R * R;
  const int b_bytes = SW_DIG * R * R * 2;
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    int e = INT_MIN;
    for (int s = 0; s < R; ++s) {
      const unsigned long long b = __double_as_longlong(W[s * R + c]) & 0x7FFFFFFFFFFFFFFFull;
      if (b == 0) continue;
      const int be = (int)(b >> 52);
      e = max(e, be == 0 ? -1021 : be - 1022);  // |x| < 2^(be - 1022)
    }
    fx[c] = e == INT_MIN ? 0 : e;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += blockDim.x) reinterpret_cast<int*>(wdig + b_bytes)[c] = fx[c];
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int s = e / R, c = e % R;
    long long n = __double2ll_rn(scalbn(W[e], 49 - fx[c]));  // |n| <= 2^49
#pragma unroll
    for (int q = SW_DIG - 1; q >= 0; --q) {
      long long d = n;
      if (q > 0) {
        d = ((n + 64) & 127) - 64;  // balanced remainder mod 128
        n = (n - d) >> 7;           // exact
      }
      *reinterpret_cast<__nv_bfloat16*>(wdig + tc::kmajor_offset(q * R + c, s, R)) =
          __float2bfloat16_rn((float)d);
    }
  }
}

// Z = M W for rows tile vb, vb + nvb, ... (see the head of this file), with
// the column sums of Z^2 and the column maxima of |Z| of those rows into
// colsq_part / colmax_part (block vb's slots).  `wdig` is the mode's W digit
// tile (wdigits_body).
template <int R>
__device__ __forceinline__ void tc_solve_body(const float* __restrict__ M,
                                              const unsigned char* __restrict__ wdig, int64_t I,
                                              float* __restrict__ Z, double* __restrict__ colsq_part,
                                              float* __restrict__ colmax_part,
                                              const int* __restrict__ err, int vb, int nvb,
                                              const uint32_t* __restrict__ mask) {
  using S = TcSolveShape<R>;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t bars[4];  // [0]: MMAs done; [1], [2]: M tiles; [3]: W digits
  __shared__ double red[TC_THREADS];
  __shared__ float redm[TC_THREADS];
  if (*(volatile const int*)err) return;

  unsigned char* sA = smem_tc;
  unsigned char* sB = sA + S::A_BYTES;
  const int* fexp = reinterpret_cast<const int*>(sB + S::B_BYTES);
  float* sM = reinterpret_cast<float*>(sB + S::WD_BYTES);  // 2 stages
  float* sZ = reinterpret_cast<float*>(sA);                // after the MMAs of a tile
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int64_t ntiles = (I + TC_ROWS - 1) / TC_ROWS;

  if (warp == 0) tc::tmem_alloc(&tmem_slot, S::NCOLS);
  if (t == 0) {
    for (int b = 0; b < 4; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  // bulk copy of tile `tile` of M into stage `st` (thread 0)
  auto fetch = [&](int64_t tile, int st) {
    fence_proxy_async_smem();  // the stage's earlier reads before the copy's writes
    const int64_t r0 = tile * TC_ROWS;
    const int64_t rows = I - r0 < TC_ROWS ? I - r0 : TC_ROWS;
    const uint32_t bytes = (uint32_t)(rows * R * 4);
    mbar_arrive_expect_tx(&bars[1 + st], bytes);
    bulk_g2s(sM + st * TC_ROWS * R, M + r0 * R, bytes, &bars[1 + st]);
  };
  bool ok = true;
  int fetched = 0;  // tiles whose copies were issued (thread 0's count)
  int mmas = 0;     // tiles whose MMAs were committed
  if (t == 0) {
    mbar_arrive_expect_tx(&bars[3], S::WD_BYTES);
    bulk_g2s(sB, wdig, S::WD_BYTES, &bars[3]);
    if (vb < ntiles) { fetch(vb, 0); fetched = 1; }
  }
  ok = mbar_wait_bounded(&bars[3], 0u);
  df sq = {0.f, 0.f};  // column (t % R) sum of Z^2 over this block's rows
  float mx = 0.f;      // and max |Z|
  int it = 0;
  if (__syncthreads_and(ok))
    for (int64_t tile = vb; tile < ntiles && ok; tile += nvb, ++it) {
      const int st = it & 1;
      if (t == 0 && tile + nvb < ntiles) { fetch(tile + nvb, st ^ 1); ++fetched; }  // prefetch
      ok = mbar_wait_bounded(&bars[1 + st], (uint32_t)((it >> 1) & 1));
      if (!__syncthreads_and(ok)) break;
      const int64_t row = tile * TC_ROWS + t;
      const bool in = row < I;
      // row t of the staged tile, read in a per-thread rotation of its
      // 16-byte chunks (rows are 4R bytes apart: unrotated, a warp's reads
      // would share banks)
      const float* mr = sM + st * TC_ROWS * R + t * R;
      float amax = 0.f;
      if (in)
#pragma unroll 4
        for (int c = 0; c < R / 4; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(mr + ((c + t) % (R / 4)) * 4);
          amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
      const int e_row = scale_expf(amax);  // |M(row, s)| < 2^e_row
      const bool fast = e_row >= -125 && e_row <= 126;
      const float inv = fast ? pow2f(-e_row) : 1.f;
#pragma unroll 2
      for (int g = 0; g < R / 8; ++g) {
        const int gg = (g + t) % (R / 8);
        float x[8];
        if (in) {
          const float4 a = *reinterpret_cast<const float4*>(mr + gg * 8);
          const float4 b = *reinterpret_cast<const float4*>(mr + gg * 8 + 4);
          x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
          x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
#pragma unroll
          for (int j = 0; j < 8; ++j) x[j] = fast ? __fmul_rn(x[j], inv) : ldexpf(x[j], -e_row);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) x[j] = 0.f;
        }
        // digit p of each value: rint of the remainder scaled by 2^7 (exact steps)
#pragma unroll
        for (int p = 0; p < SM_DIG; ++p) {
          float k[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float y = __fmul_rn(x[j], 128.f);
            k[j] = rintf(y);
            x[j] = __fsub_rn(y, k[j]);
          }
          __nv_bfloat162 h[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(k[2 * j], k[2 * j + 1]);
          *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(t, p * R + gg * 8, S::KA)) =
              *reinterpret_cast<uint4*>(h);
        }
      }
      fence_proxy_async_smem();  // digits visible to the tensor core
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (t == 0) {
        // digit p of M against W's digits q = 0 .. LMAX - p, into levels p ..
        // LMAX (columns p R ..), N split in pieces of at most 256 columns
        for (int p = 0; p < SM_DIG; ++p) {
          const int nq = TC_LMAX + 1 - p;
#pragma unroll
          for (int k16 = 0; k16 < R; k16 += 16) {
            const uint64_t da = tc::smem_desc(smem_addr(sA) + ((p * R + k16) / 8) * 128, 128,
                                              (S::KA / 8) * 128);
            for (int q0 = 0; q0 < nq; q0 += 256 / R) {
              const int n = (nq - q0 < 256 / R ? nq - q0 : 256 / R) * R;
              const uint64_t db = tc::smem_desc(
                  smem_addr(sB) + (q0 * R / 8) * (R / 8) * 128 + (k16 / 8) * 128, 128, (R / 8) * 128);
              tc::mma_bf16(tmem + (uint32_t)((p + q0) * R), da, db, tc::idesc_bf16(TC_ROWS, n),
                           p > 0 || k16 > 0);
            }
          }
        }
        tc::commit(&bars[0]);
      }
      ++mmas;
      ok = mbar_wait_bounded(&bars[0], (uint32_t)(it & 1));
      tc::fence_after_sync();
      if (!__syncthreads_and(ok)) break;
      // Z(row, c) from the levels: LMAX .. 3 in FP32 (Horner), 2 .. 0 in
      // double-float, then the scale 2^(e_row + f_c - 14) of level 0
      const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < R; c0 += 8) {
        uint32_t v[TC_LMAX + 1][8];
#pragma unroll
        for (int L = 0; L <= TC_LMAX; ++L) tc::ld8(lane_addr + (uint32_t)(L * R + c0), v[L]);
        tc::wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float h = __uint_as_float(v[TC_LMAX][j]);
#pragma unroll
          for (int L = TC_LMAX - 1; L >= 3; --L) h = fmaf(h, 0.0078125f, __uint_as_float(v[L][j]));
          df z = {__uint_as_float(v[2][j]), 0.f};
          df_add(z, __fmul_rn(h, 0.0078125f));
#pragma unroll
          for (int L = 1; L >= 0; --L) {
            z.hi = __fmul_rn(z.hi, 0.0078125f);
            z.lo = __fmul_rn(z.lo, 0.0078125f);
            df_add(z, __uint_as_float(v[L][j]));
          }
          const int k = e_row + fexp[c0 + j] - 14;
          float zf;
          if (k >= -126 && k <= 127) {
            const float sc = pow2f(k);
            zf = __fadd_rn(__fmul_rn(z.hi, sc), __fmul_rn(z.lo, sc));
          } else {
            zf = __fadd_rn(ldexpf(z.hi, k), ldexpf(z.lo, k));
          }
          sZ[t * S::ZS_STRIDE + c0 + j] = zf;
        }
      }
      tc::fence_before_sync();
      __syncthreads();
      // column sums of Z^2 and maxima of |Z| (fixed order: rows of the tile
      // in turn), and the tile of Z out (rows with nonzeros only)
      {
        constexpr int PER = TC_THREADS / R;  // threads per column
        const int c = t % R, g = t / R;
        for (int rr = g; rr < TC_ROWS; rr += PER) {
          const float zz = sZ[rr * S::ZS_STRIDE + c];
          df_add_prod(sq, zz, zz);
          mx = fmaxf(mx, fabsf(zz));
        }
      }
      for (int x = t; x < TC_ROWS * R / 4; x += TC_THREADS) {
        const int rr = x / (R / 4), c4 = (x % (R / 4)) * 4;
        const int64_t gr = tile * TC_ROWS + rr;
        if (gr < I && row_live(mask, gr)) {
          const float* zs = sZ + rr * S::ZS_STRIDE + c4;
          *reinterpret_cast<float4*>(Z + gr * R + c4) = make_float4(zs[0], zs[1], zs[2], zs[3]);
        }
      }
      __syncthreads();  // sZ and the stage are reused by the next tile
    }
  if (!ok) {
    // a wait gave up: let the copies and MMAs still in flight finish before
    // tensor memory is released and the block exits
    if (t == 0) {
      (void)mbar_wait_bounded(&bars[3], 0u, 1u << 20);
      for (int k = it; k < fetched; ++k)
        (void)mbar_wait_bounded(&bars[1 + (k & 1)], (uint32_t)((k >> 1) & 1), 1u << 20);
      if (mmas > 0) (void)mbar_wait_bounded(&bars[0], (uint32_t)((mmas - 1) & 1), 1u << 20);
      atomicOr(const_cast<int*>(err), DEV_ERR_TIMEOUT);
    }
    __syncthreads();
  }
  red[t] = df_value(sq);
  redm[t] = mx;
  tc::fence_before_sync();
  __syncthreads();
  if (t < R) {
    double s = 0.0;
    float m = 0.f;
    for (int g = 0; g < TC_THREADS / R; ++g) {
      s += red[g * R + t];
      m = fmaxf(m, redm[g * R + t]);
    }
    colsq_part[(int64_t)vb * R + t] = s;
    if (colmax_part) colmax_part[(int64_t)vb * R + t] = m;
  }
  if (warp == 0) tc::tmem_dealloc(tmem, S::NCOLS);
  if (t == 0 && ok)
    for (int b = 0; b < 4; ++b) mbar_inval(&bars[b]);
}

}  // namespace spm
