// als_tc.cuh -- the CP-ALS row solve Z = M V^{-1} on the tensor cores, with
// FP64-level accuracy from BF16 x BF16 -> FP32 MMAs (exact operand splitting).
//
// The R x R system comes from the FP64 Cholesky of the Hadamard product of
// the Grams (Sec. II-A5; system_body), W = V^{-1} in FP64.  Splitting:
//  * each row i of M (FP32) is scaled by 2^-e_i (e_i the exponent of its
//    largest magnitude) and cut into SM_DIG integer digits of 7 bits,
//    m_i = 2^e_i * sum_p k_p(i) 2^{-7(p+1)}, |k_p| <= 128;
//  * each column c of W likewise into SW_DIG digits with scale 2^f_c.
// A digit is an integer of at most 8 bits, exact in BF16; a product of two
// digits is below 2^14, and a sum of at most SM_DIG * R such products stays
// below 2^24, so the MMA accumulates it exactly in FP32.  Products of the
// same total weight p + q = L share the scale 2^(e_i + f_c - 7(L+2)), so one
// TMEM accumulator per level L collects all of them exactly:
//   D_L = sum_{p + q = L} Kp(M) Kq(W),   Z = sum_L 2^(e_i + f_c - 7(L+2)) D_L.
// Levels L <= LMAX are kept (the dropped ones weigh 2^-49 of level 0) and
// summed in double-float (exact power-of-two scalings, error-free two-sums),
// then rounded once to FP32.  The error against exact arithmetic is below
// 2^-34 of max_s |M(i,s)| * sum_s |W(s,c)| -- far under the FP32 rounding of
// Z, like the double-float solve this replaces on CUDA cores.
//
// One CTA of 128 threads per virtual block: thread t owns row t of each
// 128-row tile (TMEM lane t), the tile of M comes in by one bulk copy, the
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

#ifndef SPM_ALS_TC
#define SPM_ALS_TC 1  // 0: every rank takes the CUDA-core (double-float) row solve
#endif
__host__ __device__ constexpr bool tc_solve_rank(int R) {
  return SPM_ALS_TC && (R == 16 || R == 32 || R == 64);
}

template <int R>
struct TcSolveShape {
  static constexpr int KA = SM_DIG * R;        // K of the M-digit tile
  static constexpr int KB = SW_DIG * R;        // K of the W-digit tile
  static constexpr int A_BYTES = TC_ROWS * KA * 2;
  static constexpr int B_BYTES = R * KB * 2;
  static constexpr int MT_BYTES = TC_ROWS * R * 4;  // one tile of M (FP32)
  static constexpr int ZS_STRIDE = R + 1;           // staged Z row (floats)
  static constexpr int NCOLS_USED = (TC_LMAX + 1) * R;
  static constexpr uint32_t NCOLS = NCOLS_USED <= 32 ? 32 : NCOLS_USED <= 64 ? 64
                                  : NCOLS_USED <= 128 ? 128 : NCOLS_USED <= 256 ? 256 : 512;
  // the staged Z tile reuses the digit tile once the MMAs have read it
  static_assert(TC_ROWS * ZS_STRIDE * 4 <= A_BYTES, "Z staging fits in the digit tile");
  static constexpr size_t SMEM = (size_t)A_BYTES + B_BYTES + 2 * MT_BYTES;
};

// Integer digit q (0-based) of x in (-1, 1): rint(r_q 2^(7(q+1))), with
// r_0 = x and r_{q+1} = r_q - digit * 2^(-7(q+1)) (every step exact).
template <typename T, int NDIG>
__device__ __forceinline__ void digits(T x, float (&k)[NDIG]) {
  T r = x;
#pragma unroll
  for (int q = 0; q < NDIG; ++q) {
    const T sc = (T)(1ull << (7 * (q + 1)));
    const T d = rint(r * sc);
    k[q] = (float)d;
    r -= d / sc;
  }
}

// Exponent e with max|x| < 2^e (0 for a zero row).
__device__ __forceinline__ int scale_exp(double amax) {
  if (!(amax > 0.0)) return 0;
  int e;
  (void)frexp(amax, &e);  // amax = m 2^e, 0.5 <= m < 1
  return e;
}

__device__ __forceinline__ void df_add(df& a, float x) {  // a += x (error-free two-sum)
  const float s = __fadd_rn(a.hi, x);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, err);
}

template <int R>
__device__ __forceinline__ void tc_solve_body(const float* __restrict__ M,
                                              const double* __restrict__ W, int64_t I,
                                              float* __restrict__ Z, double* __restrict__ colsq_part,
                                              const int* __restrict__ err, int vb, int nvb,
                                              const uint32_t* __restrict__ mask) {
  using S = TcSolveShape<R>;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t bars[3];  // [0]: MMAs done; [1], [2]: M tile copies
  __shared__ int fexp[R];
  __shared__ double red[TC_THREADS];
  if (*(volatile const int*)err) return;

  unsigned char* sA = smem_tc;
  unsigned char* sB = sA + S::A_BYTES;
  float* sM = reinterpret_cast<float*>(sB + S::B_BYTES);  // 2 stages
  float* sZ = reinterpret_cast<float*>(sA);              // after the MMAs of a tile
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int64_t ntiles = (I + TC_ROWS - 1) / TC_ROWS;

  if (warp == 0) tc::tmem_alloc(&tmem_slot, S::NCOLS);
  if (t == 0) {
    for (int b = 0; b < 3; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  // column scales of W and its digits, K-major: row c of B, K index q*R + s
  if (t < R) {
    double amax = 0.0;
    for (int s = 0; s < R; ++s) amax = fmax(amax, fabs(W[s * R + t]));
    fexp[t] = scale_exp(amax);
  }
  __syncthreads();
  for (int e = t; e < R * R; e += TC_THREADS) {
    const int s = e / R, c = e % R;
    float k[SW_DIG];
    digits<double, SW_DIG>(ldexp(W[e], -fexp[c]), k);
#pragma unroll
    for (int q = 0; q < SW_DIG; ++q)
      *reinterpret_cast<__nv_bfloat16*>(sB + tc::kmajor_offset(c, q * R + s, S::KB)) =
          __float2bfloat16_rn(k[q]);
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
  const uint32_t idesc = tc::idesc_bf16(TC_ROWS, R);
  df sq = {0.f, 0.f};  // column (t % R) sum of Z^2 over this block's rows
  int it = 0;
  bool ok = true;
  int fetched = 0;  // tiles whose copies were issued (thread 0's count)
  int mmas = 0;     // tiles whose MMAs were committed
  if (t == 0 && vb < ntiles) { fetch(vb, 0); fetched = 1; }
  for (int64_t tile = vb; tile < ntiles && ok; tile += nvb, ++it) {
    const int st = it & 1;
    if (t == 0 && tile + nvb < ntiles) { fetch(tile + nvb, st ^ 1); ++fetched; }  // prefetch
    ok = mbar_wait_bounded(&bars[1 + st], (uint32_t)((it >> 1) & 1));
    if (!__syncthreads_and(ok)) break;
    const int64_t row = tile * TC_ROWS + t;
    const bool in = row < I;
    // this row's digits (zeros past the end) into the A tile
    const float* mr = sM + st * TC_ROWS * R + t * R;
    double amax = 0.0;
    if (in)
      for (int s = 0; s < R; ++s) amax = fmax(amax, (double)fabsf(mr[s]));
    const int e_row = scale_exp(amax);
#pragma unroll 4
    for (int s8 = 0; s8 < R; s8 += 8) {
      float k[8][SM_DIG];
#pragma unroll
      for (int j = 0; j < 8; ++j) digits<float, SM_DIG>(in ? ldexpf(mr[s8 + j], -e_row) : 0.f, k[j]);
#pragma unroll
      for (int p = 0; p < SM_DIG; ++p) {
        __nv_bfloat162 h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(k[2 * j][p], k[2 * j + 1][p]);
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(t, p * R + s8, S::KA)) =
            *reinterpret_cast<uint4*>(h);
      }
    }
    fence_proxy_async_smem();  // digits visible to the tensor core
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
      for (int L = 0; L <= TC_LMAX; ++L) {
        bool first = true;
        for (int p = 0; p < SM_DIG; ++p) {
          const int q = L - p;
          if (q < 0 || q >= SW_DIG) continue;
#pragma unroll
          for (int k16 = 0; k16 < R; k16 += 16) {
            const uint64_t da = tc::smem_desc(smem_addr(sA) + ((p * R + k16) / 8) * 128, 128,
                                              (S::KA / 8) * 128);
            const uint64_t db = tc::smem_desc(smem_addr(sB) + ((q * R + k16) / 8) * 128, 128,
                                              (S::KB / 8) * 128);
            tc::mma_bf16(tmem + (uint32_t)(L * R), da, db, idesc, !first);
            first = false;
          }
        }
      }
      tc::commit(&bars[0]);
    }
    ++mmas;
    ok = mbar_wait_bounded(&bars[0], (uint32_t)(it & 1));
    tc::fence_after_sync();
    if (!__syncthreads_and(ok)) break;
    // Z(row, c) = sum over levels, smallest first, in double-float
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < R; c0 += 8) {
      df z[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) z[j] = {0.f, 0.f};
#pragma unroll
      for (int L = TC_LMAX; L >= 0; --L) {
        uint32_t v[8];
        tc::ld8(lane_addr + (uint32_t)(L * R + c0), v);
        tc::wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j)
          df_add(z[j], ldexpf(__uint_as_float(v[j]), e_row + fexp[c0 + j] - 7 * (L + 2)));
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) sZ[t * S::ZS_STRIDE + c0 + j] = __fadd_rn(z[j].hi, z[j].lo);
    }
    tc::fence_before_sync();
    __syncthreads();
    // column sums of Z^2 (fixed order: rows of the tile in turn), and the
    // tile of Z out (rows with nonzeros only)
    {
      constexpr int PER = TC_THREADS / R;  // threads per column
      const int c = t % R, g = t / R;
      for (int rr = g; rr < TC_ROWS; rr += PER) {
        const float zz = sZ[rr * S::ZS_STRIDE + c];
        df_add_prod(sq, zz, zz);
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
      for (int k = it; k < fetched; ++k)
        (void)mbar_wait_bounded(&bars[1 + (k & 1)], (uint32_t)((k >> 1) & 1), 1u << 20);
      if (mmas > 0) (void)mbar_wait_bounded(&bars[0], (uint32_t)((mmas - 1) & 1), 1u << 20);
      atomicOr(const_cast<int*>(err), DEV_ERR_TIMEOUT);
    }
    __syncthreads();
  }
  red[t] = df_value(sq);
  tc::fence_before_sync();
  __syncthreads();
  if (t < R) {
    double s = 0.0;
    for (int g = 0; g < TC_THREADS / R; ++g) s += red[g * R + t];
    colsq_part[(int64_t)vb * R + t] = s;
  }
  if (warp == 0) tc::tmem_dealloc(tmem, S::NCOLS);
  if (t == 0 && ok)
    for (int b = 0; b < 3; ++b) mbar_inval(&bars[b]);
}

}  // namespace spm
