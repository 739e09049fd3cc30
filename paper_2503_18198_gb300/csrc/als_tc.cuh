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
//    once per mode by system_col_body, not per block).
// A digit is an integer of at most 8 bits, exact in BF16; a product of two
// digits is at most 2^14, and a sum of at most SM_DIG * R such products stays
// below 2^24, so the MMA accumulates it exactly in FP32.  Products of the
// same total weight p + q = L share the scale 2^(e_i + f_c - 7(L+2)), so one
// TMEM accumulator per level L collects all of them exactly:
//   D_L = sum_{p + q = L} Kp(M) Kq(W),   Z = sum_L 2^(e_i + f_c - 7(L+2)) D_L.
// One MMA per digit p of M covers every level it feeds: its B operand is the
// stack of W's digit tiles q = 0 .. LMAX - p (N = (LMAX + 1 - p) R columns)
// and its accumulator starts at level p's columns.  Levels L <= LMAX are kept
// (the dropped ones weigh 2^-49 of level 0); levels LMAX .. 2 are summed in
// FP32 (their weight is at most 2^-14 of level 0, so the rounding of that sum
// is below 2^-36 of the scale below), levels 1 and 0 in double-float with
// exact power-of-two scalings, then the sum is rounded once to FP32.
// The error against exact arithmetic is below 2^-34 of
// max_s |M(i,s)| * sum_s |W(s,c)| -- far under the FP32 rounding of Z.
//
// One CTA of 256 threads per virtual block: threads t and t + 128 own row t
// of each 128-row tile (TMEM lane t), half of its columns each; the tile of M
// comes in by one bulk copy, the
// digits are written to shared memory in the K-major layout of the MMA, one
// thread issues the MMAs and commits them to an mbarrier.  Rows without
// nonzeros (bit clear in `mask`) are not written, as in solve_body.
#pragma once

#include "als_kernels.cuh"
#include "tc_common.cuh"

namespace spm {

constexpr int TC_ROWS = 128;   // rows per tile (TMEM lanes)
constexpr int TC_THREADS = 256;  // two threads per row / lane (warps w and w + 4 share lanes)
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

// rint(y) for abs(y) <= 2^22 by the 1.5 * 2^23 shift (round half to even, like
// rintf; two adds on the FMA pipe instead of the conversion pipe).
__device__ __forceinline__ float round_int(float y) {
  return __fsub_rn(__fadd_rn(y, 12582912.f), 12582912.f);
}

// Two integer-valued floats of magnitude <= 256 as a BF16 pair (lo = a): their
// low 16 bits are zero, so the BF16 value is the high half, exactly.
__device__ __forceinline__ uint32_t pack_bf16_int(float a, float b) {
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

__device__ __forceinline__ void df_add(df& a, float x) {  // a += x (error-free two-sum)
  const float s = __fadd_rn(a.hi, x);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, err);
}

// Threads of a system_col_body block.
constexpr int SYS_THREADS = 128;

// 2^k as a double for -1022 <= k <= 1023 (exact), else via scalbn.
__device__ __forceinline__ double times_pow2(double x, int k) {
  if (k >= -1022 && k <= 1023) return __dmul_rn(x, __longlong_as_double((long long)(k + 1023) << 52));
  return scalbn(x, k);
}

// Columns c0 .. c1-1 of W = V^{-1}, V the Hadamard product of the Grams of
// every mode but d (Sec. II-A5), by one block (SYS_THREADS threads):
//  * V in FP64 and its Cholesky factor L (right-looking, lower triangle; every
//    block that solves columns of the same system computes the same L);
//  * per column c, L y = e_c, then L^T w = y (one warp, FP64): w = W(:, c);
//    warp k takes columns c0 + k, c0 + k + 4, ...
// A column's arithmetic does not depend on which block or warp solves it:
// one block per column (least latency, one tensor) and one block per system
// (least work, many tensors at once) give the same bits.
// w goes to V_out(:, c) (FP64), to winv as FP32 (hi, lo) pairs (W(s, c) at
// s R + c and R R + s R + c), and, when wdig is non-null, into the digit tile
// of the tensor-core solve: w is scaled by 2^-f_c (|w_s| < 2^f_c), rounded to
// 49 fractional bits and recoded from the least significant end into SW_DIG
// balanced 7-bit digits (|k_q| <= 64 below the leading digit, |k_0| <= 128),
// w_s 2^-f_c ~ sum_q k_q 2^{-7(q+1)}; digit q of w_s goes to row q R + c,
// column s of a K-major (K = R) BF16 tile, f_c to the int array after it.
// A pivot that is not positive and finite sets DEV_ERR_NUMERIC.
__device__ __forceinline__ void system_col_body(const double* __restrict__ grams, int N, int d,
                                                int R, int c0, int c1, double* __restrict__ V_out,
                                                float* __restrict__ winv,
                                                unsigned char* __restrict__ wdig,
                                                int* __restrict__ err) {
  __shared__ double S[64 * 64];
  __shared__ double linv[64];  // 1 / L(j, j)
  __shared__ double col[64];   // column j of L below the diagonal
  __shared__ int bad;
  const int t = threadIdx.x;
  if (t == 0) bad = *(volatile int*)err ? 1 : 0;
  __syncthreads();
  if (bad) return;
  const int RR = R * R;
  for (int e = t; e < RR; e += SYS_THREADS) {
    double v = 1.0;
    for (int w = 0; w < N; ++w)
      if (w != d) v = __dmul_rn(v, grams[(int64_t)w * RR + e]);
    S[e] = v;
  }
  __syncthreads();
  for (int j = 0; j < R; ++j) {
    if (t == 0) {
      const double piv = S[j * R + j];
      if (!(piv > 0.0) || !isfinite(piv)) {
        bad = 1;
      } else {
        const double r = rsqrt(piv);
        linv[j] = r;
        S[j * R + j] = __dmul_rn(piv, r);
      }
    }
    __syncthreads();
    if (bad) break;
    const double r = linv[j];
    for (int i = j + 1 + t; i < R; i += SYS_THREADS) {
      const double l = __dmul_rn(S[i * R + j], r);
      col[i] = l;
      S[i * R + j] = l;
    }
    __syncthreads();
    // trailing lower triangle (rows and columns j+1 .. R-1), entry e of it
    // row-major: row a, column b <= a
    const int m = R - j - 1;
    const int T = m * (m + 1) / 2;
    for (int e = t; e < T; e += SYS_THREADS) {
      int a = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while (a * (a + 1) / 2 > e) --a;
      while ((a + 1) * (a + 2) / 2 <= e) ++a;
      const int i = j + 1 + a, k = j + 1 + (e - a * (a + 1) / 2);
      S[i * R + k] = fma(-col[i], col[k], S[i * R + k]);
    }
    __syncthreads();
  }
  if (bad) {
    if (t == 0) atomicOr(err, DEV_ERR_NUMERIC);
    return;
  }
  // L^T into the strict upper triangle (S(i, k) = L(k, i), k > i) so that
  // both substitutions read rows of S
  for (int e = t; e < RR; e += SYS_THREADS) {
    const int i = e / R, k = e % R;
    if (k > i) S[e] = S[k * R + i];
  }
  __syncthreads();
  const int l = t & 31;
  for (int c = c0 + (t >> 5); c < c1; c += SYS_THREADS / 32) {
    // lane l keeps entries l and l + 32 of the right-hand side / solution
    double b0 = l == c ? 1.0 : 0.0, b1 = l + 32 == c ? 1.0 : 0.0;
    for (int i = c; i < R; ++i) {  // L y = e_c (y_i = 0 for i < c)
      const double yi = __dmul_rn(__shfl_sync(SPM_FULL_MASK, i < 32 ? b0 : b1, i & 31), linv[i]);
      if (l > i && l < R) b0 = fma(-S[i * R + l], yi, b0);
      if (l + 32 > i && l + 32 < R) b1 = fma(-S[i * R + l + 32], yi, b1);
      if (l == (i & 31)) {
        if (i < 32) b0 = yi;
        else b1 = yi;
      }
    }
    for (int i = R - 1; i >= 0; --i) {  // L^T w = y
      const double wi = __dmul_rn(__shfl_sync(SPM_FULL_MASK, i < 32 ? b0 : b1, i & 31), linv[i]);
      if (l < i) b0 = fma(-S[i * R + l], wi, b0);
      if (l + 32 < i) b1 = fma(-S[i * R + l + 32], wi, b1);
      if (l == (i & 31)) {
        if (i < 32) b0 = wi;
        else b1 = wi;
      }
    }
    int fx = INT_MIN;  // exponent bound of the column
    for (int h = 0; h < 2; ++h) {
      const int s = l + 32 * h;
      if (s >= R) continue;
      const double w = h ? b1 : b0;
      V_out[s * R + c] = w;
      const float hi = (float)w;
      winv[s * R + c] = hi;
      winv[RR + s * R + c] = (float)__dsub_rn(w, (double)hi);
      const unsigned long long bits = __double_as_longlong(w) & 0x7FFFFFFFFFFFFFFFull;
      if (bits != 0) {
        const int be = (int)(bits >> 52);
        fx = max(fx, be == 0 ? -1021 : be - 1022);  // |w| < 2^(be - 1022)
      }
    }
    if (!wdig) continue;
    fx = __reduce_max_sync(SPM_FULL_MASK, fx);
    if (fx == INT_MIN) fx = 0;
    if (l == 0) reinterpret_cast<int*>(wdig + SW_DIG * RR * 2)[c] = fx;
    for (int h = 0; h < 2; ++h) {
      const int s = l + 32 * h;
      if (s >= R) continue;
      long long n = __double2ll_rn(times_pow2(h ? b1 : b0, 49 - fx));  // |n| <= 2^49
#pragma unroll
      for (int q = SW_DIG - 1; q >= 0; --q) {
        long long dg = n;
        if (q > 0) {
          dg = ((n + 64) & 127) - 64;  // balanced remainder mod 128
          n = (n - dg) >> 7;           // exact
        }
        *reinterpret_cast<__nv_bfloat16*>(wdig + tc::kmajor_offset(q * R + c, s, R)) =
            __float2bfloat16_rn((float)dg);
      }
    }
  }
}

// Z = M W for rows tile vb, vb + nvb, ... (see the head of this file), with
// the column sums of Z^2 and the column maxima of |Z| of those rows into
// colsq_part / colmax_part (block vb's slots).  `wdig` is the mode's W digit
// tile (system_col_body).
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
  __shared__ float amax_s[2][TC_ROWS];
  if (*(volatile const int*)err) return;
  constexpr int H = R / 2;  // columns per thread

  unsigned char* sA = smem_tc;
  unsigned char* sB = sA + S::A_BYTES;
  const int* fexp = reinterpret_cast<const int*>(sB + S::B_BYTES);
  float* sM = reinterpret_cast<float*>(sB + S::WD_BYTES);  // 2 stages
  float* sZ = reinterpret_cast<float*>(sA);                // after the MMAs of a tile
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int rl = t & (TC_ROWS - 1), half = t / TC_ROWS;  // row of the tile, column half
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
      const int64_t row = tile * TC_ROWS + rl;
      const bool in = row < I;
      // this thread's half of row rl of the staged tile, read in a per-row
      // rotation of its 16-byte chunks (rows are 4R bytes apart: unrotated,
      // a warp's reads would share banks)
      const float* mr = sM + st * TC_ROWS * R + rl * R + half * H;
      float amax = 0.f;
      if (in)
#pragma unroll
        for (int c = 0; c < H / 4; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(mr + ((c + rl) % (H / 4)) * 4);
          amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
      amax_s[half][rl] = amax;
      __syncthreads();
      amax = fmaxf(amax_s[0][rl], amax_s[1][rl]);
      const int e_row = scale_expf(amax);  // |M(row, s)| < 2^e_row
      const bool fast = e_row >= -125 && e_row <= 126;
      const float inv = fast ? pow2f(-e_row) : 1.f;
#pragma unroll
      for (int g = 0; g < H / 8; ++g) {
        const int gg = (g + rl) % (H / 8);
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
            k[j] = round_int(y);
            x[j] = __fsub_rn(y, k[j]);
          }
          *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(rl, p * R + half * H + gg * 8, S::KA)) =
              make_uint4(pack_bf16_int(k[0], k[1]), pack_bf16_int(k[2], k[3]),
                         pack_bf16_int(k[4], k[5]), pack_bf16_int(k[6], k[7]));
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
      // Z(row, c) from the levels: LMAX .. 2 in FP32 (Horner), 1 and 0 in
      // double-float, then the scale 2^(e_row + f_c - 14) of level 0
      const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
      for (int c0 = half * H; c0 < half * H + H; c0 += 8) {
        uint32_t v[TC_LMAX + 1][8];
#pragma unroll
        for (int L = 0; L <= TC_LMAX; ++L) tc::ld8(lane_addr + (uint32_t)(L * R + c0), v[L]);
        tc::wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float h = __uint_as_float(v[TC_LMAX][j]);
#pragma unroll
          for (int L = TC_LMAX - 1; L >= 2; --L) h = fmaf(h, 0.0078125f, __uint_as_float(v[L][j]));
          df z = {__uint_as_float(v[1][j]), 0.f};
          df_add(z, __fmul_rn(h, 0.0078125f));
          z.hi = __fmul_rn(z.hi, 0.0078125f);
          z.lo = __fmul_rn(z.lo, 0.0078125f);
          df_add(z, __uint_as_float(v[0][j]));
          const int k = e_row + fexp[c0 + j] - 14;
          float zf;
          if (k >= -126 && k <= 127) {
            const float sc = pow2f(k);
            zf = __fadd_rn(__fmul_rn(z.hi, sc), __fmul_rn(z.lo, sc));
          } else {
            zf = __fadd_rn(ldexpf(z.hi, k), ldexpf(z.lo, k));
          }
          sZ[rl * S::ZS_STRIDE + c0 + j] = zf;
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

// ---------------------------------------------------------------------------
// Normalisation and Gram of the new factor on the tensor cores (R = 16, 32):
// Y = Z / lambda (stored type FT), G = Y^T Y from the STORED Y, and (last mode
// of a sweep) the column sums of M .* Y.
//
// Column r of Y is scaled by 2^-g_r (|Y(i, r)| < 2^(g_r - 1) for every row,
// from the column maxima of |Z| and lambda) and cut into NDIG = 128 / R
// balanced integer digits of 7 bits, Y(i, r) 2^-g_r ~ sum_p k_p 2^{-7(p+1)},
// |k_p| <= 64.  Digit p of column r is row m = p R + r of a 128 x 128 BF16
// tile A whose K index is the row of Y within a 128-row tile; one MMA chain
// D += A A^T per tile sums, for every pair of digit rows (p, r), (q, s),
//   D(pR + r, qR + s) = sum_i k_p(i, r) k_q(i, s)
// exactly in FP32 (products <= 2^12, at most GT_FLUSH * 128 rows between
// reads: sums < 2^22).  Every GT_FLUSH tiles the accumulator is read and
// folded into double-float sums acc_{p,r}(s) += sum_q 2^-7q D(pR+r, qR+s);
// at the end G(r, s) = 2^(g_r + g_s - 14) sum_p 2^-7p acc_{p,r}(s).  With
// NDIG >= 4 digits (>= 29 bits below the column maximum) the stored FP32
// values within 2^-5 of their column's maximum are represented exactly and
// the others to 2^-29 of it: the Gram error is far below the FP32 rounding
// of the factor itself.
// ---------------------------------------------------------------------------
constexpr int GT_ROWS = 128;    // rows of Y per tile (K of the MMAs)
constexpr int GT_STAGES = 2;    // Z tiles in flight (two blocks fit an SM)
constexpr int GT_FLUSH = 8;     // tiles between accumulator reads (1024 rows)

__host__ __device__ constexpr bool tc_gram_rank(int R) { return tc_solve_rank(R) && R <= 32; }

template <int R>
struct TcGramShape {
  static constexpr int NDIG = 128 / R;
  static constexpr int NQ = TC_THREADS / R;          // row slices of a tile
  static constexpr int SLICE = GT_ROWS / NQ;         // rows per slice (multiple of 8)
  static constexpr int Z_BYTES = GT_ROWS * R * 4;
  static constexpr int A_BYTES = 128 * GT_ROWS * 2;  // one digit tile
  static constexpr int RED_BYTES = NDIG * R * R * 8; // the final per-digit Gram parts
  static_assert(RED_BYTES <= 2 * A_BYTES, "final reduction fits in the digit tiles");
  static_assert(SLICE % 8 == 0, "digit groups of 8 rows");
  static constexpr size_t SMEM = (size_t)GT_STAGES * Z_BYTES + 2 * A_BYTES;
};

// Virtual blocks of the tensor-core normalisation/Gram pass over I rows (a
// function of I and the partial-buffer size only: batched and single-tensor
// sweeps split alike).
inline int tc_gram_blocks(int64_t I, int cap) {
  const int64_t tiles = (I + GT_ROWS - 1) / GT_ROWS;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, cap / 2));
}

// The pass over tiles vb, vb + nvb, ... of Z (see above).  `lam` holds
// lambda (R values) then the column scale exponents g_r (R values, from
// lambda_body).  Writes Y, gram_part[vb] (R x R) and, when M is non-null,
// inner_part[vb] (R).  Rows without nonzeros (bit clear in `mask`) get Y = 0.
template <typename FT, int R>
__device__ __forceinline__ void tc_scale_gram_body(const float* __restrict__ Z,
                                                   const double* __restrict__ lam, int64_t I,
                                                   FT* __restrict__ Y, const float* __restrict__ M,
                                                   double* __restrict__ gram_part,
                                                   double* __restrict__ inner_part,
                                                   const int* __restrict__ err, int vb, int nvb,
                                                   const uint32_t* __restrict__ mask) {
  using S = TcGramShape<R>;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t bars[GT_STAGES + 2];  // Z stages; MMAs of digit tile 0 / 1
  __shared__ double red_in[TC_THREADS];
  __shared__ int gx[R];
  if (*(volatile const int*)err) return;

  float* sZ = reinterpret_cast<float*>(smem_tc);
  unsigned char* sA = smem_tc + GT_STAGES * S::Z_BYTES;
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int r = t % R, kq = t / R;  // digitising: column r, rows kq * SLICE .. of a tile
  // reading D: thread t < 128 owns accumulator lane t = digit row (p, r) = (t / R, t % R)
  const int64_t ntiles = (I + GT_ROWS - 1) / GT_ROWS;
  const int nloc = vb < ntiles ? (int)((ntiles - 1 - vb) / nvb + 1) : 0;

  const double lr = lam[r];
  const float inv = lr > 0.0 ? (float)(1.0 / lr) : 1.f;
  const int g = (int)lam[R + r];
  const bool gfast = g >= -125 && g <= 126;
  const float gs = gfast ? pow2f(-g) : 1.f;
  if (t < R) gx[t] = (int)lam[R + t];
  if (warp == 0) tc::tmem_alloc(&tmem_slot, 128);
  if (t == 0) {
    for (int b = 0; b < GT_STAGES + 2; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  auto fetch = [&](int j) {  // local tile j into stage j % GT_STAGES (thread 0)
    fence_proxy_async_smem();
    const int64_t r0 = ((int64_t)vb + (int64_t)j * nvb) * GT_ROWS;
    const int64_t rows = I - r0 < GT_ROWS ? I - r0 : GT_ROWS;
    const uint32_t bytes = (uint32_t)(rows * R * 4);
    mbar_arrive_expect_tx(&bars[j % GT_STAGES], bytes);
    bulk_g2s(sZ + (j % GT_STAGES) * GT_ROWS * R, Z + r0 * R, bytes, &bars[j % GT_STAGES]);
  };
  int fetched = 0;  // thread 0's count of issued tile copies
  if (t == 0)
    for (; fetched < nloc && fetched < GT_STAGES; ++fetched) fetch(fetched);

  df acc[R];  // digit row t of D folded over q: acc(s) = sum_q 2^-7q D(t, qR + s)
#pragma unroll
  for (int s = 0; s < R; ++s) acc[s] = {0.f, 0.f};
  df inn = {0.f, 0.f};
  bool ok = true;
  int j = 0, committed = 0;
  for (; j < nloc && ok; ++j) {
    const int st = j % GT_STAGES, b = j & 1;
    const int64_t row0 = ((int64_t)vb + (int64_t)j * nvb) * GT_ROWS;
    ok = mbar_wait_bounded(&bars[st], (uint32_t)((j / GT_STAGES) & 1));
    if (ok && j >= 2) ok = mbar_wait_bounded(&bars[GT_STAGES + b], (uint32_t)(((j - 2) >> 1) & 1));
    if (!__syncthreads_and(ok)) break;
    const float* zs = sZ + st * GT_ROWS * R;
    unsigned char* A = sA + b * S::A_BYTES;
#pragma unroll 1
    for (int k0 = kq * S::SLICE; k0 < (kq + 1) * S::SLICE; k0 += 8) {
      // rows row0 + k0 .. + 7 share one word of the mask (row0 + k0 is a multiple of 8)
      const uint32_t live8 =
          mask ? (__ldg(&mask[(row0 + k0) >> 5]) >> ((row0 + k0) & 31)) & 0xFFu : 0xFFu;
      float x[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int64_t row = row0 + k0 + jj;
        float y = 0.f;
        if (row < I) {
          const bool lv = (live8 >> jj) & 1u;
          const float z = lv ? zs[(k0 + jj) * R + r] : 0.f;
          const FT ys = store_cvt<FT>(lr > 0.0 ? __fmul_rn(z, inv) : z);
          Y[row * R + r] = ys;
          y = load_f<FT>(&ys, 0);
          if (M && lv) df_add_prod(inn, M[row * R + r], y);
        }
        x[jj] = gfast ? __fmul_rn(y, gs) : ldexpf(y, -g);
      }
#pragma unroll
      for (int p = 0; p < S::NDIG; ++p) {
        float k[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const float yy = __fmul_rn(x[jj], 128.f);
          k[jj] = round_int(yy);
          x[jj] = __fsub_rn(yy, k[jj]);
        }
        *reinterpret_cast<uint4*>(A + tc::kmajor_offset(p * R + r, k0, GT_ROWS)) =
            make_uint4(pack_bf16_int(k[0], k[1]), pack_bf16_int(k[2], k[3]),
                       pack_bf16_int(k[4], k[5]), pack_bf16_int(k[6], k[7]));
      }
    }
    fence_proxy_async_smem();  // digits visible to the tensor core
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
      if (fetched < nloc) { fetch(fetched); ++fetched; }  // into stage st, read by now
      const bool first = (j % GT_FLUSH) == 0;
      const uint32_t a0 = smem_addr(A);
#pragma unroll
      for (int k16 = 0; k16 < GT_ROWS; k16 += 16) {
        const uint64_t da = tc::smem_desc(a0 + (k16 / 8) * 128, 128, (GT_ROWS / 8) * 128);
        tc::mma_bf16(tmem, da, da, tc::idesc_bf16(128, 128), !(first && k16 == 0));
      }
      tc::commit(&bars[GT_STAGES + b]);
    }
    committed = j + 1;
    if ((j % GT_FLUSH) == GT_FLUSH - 1 || j == nloc - 1) {
      ok = mbar_wait_bounded(&bars[GT_STAGES + b], (uint32_t)((j >> 1) & 1));
      tc::fence_after_sync();
      if (!__syncthreads_and(ok)) break;
      if (t < 128) {  // warps 0 .. 3: one accumulator lane each
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int q = 0; q < S::NDIG; ++q) {
          uint32_t v[R / 8][8];
#pragma unroll
          for (int c8 = 0; c8 < R / 8; ++c8) tc::ld8(lane_addr + (uint32_t)(q * R + c8 * 8), v[c8]);
          tc::wait_ld();
          const float wq = pow2f(-7 * q);
#pragma unroll
          for (int s = 0; s < R; ++s) df_add(acc[s], __fmul_rn(__uint_as_float(v[s / 8][s % 8]), wq));
        }
      }
      tc::fence_before_sync();
      __syncthreads();  // every read done before the next MMA overwrites D
    }
  }
  if (!ok) {
    // a wait gave up: let the copies and MMAs in flight finish before the
    // shared and tensor memory are reused or released
    if (t == 0) {
      for (int k = j; k < fetched; ++k)
        (void)mbar_wait_bounded(&bars[k % GT_STAGES], (uint32_t)((k / GT_STAGES) & 1), 1u << 20);
      if (committed > 0) {
        const int jc = committed - 1;
        (void)mbar_wait_bounded(&bars[GT_STAGES + (jc & 1)], (uint32_t)((jc >> 1) & 1), 1u << 20);
      }
      atomicOr(const_cast<int*>(err), DEV_ERR_TIMEOUT);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  // per-digit parts of the Gram into the digit tiles (all MMAs have completed)
  double* red = reinterpret_cast<double*>(sA);
  if (t < 128)
#pragma unroll
    for (int s = 0; s < R; ++s) red[t * R + s] = times_pow2(df_value(acc[s]), -7 * (t / R));
  red_in[t] = df_value(inn);
  __syncthreads();
  if (ok) {
    const int RR = R * R;
    for (int e = t; e < RR; e += TC_THREADS) {
      const int rr = e / R, ss = e % R;
      if (ss > rr) continue;
      double v = 0.0;
#pragma unroll
      for (int p = 0; p < S::NDIG; ++p) v += red[(p * R + rr) * R + ss];
      v = times_pow2(v, gx[rr] + gx[ss] - 14);
      gram_part[(int64_t)vb * RR + rr * R + ss] = v;
      gram_part[(int64_t)vb * RR + ss * R + rr] = v;
    }
    if (M && t < R) {
      double sum = 0.0;
      for (int q = 0; q < S::NQ; ++q) sum += red_in[q * R + t];
      inner_part[(int64_t)vb * R + t] = sum;
    }
  }
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
  if (t == 0 && ok)
    for (int b = 0; b < GT_STAGES + 2; ++b) mbar_inval(&bars[b]);
}

}  // namespace spm
