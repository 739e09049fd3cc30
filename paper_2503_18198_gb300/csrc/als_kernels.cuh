// als_kernels.cuh -- device bodies of the CP-ALS update kernels (Sec. II-A5).
//
// Each body works on one tensor; row-pass bodies take a virtual block index
// vb of nvb, so the same code serves the single-tensor launches (vb =
// blockIdx.x) and the batched launches, whose blocks map to (tensor, vb)
// pairs.  FP64 is confined to the R x R system; the O(I R^2) passes use
// error-free FP32 transformations (two-product via FMA, two-sum).
#pragma once

#include <algorithm>

#include "plan.cuh"

namespace spm {

constexpr int ALS_THREADS = 256;
constexpr int GRAM_TILE_ROWS = 32;
// Fewest rows a virtual block of a row pass takes: per-block partials (R x R
// for the Gram, R for the column sums) and the per-block load of V^{-1} are
// then small next to the rows themselves.
constexpr int ALS_MIN_ROWS = 256;

// ---- double-float helpers (Dekker / Knuth error-free transformations) ----
// Every operation is an explicitly rounded intrinsic: the compiler may not
// contract a multiply and an add into one FMA, so the bits do not depend on
// which kernel (or translation unit) the code is compiled into -- a tensor's
// batched and single-tensor sweeps must agree bitwise.
struct df {
  float hi, lo;
};
__device__ __forceinline__ void df_add_prod(df& acc, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);  // exact: a*b = p + e
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ void df_add_prod2(df& acc, float a, float bh, float bl) {
  const float p = __fmul_rn(a, bh);
  float e = fmaf(a, bh, -p);
  e = fmaf(a, bl, e);
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ double df_value(const df& a) { return __dadd_rn((double)a.hi, (double)a.lo); }

// Sum of x[0], x[stride], ..., x[(n-1) stride] by one warp in a fixed order:
// lane l adds elements l, l + 32, ... in turn, then a fixed butterfly over the
// lanes; lane 0's total is returned to every lane.  The bits do not depend on
// which warp or launch does the sum.
__device__ __forceinline__ double warp_sum_strided(const double* __restrict__ x, int n,
                                                   int64_t stride, int lane) {
  double s = 0.0;
  // loads 8 at a time ahead of the (ordered) additions: the latency of the
  // strided reads overlaps, the sum is the same
  int b = lane;
  for (; b + 7 * 32 < n; b += 8 * 32) {
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = x[(int64_t)(b + 32 * k) * stride];
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
  }
  for (; b < n; b += 32) s += x[(int64_t)b * stride];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(SPM_FULL_MASK, s, o);
  return __shfl_sync(SPM_FULL_MASK, s, 0);
}

// Row i is non-empty (has a nonzero in the output mode) when its bit is set;
// a null mask counts every row as non-empty.  Rows without nonzeros have a
// zero MTTKRP row, so their update is exactly zero and their share of every
// row pass below is exactly zero too: skipping them leaves each sum's bits
// unchanged.
__device__ __forceinline__ bool row_live(const uint32_t* __restrict__ mask, int64_t i) {
  return !mask || ((__ldg(&mask[i >> 5]) >> (i & 31)) & 1u);
}

// Partial counts up to this are summed by one thread per entry (reads
// coalesced across entries); more by one warp per entry.  The choice depends
// on the count only, so a tensor's sums are the same in every launch shape.
constexpr int ALS_SERIAL_PARTIALS = 64;

// The plan's sticky error flag as seen by lane 0, for every lane of the warp
// (so that the warp takes one branch around its shuffles).
__device__ __forceinline__ int warp_err(const int* __restrict__ err) {
  int e = 0;
  if ((threadIdx.x & 31) == 0) e = *reinterpret_cast<const volatile int*>(err);
  return __shfl_sync(SPM_FULL_MASK, e, 0);
}

template <typename FT>
__device__ __forceinline__ float load_f(const FT* p, int64_t i);
template <>
__device__ __forceinline__ float load_f<float>(const float* p, int64_t i) { return p[i]; }
template <>
__device__ __forceinline__ float load_f<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}
template <typename FT>
__device__ __forceinline__ FT store_cvt(float x);
template <>
__device__ __forceinline__ float store_cvt<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 store_cvt<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}

// ---------------------------------------------------------------------------
// Gram partials: block b sums rows [i0, i1) of Y.  Only the lower triangle
// r >= s is accumulated (G is symmetric): thread t owns entries
// e = t, t + 256, ... of the R(R+1)/2 triangle entries in row-major order,
// and mirrors them when it stores.  Requires R <= 16 * GT.
// ---------------------------------------------------------------------------
template <typename FT, int GT>
__device__ __forceinline__ void gram_partial_body(const FT* __restrict__ Y, int64_t I, int R,
                                                  int64_t rows_per_block, double* __restrict__ part,
                                                  int vb, const uint32_t* __restrict__ mask) {
  constexpr int RMAX = 16 * GT;
  constexpr int EPT = (RMAX * (RMAX + 1) / 2 + ALS_THREADS - 1) / ALS_THREADS;  // entries per thread
  __shared__ float tile[GRAM_TILE_ROWS][RMAX + 1];
  __shared__ int live[GRAM_TILE_ROWS];
  const int64_t i0 = (int64_t)vb * rows_per_block;
  const int64_t i1 = std::min<int64_t>(I, i0 + rows_per_block);
  const int T = R * (R + 1) / 2;
  int er[EPT], es[EPT];
  df acc[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = threadIdx.x + k * ALS_THREADS;
    int r = 0;
    while ((r + 1) * (r + 2) / 2 <= e) ++r;  // e = r (r + 1) / 2 + s, s <= r
    er[k] = e < T ? r : 0;
    es[k] = e < T ? e - r * (r + 1) / 2 : 0;
    acc[k] = {0.f, 0.f};
  }
  for (int64_t t0 = i0; t0 < i1; t0 += GRAM_TILE_ROWS) {
    const int nrow = (int)std::min<int64_t>(GRAM_TILE_ROWS, i1 - t0);
    __syncthreads();
    if (threadIdx.x < GRAM_TILE_ROWS)
      live[threadIdx.x] = threadIdx.x < nrow && row_live(mask, t0 + threadIdx.x);
    __syncthreads();
    for (int e = threadIdx.x; e < GRAM_TILE_ROWS * RMAX; e += ALS_THREADS) {
      const int rr = e / RMAX, cc = e % RMAX;
      tile[rr][cc] = (live[rr] && cc < R) ? load_f<FT>(Y, (t0 + rr) * R + cc) : 0.f;
    }
    __syncthreads();
    for (int rr = 0; rr < nrow; ++rr) {
      if (!live[rr]) continue;
#pragma unroll
      for (int k = 0; k < EPT; ++k) df_add_prod(acc[k], tile[rr][er[k]], tile[rr][es[k]]);
    }
  }
  double* out = part + (int64_t)vb * R * R;
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = threadIdx.x + k * ALS_THREADS;
    if (e < T) {
      const double v = df_value(acc[k]);
      out[er[k] * R + es[k]] = v;
      out[es[k] * R + er[k]] = v;
    }
  }
}

// G = sum over blocks of the partials (FP64, fixed order).  Up to
// ALS_SERIAL_PARTIALS partials one thread sums an entry in block order;
// beyond that one warp does (lane-strided sums, then warp_sum_strided's
// shuffle tree, lane 0's value kept).  Virtual block vb of nvb takes its
// share of the entries, GR_ENTRIES at a time side by side so that their
// loads are in flight together; an entry's order of addition does not
// depend on the launch shape.
constexpr int GR_ENTRIES = 4;
__device__ __forceinline__ void gram_reduce_body(const double* __restrict__ part, int nblocks,
                                                 int R, double* __restrict__ G,
                                                 const int* __restrict__ err, int vb, int nvb) {
  if (warp_err(err)) return;
  const int RR = R * R;
  if (nblocks <= ALS_SERIAL_PARTIALS) {
    // thread t takes entries e, e + step, ..., GR_ENTRIES of them at a time
    const int step = nvb * blockDim.x;
    for (int e = vb * blockDim.x + threadIdx.x; e < RR; e += GR_ENTRIES * step) {
      double v[GR_ENTRIES];
#pragma unroll
      for (int k = 0; k < GR_ENTRIES; ++k) v[k] = 0.0;
#pragma unroll 4
      for (int b = 0; b < nblocks; ++b) {
        const double* pb = part + (int64_t)b * RR + e;
#pragma unroll
        for (int k = 0; k < GR_ENTRIES; ++k)
          if (e + k * step < RR) v[k] += pb[k * step];
      }
#pragma unroll
      for (int k = 0; k < GR_ENTRIES; ++k)
        if (e + k * step < RR) G[e + k * step] = v[k];
    }
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = (vb * nw + warp) * GR_ENTRIES; e < RR; e += nvb * nw * GR_ENTRIES) {
    double v[GR_ENTRIES];
#pragma unroll
    for (int k = 0; k < GR_ENTRIES; ++k) v[k] = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
      const double* pb = part + (int64_t)b * RR + e;
#pragma unroll
      for (int k = 0; k < GR_ENTRIES; ++k)
        if (e + k < RR) v[k] += pb[k];
    }
#pragma unroll
    for (int k = 0; k < GR_ENTRIES; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(SPM_FULL_MASK, v[k], o);
      if (lane == 0 && e + k < RR) G[e + k] = v[k];
    }
  }
}

// ---------------------------------------------------------------------------
// Z = M W (double-float), column sums of Z^2 per block.  LPR lanes hold one
// row (LPR = 8, 16 or 32 >= R, or 32 with RPL = 2 for R <= 64), so a warp
// instruction covers 32 / LPR rows and one warp iteration ROWS of those;
// lane (h, rl) owns ranks rl + LPR j (j < RPL) of its rows.  A row's sum
// over the ranks has the same order for every LPR.
// ---------------------------------------------------------------------------
template <int RPL, int LPR = 32>
__device__ __forceinline__ void solve_body(const float* __restrict__ M,
                                           const float* __restrict__ winv, int64_t I, int R,
                                           float* __restrict__ Z, double* __restrict__ colsq_part,
                                           const int* __restrict__ err, int vb, int nvb,
                                           const uint32_t* __restrict__ mask) {
  static_assert(LPR == 32 || RPL == 1, "narrow rows take one rank per lane");
  constexpr int ROWS = 4;
  constexpr int RPR = 32 / LPR;         // rows side by side in one warp instruction
  constexpr int GROUP = ROWS * RPR;     // rows per warp iteration
  __shared__ double red[ALS_THREADS / 32][32 * RPL];
  __shared__ float2 w_s[(32 * RPL) * (32 * RPL)];  // V^{-1} as (hi, lo) pairs
  if (*err) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = lane / LPR, rl = lane % LPR;  // row within the instruction, rank slot
  const int RR = R * R;
  for (int e = threadIdx.x; e < RR; e += ALS_THREADS) w_s[e] = make_float2(winv[e], winv[RR + e]);
  __syncthreads();
  const int64_t gwarp = (int64_t)vb * (ALS_THREADS / 32) + warp;
  const int64_t nwarps = (int64_t)nvb * (ALS_THREADS / 32);
  df sq[RPL];
#pragma unroll
  for (int j = 0; j < RPL; ++j) sq[j] = {0.f, 0.f};
  for (int64_t i0 = gwarp * GROUP; i0 < I; i0 += nwarps * GROUP) {
    if (mask) {  // a group of empty rows: Z is not written (scale_body reads no Z there)
      // i0 is a multiple of GROUP (4, 8 or 16), so the group's bits share one
      // word; bits past the last row are clear
      const uint32_t bits = __ldg(&mask[i0 >> 5]) >> (i0 & 31);
      if ((bits & ((1u << GROUP) - 1u)) == 0u) continue;
    }
    df acc[ROWS][RPL];
#pragma unroll
    for (int q = 0; q < ROWS; ++q)
#pragma unroll
      for (int j = 0; j < RPL; ++j) acc[q][j] = {0.f, 0.f};
    // lane (h, rl) holds M(i0 + q RPR + h, rl + LPR c); broadcast by shuffles below
    float mrow[ROWS][RPL];
#pragma unroll
    for (int q = 0; q < ROWS; ++q)
#pragma unroll
      for (int c = 0; c < RPL; ++c) {
        const int64_t row = i0 + q * RPR + h;
        const int s = rl + LPR * c;
        mrow[q][c] = (row < I && s < R) ? M[row * R + s] : 0.f;
      }
#pragma unroll
    for (int c = 0; c < RPL; ++c) {
      const int send = min(LPR, R - LPR * c);
      for (int sl = 0; sl < send; ++sl) {
        const int s = LPR * c + sl;
        float m[ROWS];
#pragma unroll
        for (int q = 0; q < ROWS; ++q) m[q] = __shfl_sync(SPM_FULL_MASK, mrow[q][c], (lane & ~(LPR - 1)) | sl);
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
          const int r = rl + LPR * j;
          if (r < R) {
            const float2 w = w_s[s * R + r];
#pragma unroll
            for (int q = 0; q < ROWS; ++q) df_add_prod2(acc[q][j], m[q], w.x, w.y);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      const int64_t row = i0 + q * RPR + h;
      if (row >= I) break;
#pragma unroll
      for (int j = 0; j < RPL; ++j) {
        const int r = rl + LPR * j;
        if (r < R) {
          const float z = __fadd_rn(acc[q][j].hi, acc[q][j].lo);
          Z[row * R + r] = z;
          df_add_prod(sq[j], z, z);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < RPL; ++j) red[warp][lane + 32 * j] = df_value(sq[j]);
  __syncthreads();
  // column r is held by lanes r + LPR h' (h' < RPR) of every warp
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < ALS_THREADS / 32; ++w)
      for (int hh = 0; hh < RPR; ++hh) s += red[w][r + LPR * hh];
    colsq_part[(int64_t)vb * R + r] = s;
  }
}

// Scale exponent g of a column of the new factor for the tensor-core Gram:
// |Y(i, r)| < 2^(g - 1) for Y = Z / lambda rounded to FP32 or BF16, from the
// column's max |Z| (0 for a zero column).
__device__ __forceinline__ int gram_scale_exp(float cmax, double lam) {
  const float inv = lam > 0.0 ? (float)(1.0 / lam) : 1.f;
  const double b = (double)cmax * (double)inv * (1.0 + 1.0 / 128.0);
  if (!(b > 0.0)) return 0;
  int e;
  (void)frexp(b, &e);  // b < 2^e
  return e + 1;
}

// lambda(r) = sqrt(sum of the column-r partials of Z^2) and, when
// colmax_part is non-null, lambda(R + r) = the Gram scale exponent of column r
// -- one warp per column (FP64 work spread over blocks: the FP64 pipe of one
// SM would serialise a whole mode's columns).
__device__ __forceinline__ void lambda_body(const double* __restrict__ colsq_part,
                                            const float* __restrict__ colmax_part, int nblocks,
                                            int R, double* __restrict__ lambda,
                                            const int* __restrict__ err, int r) {
  if (warp_err(err) || r >= R) return;
  const int lane = threadIdx.x & 31;
  double v;
  if (nblocks <= ALS_SERIAL_PARTIALS) {
    v = 0.0;
    if (lane == 0)
      for (int b = 0; b < nblocks; ++b) v += colsq_part[(int64_t)b * R + r];
  } else {
    v = warp_sum_strided(colsq_part + r, nblocks, R, lane);
  }
  int mb = 0;  // max |Z| as the bits of a non-negative float
  if (colmax_part) {
    for (int b = lane; b < nblocks; b += 32) mb = max(mb, __float_as_int(colmax_part[(int64_t)b * R + r]));
    mb = __reduce_max_sync(SPM_FULL_MASK, mb);
  }
  if (lane == 0) {
    lambda[r] = sqrt(v);
    if (colmax_part) lambda[R + r] = (double)gram_scale_exp(__int_as_float(mb), lambda[r]);
  }
}

// Y_d = Z / lambda (stored type FT); optionally sums M .* Y per column.
template <typename FT>
__device__ __forceinline__ void scale_body(const float* __restrict__ Z,
                                           const double* __restrict__ lambda, int64_t I, int R,
                                           FT* __restrict__ Y, const float* __restrict__ M,
                                           double* __restrict__ inner_part,
                                           const int* __restrict__ err, int vb, int nvb,
                                           const uint32_t* __restrict__ mask) {
  __shared__ double red[ALS_THREADS];
  if (*err) return;
  // each thread walks a fixed rank r = t % R over rows (t / R) + k * stride
  // (requires R <= ALS_THREADS)
  const int per = ALS_THREADS / R;
  const int r = threadIdx.x % R;
  const int sub = threadIdx.x / R;
  const bool active = sub < per;
  const double lam = lambda[r];
  const float inv = lam > 0.0 ? (float)(1.0 / lam) : 1.f;
  df in = {0.f, 0.f};
  if (active) {
    const int64_t stride = (int64_t)nvb * per;
    for (int64_t i = (int64_t)vb * per + sub; i < I; i += stride) {
      const bool lv = row_live(mask, i);
      const float z = lv ? Z[i * R + r] : 0.f;
      const float y = lam > 0.0 ? z * inv : z;
      const FT ys = store_cvt<FT>(y);
      Y[i * R + r] = ys;
      if (M && lv) df_add_prod(in, M[i * R + r], load_f<FT>(&ys, 0));
    }
  }
  if (!M) return;
  red[threadIdx.x] = active ? df_value(in) : 0.0;
  __syncthreads();
  if (threadIdx.x < R) {
    double s = 0.0;
    for (int q = 0; q < per; ++q) s += red[q * R + threadIdx.x];
    inner_part[(int64_t)vb * R + threadIdx.x] = s;
  }
}

// fit from |X|^2, lambda, all Grams and the inner-product partials.
__device__ __forceinline__ void fit_body(const double* __restrict__ grams, int N, int R,
                                         const double* __restrict__ lambda,
                                         const double* __restrict__ inner_part, int nblocks,
                                         const double* __restrict__ normX2,
                                         double* __restrict__ fit, double* __restrict__ lambda_out,
                                         const int* __restrict__ err) {
  __shared__ double red[ALS_THREADS];
  __shared__ double red2[ALS_THREADS];
  const int RR = R * R;
  double xh = 0.0, inn = 0.0;
  const bool bad = warp_err(err) != 0;
  if (!bad) {
    for (int e = threadIdx.x; e < RR; e += blockDim.x) {
      double h = 1.0;
      for (int w = 0; w < N; ++w) h = __dmul_rn(h, grams[(int64_t)w * RR + e]);
      xh = fma(__dmul_rn(lambda[e / R], lambda[e % R]), h, xh);
    }
    if (nblocks <= ALS_SERIAL_PARTIALS) {
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += inner_part[(int64_t)b * R + r];
        inn = fma(lambda[r], v, inn);
        lambda_out[r] = lambda[r];
      }
    } else {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int r = warp; r < R; r += nw) {
        const double v = warp_sum_strided(inner_part + r, nblocks, R, lane);
        if (lane == 0) {
          inn = fma(lambda[r], v, inn);
          lambda_out[r] = lambda[r];
        }
      }
    }
  }
  red[threadIdx.x] = xh;
  red2[threadIdx.x] = inn;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x] += red[threadIdx.x + o];
      red2[threadIdx.x] += red2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && fit && !bad) {
    const double nx = *normX2;
    double res = fma(-2.0, red2[0], __dadd_rn(nx, red[0]));
    if (res < 0.0) res = 0.0;
    *fit = nx > 0.0 ? 1.0 - sqrt(res) / sqrt(nx) : 1.0;
  }
}

__device__ __forceinline__ void copy_lambda_body(const double* __restrict__ src, int R,
                                                 double* __restrict__ dst,
                                                 const int* __restrict__ err) {
  if (*err) return;
  for (int r = threadIdx.x; r < R; r += blockDim.x) dst[r] = src[r];
}


__host__ __device__ inline int gram_tile(int R) { return R <= 16 ? 1 : R <= 32 ? 2 : R <= 64 ? 4 : 0; }

// Virtual blocks of a row pass over I rows: at least rows_per_block_min rows
// each, at most cap blocks.
inline int work_blocks(int64_t I, int64_t rows_per_block_min, int cap) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(cap, ceil_div<int64_t>(I, rows_per_block_min)));
}

// The block split of every row pass of a mode with I rows (Gram partials,
// solve, scale).  A function of I and the plan's cap only, so that a tensor's
// sums are grouped the same way alone and in a batch.
inline int als_row_blocks(int64_t I, int cap) { return work_blocks(I, ALS_MIN_ROWS, cap); }

}  // namespace spm
