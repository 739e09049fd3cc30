// plan.cu -- building the mode-specific tensor copies and their partitions.
//
// Sec. III-C keeps one COO copy of the tensor per output mode d, ordered for
// that mode; Sec. III-B2 orders the nonzeros by the output-mode index and
// Sec. III-B1 / III-B2 split them into kappa partitions, one per SM.
//
// Ordering used for copy d: (c_d, then c_w for w != d in ascending w, then the
// input position), i.e. a stable sort.  It is built with a device LSD radix
// sort:
//   * copy 0: the full lexicographic key (c_0, c_1, ..., c_{N-1}) packed into
//     64-bit words (several words, least significant first, when the index
//     bits exceed 64), 8-bit digits, stable passes, payload = input position;
//   * copy d >= 1: a stable sort of copy 0 by c_d alone.  Among nonzeros with
//     equal c_d, copy 0's order is lexicographic on the remaining modes in
//     ascending order, which is exactly the tie-break of copy d.
// Records of copy d hold [c_d, other indices ascending, value bits, padding].
#include <algorithm>
#include <vector>

#include "plan.cuh"

namespace spm {
namespace {

constexpr int RS_WARPS = 8;
constexpr int RS_THREADS = RS_WARPS * 32;  // == RS_BINS (used by the scan)
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_BINS = 256;

struct IdxPtrs {
  const int32_t* p[SPM_MAX_MODES];
};

// ---------------------------------------------------------------------------
// LSD radix sort of (key, int32 payload) pairs, 8 bits per pass, stable.
// ---------------------------------------------------------------------------

template <typename K>
__global__ void __launch_bounds__(RS_THREADS)
    rs_hist_kernel(const K* __restrict__ keys, int64_t n, int shift,
                   uint32_t* __restrict__ hist, int nblocks) {
  __shared__ uint32_t cnt[RS_BINS];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (32 * RS_ITEMS);
#pragma unroll 4
  for (int i = 0; i < RS_ITEMS; ++i) {
    const int64_t k = wbase + i * 32 + lane;
    const unsigned d = k < n ? (unsigned)((keys[k] >> shift) & (RS_BINS - 1)) : RS_BINS;
    const unsigned peers = __match_any_sync(SPM_FULL_MASK, d);
    if (d < RS_BINS && (__ffs(peers) - 1) == lane) atomicAdd(&cnt[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// One block per digit: exclusive scan of hist[d][0..nblocks) in place and the
// digit total into dtot[d].
__global__ void __launch_bounds__(1024)
    rs_scan_rows_kernel(uint32_t* __restrict__ hist, int nblocks, uint32_t* __restrict__ dtot) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  uint32_t* row = hist + (int64_t)blockIdx.x * nblocks;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblocks; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < nblocks ? row[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(SPM_FULL_MASK, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t s = lane < nwarps ? wsum[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(SPM_FULL_MASK, s, o);
        if (lane >= o) s += y;
      }
      wsum[lane] = s;
    }
    __syncthreads();
    const uint32_t excl = carry + (warp ? wsum[warp - 1] : 0u) + x - v;
    if (i < nblocks) row[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) dtot[blockIdx.x] = carry;
}

template <typename K>
__global__ void __launch_bounds__(RS_THREADS)
    rs_scatter_kernel(const K* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
                      K* __restrict__ keys_out, int32_t* __restrict__ vals_out, int64_t n,
                      int shift, const uint32_t* __restrict__ hist, const uint32_t* __restrict__ dtot,
                      int nblocks) {
  __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];
  __shared__ uint32_t gbase[RS_BINS];
  __shared__ uint32_t wsum[RS_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < RS_WARPS * RS_BINS; t += RS_THREADS) (&wcnt[0][0])[t] = 0;
  {
    // gbase[d] = sum_{d' < d} dtot[d'] + hist[d][block]   (block exclusive scan)
    const uint32_t v = dtot[threadIdx.x];
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(SPM_FULL_MASK, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < warp; ++w) pre += wsum[w];
    gbase[threadIdx.x] = pre + x - v + hist[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  }
  __syncthreads();
  K key[RS_ITEMS];
  int32_t val[RS_ITEMS];
  uint32_t lrank[RS_ITEMS];
  const unsigned lt = (1u << lane) - 1u;
  const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (32 * RS_ITEMS);
#pragma unroll
  for (int i = 0; i < RS_ITEMS; ++i) {
    const int64_t k = wbase + i * 32 + lane;
    const bool valid = k < n;
    key[i] = valid ? keys_in[k] : K(0);
    val[i] = valid ? vals_in[k] : 0;
    const unsigned d = valid ? (unsigned)((key[i] >> shift) & (RS_BINS - 1)) : RS_BINS;
    const unsigned peers = __match_any_sync(SPM_FULL_MASK, d);
    const uint32_t r = __popc(peers & lt);
    uint32_t b = 0;
    if (valid) b = wcnt[warp][d];
    __syncwarp();
    lrank[i] = b + r;
    if (valid && r == 0) wcnt[warp][d] = b + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      const uint32_t c = wcnt[w][threadIdx.x];
      wcnt[w][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < RS_ITEMS; ++i) {
    const int64_t k = wbase + i * 32 + lane;
    if (k < n) {
      const unsigned d = (unsigned)((key[i] >> shift) & (RS_BINS - 1));
      const uint32_t pos = gbase[d] + wcnt[warp][d] + lrank[i];
      keys_out[pos] = key[i];
      vals_out[pos] = val[i];
    }
  }
}

struct SortScratch {
  uint32_t* hist = nullptr;
  uint32_t* dtot = nullptr;
};

// Sorts (keys, vals) by the low `bits` bits of the keys, stably.  The result
// ends in (keys, vals) (buffers are swapped internally as needed).
template <typename K>
spm_status radix_sort_pairs(K*& keys, int32_t*& vals, K*& keys_alt, int32_t*& vals_alt,
                            int64_t n, int bits, const SortScratch& sc, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return SPM_OK;
  const int nblocks = (int)ceil_div<int64_t>(n, RS_TILE);
  for (int shift = 0; shift < bits; shift += 8) {
    rs_hist_kernel<K><<<nblocks, RS_THREADS, 0, s>>>(keys, n, shift, sc.hist, nblocks);
    rs_scan_rows_kernel<<<RS_BINS, 1024, 0, s>>>(sc.hist, nblocks, sc.dtot);
    rs_scatter_kernel<K><<<nblocks, RS_THREADS, 0, s>>>(keys, vals, keys_alt, vals_alt, n, shift,
                                                        sc.hist, sc.dtot, nblocks);
    SPM_CUDA_TRY(cudaGetLastError());
    std::swap(keys, keys_alt);
    std::swap(vals, vals_alt);
  }
  return SPM_OK;
}

// ---------------------------------------------------------------------------
// Small element-wise kernels.
// ---------------------------------------------------------------------------

__global__ void validate_kernel(IdxPtrs idx, int nmodes, const int64_t* __restrict__ dims,
                                int64_t n, int* __restrict__ err) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    bool bad = false;
    for (int w = 0; w < nmodes; ++w) {
      const int32_t c = idx.p[w][k];
      bad |= (c < 0) || ((int64_t)c >= dims[w]);
    }
    if (bad) atomicOr(err, DEV_ERR_INDEX);
  }
}

__global__ void iota_kernel(int32_t* __restrict__ a, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    a[k] = (int32_t)k;
}

// key[k] = packed (c_lo, ..., c_hi) of input position perm[k] (identity if
// perm == nullptr); mode w occupies bits [shift[w], shift[w] + bits[w]).
struct PackSpec {
  int lo, hi;
  int shift[SPM_MAX_MODES];
};

__global__ void pack_keys_kernel(IdxPtrs idx, PackSpec spec, const int32_t* __restrict__ perm,
                                 int64_t n, unsigned long long* __restrict__ key) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = perm ? perm[k] : k;
    unsigned long long v = 0;
    for (int w = spec.lo; w <= spec.hi; ++w)
      v |= (unsigned long long)(uint32_t)idx.p[w][src] << spec.shift[w];
    key[k] = v;
  }
}

// Copy-0 records from the input arrays: [c_0, ..., c_{N-1}, val, 0...].
template <int RI>
__global__ void records_from_input_kernel(IdxPtrs idx, const float* __restrict__ vals,
                                          const int32_t* __restrict__ perm, int nmodes,
                                          int64_t n, int4* __restrict__ rec) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = perm[k];
    int words[4 * RI];
#pragma unroll
    for (int j = 0; j < 4 * RI; ++j) words[j] = 0;
#pragma unroll
    for (int w = 0; w < SPM_MAX_MODES && w < 4 * RI; ++w)
      if (w < nmodes) words[w] = idx.p[w][src];
    // value bits right after the indices
#pragma unroll
    for (int j = 0; j < 4 * RI; ++j)
      if (j == nmodes) words[j] = __float_as_int(vals[src]);
#pragma unroll
    for (int q = 0; q < RI; ++q)
      rec[k * RI + q] = make_int4(words[4 * q], words[4 * q + 1], words[4 * q + 2], words[4 * q + 3]);
  }
}

// key[k] = word `d` of the copy-0 record k (that is c_d in copy-0 order).
template <int RI>
__global__ void key_from_records_kernel(const int4* __restrict__ rec, int d, int64_t n,
                                        uint32_t* __restrict__ key) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int* w = reinterpret_cast<const int*>(rec + k * RI);
    key[k] = (uint32_t)w[d];
  }
}

// Copy-d record k from copy-0 record rel[k]: rotate c_d to the front,
// keep the others in ascending mode order; perm_d[k] = perm_0[rel[k]].
template <int RI>
__global__ void records_from_copy0_kernel(const int4* __restrict__ rec0,
                                          const int32_t* __restrict__ perm0,
                                          const int32_t* __restrict__ rel, int nmodes, int d,
                                          int64_t n, int4* __restrict__ recd,
                                          int32_t* __restrict__ permd) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = rel[k];
    int in[4 * RI], out[4 * RI];
#pragma unroll
    for (int q = 0; q < RI; ++q) {
      const int4 v = rec0[src * RI + q];
      in[4 * q] = v.x; in[4 * q + 1] = v.y; in[4 * q + 2] = v.z; in[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int j = 0; j < 4 * RI; ++j) out[j] = in[j];
    // words 0..d of copy d are (c_d, c_0, ..., c_{d-1}); words > d unchanged.
    if (d > 0) {
      int cd = 0;
#pragma unroll
      for (int j = 0; j < 4 * RI; ++j)
        if (j == d) cd = in[j];
#pragma unroll
      for (int j = 4 * RI - 1; j >= 1; --j)
        if (j <= d) out[j] = in[j - 1];
      out[0] = cd;
    }
#pragma unroll
    for (int q = 0; q < RI; ++q)
      recd[k * RI + q] = make_int4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
    permd[k] = perm0[src];
  }
}

// Gather records and permutation of one copy through rel (in -> out).
template <int RI>
__global__ void reorder_copy_kernel(const int4* __restrict__ rec_in, const int32_t* __restrict__ perm_in,
                                    const int32_t* __restrict__ rel, int64_t n,
                                    int4* __restrict__ rec_out, int32_t* __restrict__ perm_out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = rel[k];
#pragma unroll
    for (int q = 0; q < RI; ++q) rec_out[k * RI + q] = rec_in[src * RI + q];
    perm_out[k] = perm_in[src];
  }
}

// Scheme 2 offsets floor(z*nnz/kappa).
__global__ void equal_offsets_kernel(int64_t nnz, int kappa, int64_t* __restrict__ off) {
  for (int z = blockIdx.x * blockDim.x + threadIdx.x; z <= kappa; z += gridDim.x * blockDim.x)
    off[z] = ((int64_t)z * nnz) / kappa;
}

// Row degree from the runs of equal c_d in a copy sorted by c_d.
template <int RI>
__global__ void row_degree_kernel(const int4* __restrict__ rec, int64_t n,
                                  int32_t* __restrict__ deg) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int c = rec[k * RI].x;
    const bool start = (k == 0) || rec[(k - 1) * RI].x != c;
    if (start) {
      // run length by galloping then binary search over the sorted rows
      int64_t lo = k, step = 1, hi = k + 1;
      while (hi < n && rec[hi * RI].x == c) {
        lo = hi;
        hi = k + (step <<= 1);
      }
      if (hi > n) hi = n;
      // rec[lo].x == c, and rec[hi].x != c or hi == n
      while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (rec[mid * RI].x == c) lo = mid; else hi = mid;
      }
      deg[c] = (int32_t)(hi - k);
    }
  }
}

// Key that orders rows by (degree descending, index ascending); empty rows last.
__global__ void row_order_key_kernel(const int32_t* __restrict__ deg, int64_t I,
                                     unsigned long long* __restrict__ key,
                                     int32_t* __restrict__ row) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t dg = (uint32_t)deg[i];
    key[i] = dg ? ((unsigned long long)(0xFFFFFFFFu - dg) << 32) | (unsigned long long)i
                : ~0ull;
    row[i] = (int32_t)i;
  }
}

// Cyclic deal: the t-th row in degree order goes to partition t mod kappa.
__global__ void deal_rows_kernel(const int32_t* __restrict__ row_sorted,
                                 const int32_t* __restrict__ deg, int64_t I, int kappa,
                                 int32_t* __restrict__ part) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < I;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = row_sorted[t];
    part[r] = deg[r] ? (int32_t)(t % kappa) : -1;
  }
}

template <int RI>
__global__ void part_key_kernel(const int4* __restrict__ rec, const int32_t* __restrict__ part,
                                int64_t n, uint32_t* __restrict__ key) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    key[k] = (uint32_t)part[rec[k * RI].x];
}

// off[z] = first position whose (sorted) key is >= z.
__global__ void lower_bound_offsets_kernel(const uint32_t* __restrict__ key, int64_t n,
                                           int kappa, int64_t* __restrict__ off) {
  for (int z = blockIdx.x * blockDim.x + threadIdx.x; z <= kappa; z += gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (key[mid] < (uint32_t)z) lo = mid + 1; else hi = mid;
    }
    off[z] = lo;
  }
}

// |X|^2 over copy 0 (fully sorted, so repeated coordinates are adjacent and
// are summed before squaring).  Block partials in FP64, fixed order.
template <int RI>
__global__ void __launch_bounds__(256)
    norm_partial_kernel(const int4* __restrict__ rec, int nmodes, int64_t n,
                        double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int* w = reinterpret_cast<const int*>(rec + k * RI);
    bool start = (k == 0);
    if (!start) {
      const int* p = reinterpret_cast<const int*>(rec + (k - 1) * RI);
      for (int j = 0; j < nmodes; ++j) start |= (w[j] != p[j]);
    }
    if (!start) continue;
    double cell = (double)__int_as_float(w[nmodes]);
    for (int64_t q = k + 1; q < n; ++q) {
      const int* x = reinterpret_cast<const int*>(rec + q * RI);
      bool same = true;
      for (int j = 0; j < nmodes; ++j) same &= (x[j] == w[j]);
      if (!same) break;
      cell += (double)__int_as_float(x[nmodes]);
    }
    acc += cell * cell;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

// ---- work units -----------------------------------------------------------

// Scheme 1 / Scheme 2: unit w of partition z starts at
// off[z] + floor((off[z+1] - off[z]) * w / units).
__global__ void units_from_partitions_kernel(const int64_t* __restrict__ off, int kappa, int units,
                                             int64_t* __restrict__ woff) {
  const int64_t P = (int64_t)kappa * units;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= P;
       j += (int64_t)gridDim.x * blockDim.x) {
    if (j == P) {
      woff[j] = off[kappa];
    } else {
      const int z = (int)(j / units), w = (int)(j % units);
      woff[j] = off[z] + ((off[z + 1] - off[z]) * w) / units;
    }
  }
}

__global__ void partitions_from_units_kernel(const int64_t* __restrict__ woff, int kappa, int units,
                                             int64_t* __restrict__ off) {
  for (int z = blockIdx.x * blockDim.x + threadIdx.x; z <= kappa; z += gridDim.x * blockDim.x)
    off[z] = woff[(int64_t)z * units];
}

// Row starts per tile of RS_TILE copy positions.  The row of copy position k
// is rows[k * stride] (a copy's records, or a gathered key array).
__global__ void __launch_bounds__(RS_THREADS)
    head_count_kernel(const int* __restrict__ rows, int64_t stride, int64_t n,
                      uint32_t* __restrict__ bsum) {
  __shared__ uint32_t red[RS_THREADS];
  const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
  uint32_t c = 0;
  for (int i = 0; i < RS_ITEMS; ++i) {
    const int64_t k = base + i;
    if (k < n) c += (k == 0 || rows[k * stride] != rows[(k - 1) * stride]) ? 1u : 0u;
  }
  red[threadIdx.x] = c;
  __syncthreads();
  for (int o = RS_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = red[0];
}

// heads_before[k] = number of row starts at positions < k (bsum scanned).
__global__ void __launch_bounds__(RS_THREADS)
    head_prefix_kernel(const int* __restrict__ rows, int64_t stride, int64_t n,
                       const uint32_t* __restrict__ bexcl, uint32_t* __restrict__ before) {
  __shared__ uint32_t sc[RS_THREADS];
  const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
  uint32_t c = 0;
  for (int i = 0; i < RS_ITEMS; ++i) {
    const int64_t k = base + i;
    if (k < n) c += (k == 0 || rows[k * stride] != rows[(k - 1) * stride]) ? 1u : 0u;
  }
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = 1; o < RS_THREADS; o <<= 1) {  // inclusive Hillis-Steele scan
    const uint32_t t = threadIdx.x >= o ? sc[threadIdx.x - o] : 0u;
    __syncthreads();
    sc[threadIdx.x] += t;
    __syncthreads();
  }
  uint32_t run = bexcl[blockIdx.x] + sc[threadIdx.x] - c;
  for (int i = 0; i < RS_ITEMS; ++i) {
    const int64_t k = base + i;
    if (k < n) {
      before[k] = run;
      run += (k == 0 || rows[k * stride] != rows[(k - 1) * stride]) ? 1u : 0u;
    }
  }
}

// woff[j] = min{k in [0, n] : C(k) * P >= j * C(n)},
// C(k) = k + row_cost * before[k], C(n) = n + row_cost * total_heads.
__global__ void balanced_units_kernel(const uint32_t* __restrict__ before,
                                      const uint32_t* __restrict__ total_heads, int64_t n,
                                      int64_t P, int row_cost, int64_t* __restrict__ woff) {
  const int64_t Ct = n + (int64_t)row_cost * (int64_t)(*total_heads);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= P;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t target = j * Ct;  // compare C(k) * P >= target
    int64_t lo = 0, hi = n;         // C(n) * P >= target always holds
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      const int64_t C = mid + (int64_t)row_cost * (int64_t)before[mid];
      if (C * P >= target) hi = mid; else lo = mid + 1;
    }
    woff[j] = lo;
  }
}

// Bitmap of non-empty output rows of a copy (rows[k * stride] is the row of
// copy position k; every nonzero sets its row's bit).
__global__ void row_mask_kernel(const int* __restrict__ rows, int64_t stride, int64_t n,
                                uint32_t* __restrict__ mask) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int r = rows[k * stride];
    if (k == 0 || rows[(k - 1) * stride] != r) atomicOr(&mask[r >> 5], 1u << (r & 31));
  }
}

// Lean copy d: row of each copy position, gathered from copy 0 (word d of
// the copy-0 record is c_d).
__global__ void gather_rows_kernel(const int* __restrict__ rec0, int64_t words, const int32_t* __restrict__ src,
                                   int d, int64_t n, int* __restrict__ rows) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    rows[k] = rec0[(int64_t)src[k] * words + d];
}

__global__ void popc_kernel(const uint32_t* __restrict__ mask, int64_t words,
                            unsigned long long* __restrict__ count) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
       i += (int64_t)gridDim.x * blockDim.x)
    c += __popc(mask[i]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(SPM_FULL_MASK, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

int grid_for(int64_t n, int threads) {
  const int64_t b = ceil_div<int64_t>(n > 0 ? n : 1, threads);
  return (int)std::min<int64_t>(b, 152 * 32);
}

int bits_for(int64_t dim) {
  int b = 0;
  while (b < 63 && ((int64_t)1 << b) < dim) ++b;
  return b;  // enough bits for values 0..dim-1
}

constexpr int NORM_BLOCKS = 1024;

// The rows of copy d in copy order as (pointer, stride): the copy's records,
// or for a lean copy a key array gathered into `scratch` (>= nnz ints).
const int* copy_rows(spmttkrp_plan_s* p, int d, int* scratch, int64_t* stride, cudaStream_t s) {
  const int RI = record_int4s(p->N);
  if (!p->lean || d == 0) {
    *stride = 4 * RI;
    return reinterpret_cast<const int*>(p->mode[d].rec);
  }
  const int64_t n = p->nnz;
  gather_rows_kernel<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const int*>(p->mode[0].rec),
                                                     4 * RI, p->mode[d].src, d, n, scratch);
  *stride = 1;
  return scratch;
}

// P2 for a copy under the cost-balanced policy (scheme 0) or Scheme 2, and
// for an empty tensor under any policy: partition offsets off[0..kappa] and
// work-unit offsets woff[0..kappa*nu].  rows/stride: the copy's rows in copy
// order.  Scratch: hist >= ceil(nnz/RS_TILE) words, dtot >= 1 word,
// before >= nnz words.
void partition_copy(spmttkrp_plan_s* p, int d, const int* rows, int64_t stride, uint32_t* hist,
                    uint32_t* dtot, uint32_t* before, cudaStream_t s) {
  const int T = 256;
  const int64_t n = p->nnz;
  const int units = p->nu;
  const int64_t P = (int64_t)p->kappa * units;
  spm_mode_copy& c = p->mode[d];
  if (c.scheme == 0 && n > 0) {
    // cost-balanced work units over the copy order
    const int nb = (int)ceil_div<int64_t>(n, RS_TILE);
    head_count_kernel<<<nb, RS_THREADS, 0, s>>>(rows, stride, n, hist);
    rs_scan_rows_kernel<<<1, 1024, 0, s>>>(hist, nb, dtot);
    head_prefix_kernel<<<nb, RS_THREADS, 0, s>>>(rows, stride, n, hist, before);
    balanced_units_kernel<<<grid_for(P + 1, T), T, 0, s>>>(before, dtot, n, P, SPM_ROW_COST,
                                                          c.woff);
    partitions_from_units_kernel<<<grid_for(p->kappa + 1, T), T, 0, s>>>(c.woff, p->kappa,
                                                                        units, c.off);
    return;
  }
  equal_offsets_kernel<<<grid_for(p->kappa + 1, T), T, 0, s>>>(n, p->kappa, c.off);
  units_from_partitions_kernel<<<grid_for(P + 1, T), T, 0, s>>>(c.off, p->kappa, units, c.woff);
}

// Entries of the build's sort scratch: the nonzeros, or the rows of the
// longest mode when some mode is partitioned by Scheme 1 (its rows are
// sorted by degree); policy is SPM_POLICY_* >> 4.
int64_t sort_capacity(int N, const int64_t* dims, int64_t nn, int policy, int kappa) {
  int64_t rows = 0;
  for (int w = 0; w < N; ++w) {
    const bool scheme1 = policy == (int)(SPM_POLICY_SCHEME1 >> 4) ||
                         (policy == (int)(SPM_POLICY_ADAPTIVE >> 4) && dims[w] >= kappa);
    if (scheme1) rows = std::max(rows, dims[w]);
  }
  return std::max(nn, rows);
}

template <int RI>
spm_status build_copies_t(spmttkrp_plan_s* p, const int32_t* const* idx_in, const float* vals,
                          cudaStream_t s) {
  const int N = p->N;
  const int64_t n = p->nnz;
  IdxPtrs idx{};
  for (int w = 0; w < N; ++w) idx.p[w] = idx_in[w];
  const int T = 256;
  const int G = grid_for(n, T);

  // scratch (stream-ordered, freed at the end)
  unsigned long long *k64a = nullptr, *k64b = nullptr;
  int32_t *va = nullptr, *vb = nullptr;
  SortScratch sc;
  int64_t* d_dims = nullptr;
  const int64_t nn = n > 0 ? n : 1;
  // the keys, payloads and histograms hold nnz entries, or I_d entries where
  // Scheme 1 sorts the rows of a mode by degree
  const int64_t cap = sort_capacity(N, p->dims, nn, p->policy, p->kappa);
  const int nblocks_max = (int)ceil_div<int64_t>(cap, RS_TILE);
  SPM_CUDA_TRY(cudaMallocAsync((void**)&k64a, sizeof(unsigned long long) * cap, s));
  SPM_CUDA_TRY(cudaMallocAsync((void**)&k64b, sizeof(unsigned long long) * cap, s));
  SPM_CUDA_TRY(cudaMallocAsync((void**)&va, sizeof(int32_t) * cap, s));
  SPM_CUDA_TRY(cudaMallocAsync((void**)&vb, sizeof(int32_t) * cap, s));
  SPM_CUDA_TRY(cudaMallocAsync((void**)&sc.hist, sizeof(uint32_t) * RS_BINS * (size_t)nblocks_max, s));
  SPM_CUDA_TRY(cudaMallocAsync((void**)&sc.dtot, sizeof(uint32_t) * RS_BINS, s));
  SPM_CUDA_TRY(cudaMallocAsync((void**)&d_dims, sizeof(int64_t) * SPM_MAX_MODES, s));
  SPM_CUDA_TRY(cudaMemcpyAsync(d_dims, p->dims, sizeof(int64_t) * N, cudaMemcpyHostToDevice, s));

  // Validation: every index within its dimension.
  if (n > 0) validate_kernel<<<G, T, 0, s>>>(idx, N, d_dims, n, p->dev_err);
  int herr = 0;
  SPM_CUDA_TRY(cudaMemcpyAsync(&herr, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  spm_status st = SPM_OK;
  if (herr & DEV_ERR_INDEX) st = SPM_ERR_INDEX_OUT_OF_RANGE;

  // Allocate the copies (a lean copy: positions into copy 0, padded by 16
  // bytes so that 16-byte-aligned bulk copies of any range stay inside).
  for (int d = 0; d < N && st == SPM_OK; ++d) {
    if (p->lean && d > 0) {
      st = plan_alloc(p, (void**)&p->mode[d].src, sizeof(int32_t) * (size_t)nn + 16);
    } else {
      st = plan_alloc(p, (void**)&p->mode[d].rec, sizeof(int4) * RI * (size_t)nn + 256);
      if (st == SPM_OK) st = plan_alloc(p, (void**)&p->mode[d].perm, sizeof(int32_t) * (size_t)nn);
    }
    if (st == SPM_OK)
      st = plan_alloc(p, (void**)&p->mode[d].off, sizeof(int64_t) * (size_t)(p->kappa + 1));
    if (st == SPM_OK)
      st = plan_alloc(p, (void**)&p->mode[d].woff,
                      sizeof(int64_t) * ((size_t)p->kappa * p->nu + 1));
    if (st == SPM_OK)
      st = plan_alloc(p, (void**)&p->mode[d].rowmask,
                      sizeof(uint32_t) * (size_t)((p->dims[d] + 31) / 32));
  }

  if (st == SPM_OK && n > 0) {
    // ---- copy 0: full lexicographic order, least significant key word first.
    int bits[SPM_MAX_MODES];
    for (int w = 0; w < N; ++w) bits[w] = bits_for(p->dims[w]);
    // group modes into <=64-bit words from the last mode backwards
    struct Group { int lo, hi, nbits; };
    std::vector<Group> groups;
    {
      int hi = N - 1, acc = 0, lo = N - 1;
      for (int w = N - 1; w >= 0; --w) {
        if (acc + bits[w] > 64) {
          groups.push_back({w + 1, hi, acc});
          hi = w;
          acc = 0;
        }
        acc += bits[w];
        lo = w;
      }
      groups.push_back({lo, hi, acc});
    }
    // perm in va (identity), keys in k64a
    iota_kernel<<<G, T, 0, s>>>(va, n);
    unsigned long long *ka = k64a, *kb = k64b;
    int32_t *pa = va, *pb = vb;
    for (const Group& g : groups) {  // least significant group first
      PackSpec spec{};
      spec.lo = g.lo;
      spec.hi = g.hi;
      int sh = 0;
      for (int w = g.hi; w >= g.lo; --w) {
        spec.shift[w] = sh;
        sh += bits[w];
      }
      pack_keys_kernel<<<G, T, 0, s>>>(idx, spec, pa, n, ka);
      st = radix_sort_pairs<unsigned long long>(ka, pa, kb, pb, n, g.nbits, sc, s);
      if (st != SPM_OK) break;
    }
    if (st == SPM_OK) {
      spm_mode_copy& c0 = p->mode[0];
      SPM_CUDA_TRY(cudaMemcpyAsync(c0.perm, pa, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
      records_from_input_kernel<RI><<<G, T, 0, s>>>(idx, vals, c0.perm, N, n, c0.rec);
      // |X|^2 (duplicates summed) from copy 0
      norm_partial_kernel<RI><<<NORM_BLOCKS, 256, 0, s>>>(c0.rec, N, n, p->norm_part);
      sum_partials_kernel<<<1, 32, 0, s>>>(p->norm_part, NORM_BLOCKS, p->normX2);
    }
    // ---- copies d >= 1: stable sort of copy 0 by c_d.
    for (int d = 1; d < N && st == SPM_OK; ++d) {
      uint32_t* ka32 = reinterpret_cast<uint32_t*>(k64a);
      uint32_t* kb32 = reinterpret_cast<uint32_t*>(k64b);
      int32_t *ra = va, *rb = vb;
      key_from_records_kernel<RI><<<G, T, 0, s>>>(p->mode[0].rec, d, n, ka32);
      iota_kernel<<<G, T, 0, s>>>(ra, n);
      st = radix_sort_pairs<uint32_t>(ka32, ra, kb32, rb, n, bits[d], sc, s);
      if (st != SPM_OK) break;
      if (p->lean)
        SPM_CUDA_TRY(cudaMemcpyAsync(p->mode[d].src, ra, sizeof(int32_t) * n,
                                     cudaMemcpyDeviceToDevice, s));
      else
        records_from_copy0_kernel<RI><<<G, T, 0, s>>>(p->mode[0].rec, p->mode[0].perm, ra, N, d,
                                                       n, p->mode[d].rec, p->mode[d].perm);
    }
  } else if (st == SPM_OK) {
    SPM_CUDA_TRY(cudaMemsetAsync(p->normX2, 0, sizeof(double), s));
  }

  // ---- partitions (Sec. III-B) and work units
  const int units = p->nu;
  const int64_t P = (int64_t)p->kappa * units;
  for (int d = 0; d < N && st == SPM_OK; ++d) {
    spm_mode_copy& c = p->mode[d];
    int scheme = 0;
    if (p->policy == (int)(SPM_POLICY_SCHEME2 >> 4)) scheme = 2;
    if (p->policy == (int)(SPM_POLICY_SCHEME1 >> 4)) scheme = 1;
    if (p->policy == (int)(SPM_POLICY_ADAPTIVE >> 4)) scheme = p->dims[d] >= p->kappa ? 1 : 2;
    c.scheme = scheme;
    if (scheme != 1 || n == 0) {
      int64_t stride = 0;
      const int* rows = n > 0 ? copy_rows(p, d, reinterpret_cast<int*>(k64b), &stride, s) : nullptr;
      partition_copy(p, d, rows, stride, sc.hist, sc.dtot, reinterpret_cast<uint32_t*>(va), s);
      continue;
    }
    // Scheme 1: degree-ordered cyclic deal of the rows, copy ordered by partition.
    const int64_t I = p->dims[d];
    int32_t* deg = nullptr;
    int32_t* part = nullptr;
    int4* rec_tmp = nullptr;
    int32_t* perm_tmp = nullptr;
    SPM_CUDA_TRY(cudaMallocAsync((void**)&deg, sizeof(int32_t) * I, s));
    SPM_CUDA_TRY(cudaMallocAsync((void**)&part, sizeof(int32_t) * I, s));
    SPM_CUDA_TRY(cudaMallocAsync((void**)&rec_tmp, sizeof(int4) * RI * (size_t)n, s));
    SPM_CUDA_TRY(cudaMallocAsync((void**)&perm_tmp, sizeof(int32_t) * (size_t)n, s));
    SPM_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int32_t) * I, s));
    row_degree_kernel<RI><<<G, T, 0, s>>>(c.rec, n, deg);
    {
      unsigned long long *ka = k64a, *kb = k64b;
      int32_t *ra = va, *rb = vb;
      row_order_key_kernel<<<grid_for(I, T), T, 0, s>>>(deg, I, ka, ra);
      st = radix_sort_pairs<unsigned long long>(ka, ra, kb, rb, I, 64, sc, s);
      if (st == SPM_OK) deal_rows_kernel<<<grid_for(I, T), T, 0, s>>>(ra, deg, I, p->kappa, part);
    }
    if (st == SPM_OK) {
      uint32_t* ka32 = reinterpret_cast<uint32_t*>(k64a);
      uint32_t* kb32 = reinterpret_cast<uint32_t*>(k64b);
      int32_t *ra = va, *rb = vb;
      part_key_kernel<RI><<<G, T, 0, s>>>(c.rec, part, n, ka32);
      iota_kernel<<<G, T, 0, s>>>(ra, n);
      st = radix_sort_pairs<uint32_t>(ka32, ra, kb32, rb, n, bits_for(p->kappa), sc, s);
      if (st == SPM_OK) {
        reorder_copy_kernel<RI><<<G, T, 0, s>>>(c.rec, c.perm, ra, n, rec_tmp, perm_tmp);
        SPM_CUDA_TRY(cudaMemcpyAsync(c.rec, rec_tmp, sizeof(int4) * RI * (size_t)n,
                                     cudaMemcpyDeviceToDevice, s));
        SPM_CUDA_TRY(cudaMemcpyAsync(c.perm, perm_tmp, sizeof(int32_t) * (size_t)n,
                                     cudaMemcpyDeviceToDevice, s));
        lower_bound_offsets_kernel<<<grid_for(p->kappa + 1, T), T, 0, s>>>(ka32, n, p->kappa,
                                                                          c.off);
        units_from_partitions_kernel<<<grid_for(P + 1, T), T, 0, s>>>(c.off, p->kappa, units,
                                                                      c.woff);
      }
    }
    SPM_CUDA_TRY(cudaFreeAsync(deg, s));
    SPM_CUDA_TRY(cudaFreeAsync(part, s));
    SPM_CUDA_TRY(cudaFreeAsync(rec_tmp, s));
    SPM_CUDA_TRY(cudaFreeAsync(perm_tmp, s));
  }
  // ---- non-empty row bitmaps (rows without nonzeros are zeroed per run)
  unsigned long long* d_cnt = nullptr;
  unsigned long long h_cnt[SPM_MAX_MODES] = {};
  if (st == SPM_OK) {
    SPM_CUDA_TRY(cudaMallocAsync((void**)&d_cnt, sizeof(unsigned long long) * SPM_MAX_MODES, s));
    SPM_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * SPM_MAX_MODES, s));
    for (int d = 0; d < N; ++d) {
      const int64_t words = (p->dims[d] + 31) / 32;
      SPM_CUDA_TRY(cudaMemsetAsync(p->mode[d].rowmask, 0, sizeof(uint32_t) * words, s));
      if (n > 0) {
        int64_t stride = 0;
        const int* rows = copy_rows(p, d, reinterpret_cast<int*>(k64b), &stride, s);
        row_mask_kernel<<<G, T, 0, s>>>(rows, stride, n, p->mode[d].rowmask);
      }
      popc_kernel<<<grid_for(words, T), T, 0, s>>>(p->mode[d].rowmask, words, d_cnt + d);
    }
    SPM_CUDA_TRY(cudaMemcpyAsync(h_cnt, d_cnt, sizeof(unsigned long long) * SPM_MAX_MODES,
                                 cudaMemcpyDeviceToHost, s));
    SPM_CUDA_TRY(cudaFreeAsync(d_cnt, s));
  }
  SPM_CUDA_TRY(cudaGetLastError());
  SPM_CUDA_TRY(cudaFreeAsync(k64a, s));
  SPM_CUDA_TRY(cudaFreeAsync(k64b, s));
  SPM_CUDA_TRY(cudaFreeAsync(va, s));
  SPM_CUDA_TRY(cudaFreeAsync(vb, s));
  SPM_CUDA_TRY(cudaFreeAsync(sc.hist, s));
  SPM_CUDA_TRY(cudaFreeAsync(sc.dtot, s));
  SPM_CUDA_TRY(cudaFreeAsync(d_dims, s));
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  for (int d = 0; d < N; ++d) p->mode[d].empty_rows = p->dims[d] - (int64_t)h_cnt[d];
  return st;
}

}  // namespace

void plan_bytes_estimate(int N, const int64_t* dims, int64_t nnz, int R, int kappa, bool als,
                         bool lean, size_t* resident, size_t* transient, bool fibre, int policy) {
  // mirrors the plan_alloc calls of spmttkrp_plan, build_copies and
  // ensure_als_state (each allocation of 0 bytes counts 16)
  const int RI = record_int4s(N);
  const int nu = fibre ? 32 * fibre_slots(R) : SPM_UNITS_PER_PARTITION(R);
  const int64_t nn = nnz > 0 ? nnz : 1;
  int64_t Imax = 1;
  for (int w = 0; w < N; ++w) Imax = std::max(Imax, dims[w]);
  size_t b = sizeof(int) + sizeof(double);  // dev_err, normX2
  b += sizeof(float) * 2 * (size_t)kappa * R + sizeof(int) * 4 * (size_t)kappa;
  b += sizeof(double) * NORM_BLOCKS;
  for (int d = 0; d < N; ++d) {
    if (lean && d > 0) {
      b += sizeof(int32_t) * (size_t)nn + 16;
    } else if (fibre) {
      // at most one fibre per nonzero: an upper bound (the count is data-dependent)
      b += sizeof(int2) * (size_t)(2 * (size_t)(nnz > 0 ? nnz : 0) + 2);
      b += sizeof(FibreUnit) * (size_t)kappa * nu;
      b += sizeof(int32_t) * (size_t)nn;
    } else {
      b += sizeof(int4) * RI * (size_t)nn + 256;
      b += sizeof(int32_t) * (size_t)nn;
    }
    b += sizeof(int64_t) * (size_t)(kappa + 1);
    b += sizeof(int64_t) * ((size_t)kappa * nu + 1);
    b += sizeof(uint32_t) * (size_t)((dims[d] + 31) / 32);
  }
  if (als) {
    const size_t gb = (size_t)std::max(1, sm_count()) * 4;
    const size_t RR = (size_t)R * R;
    b += sizeof(double) * RR * N + sizeof(double) * RR * gb + sizeof(double) * RR;
    b += sizeof(float) * 2 * RR + sizeof(double) * R * gb * 2 + sizeof(double) * 2 * R;
    b += sizeof(float) * R * gb + als_wdig_bytes(R);  // column maxima of Z, W digit tiles
    b += sizeof(float) * (size_t)Imax * R * 2;
  }
  *resident = b;
  // stream-ordered scratch of the build (keys, payloads, histograms)
  const int64_t cap = sort_capacity(N, dims, nn, policy, kappa);
  *transient = sizeof(unsigned long long) * 2 * (size_t)cap + sizeof(int32_t) * 2 * (size_t)cap +
               sizeof(uint32_t) * RS_BINS * (size_t)ceil_div<int64_t>(cap, RS_TILE) +
               sizeof(uint32_t) * RS_BINS + sizeof(int64_t) * SPM_MAX_MODES +
               sizeof(unsigned long long) * SPM_MAX_MODES;
  if (fibre)  // the record copies live until every fibre stream is built
    *transient = std::max<size_t>(*transient, (sizeof(int4) * RI + 256) * (size_t)nn * N +
                                                  sizeof(int32_t) * (size_t)nn);
}

spm_status plan_repartition(spmttkrp_plan_s* p, int kappa, cudaStream_t s) {
  if (kappa < 1 || kappa > 0xFFFF) return SPM_ERR_INVALID_ARG;
  if (p->fibre) return SPM_ERR_UNSUPPORTED;  // work units are baked into the fibre streams
  if (p->policy != (int)(SPM_POLICY_BALANCED >> 4) && p->policy != (int)(SPM_POLICY_SCHEME2 >> 4))
    return SPM_ERR_UNSUPPORTED;
  if (kappa == p->kappa) return SPM_OK;
  if (kappa > p->kappa_cap) {
    // the old arrays may still be read by queued work
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int d = 0; d < p->N; ++d) {
      SPM_TRY(plan_realloc(p, (void**)&p->mode[d].off, sizeof(int64_t) * (size_t)(kappa + 1)));
      SPM_TRY(plan_realloc(p, (void**)&p->mode[d].woff,
                           sizeof(int64_t) * ((size_t)kappa * p->nu + 1)));
    }
    SPM_TRY(plan_realloc(p, (void**)&p->cta_part, sizeof(float) * 2 * (size_t)kappa * p->R));
    SPM_TRY(plan_realloc(p, (void**)&p->cta_meta, sizeof(int) * 4 * (size_t)kappa));
    p->kappa_cap = kappa;
  }
  p->kappa = kappa;
  const int64_t n = p->nnz;
  const int64_t nn = n > 0 ? n : 1;
  uint32_t *hist = nullptr, *dtot = nullptr, *before = nullptr;
  int* rows_tmp = nullptr;
  SPM_CUDA_TRY(cudaMallocAsync((void**)&hist, sizeof(uint32_t) * ceil_div<int64_t>(nn, RS_TILE), s));
  SPM_CUDA_TRY(cudaMallocAsync((void**)&dtot, sizeof(uint32_t), s));
  SPM_CUDA_TRY(cudaMallocAsync((void**)&before, sizeof(uint32_t) * nn, s));
  if (p->lean) SPM_CUDA_TRY(cudaMallocAsync((void**)&rows_tmp, sizeof(int) * nn, s));
  for (int d = 0; d < p->N; ++d) {
    int64_t stride = 0;
    const int* rows = n > 0 ? copy_rows(p, d, rows_tmp, &stride, s) : nullptr;
    partition_copy(p, d, rows, stride, hist, dtot, before, s);
  }
  SPM_CUDA_TRY(cudaGetLastError());
  SPM_CUDA_TRY(cudaFreeAsync(hist, s));
  SPM_CUDA_TRY(cudaFreeAsync(dtot, s));
  SPM_CUDA_TRY(cudaFreeAsync(before, s));
  if (rows_tmp) SPM_CUDA_TRY(cudaFreeAsync(rows_tmp, s));
  return SPM_OK;
}

spm_status build_fibre_copies(spmttkrp_plan_s* p, cudaStream_t s);  // fibre_plan.cu

spm_status build_copies(spmttkrp_plan_s* p, const int32_t* const* idx, const float* vals,
                        cudaStream_t s) {
  SPM_TRY(plan_alloc(p, (void**)&p->norm_part, sizeof(double) * NORM_BLOCKS));
  if (record_int4s(p->N) == 1) {
    SPM_TRY(build_copies_t<1>(p, idx, vals, s));
    // the fibre layout is made from the finished record copies (3 modes)
    return p->fibre ? build_fibre_copies(p, s) : SPM_OK;
  }
  return build_copies_t<2>(p, idx, vals, s);
}

}  // namespace spm
