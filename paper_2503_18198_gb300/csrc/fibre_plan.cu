// fibre_plan.cu -- the fibre layout of 3-mode copies (SPM_PLAN_FIBRE).
//
// A mode-d copy in the P1 key order (c_d, c_a, c_b, position) is cut into
// fibres: maximal runs of nonzeros that share (c_d, c_a), a being the first
// input mode.  The copy is then stored as one stream of 8-byte entries, each
// fibre a header {c_a | 2^31, c_d} followed by one entry {c_b, value bits}
// per nonzero (the first word always the row to gather, its top bit telling
// which factor): the row Y_a(c_a) is gathered once per fibre, and the copy
// takes 8 bytes per nonzero plus 8 per fibre instead of a 16-byte record per
// nonzero.  This is the compressed-fibre idea of the CSF formats that Sec. II
// contrasts with the paper's per-mode COO copies (Sec. III-C), kept on the
// same order, partitions and work units.
//
// Building it from the record copy: fibre starts, their running count (a
// two-level scan), the stream entries at position k + fibre(k) + 1, and per
// work unit its stream range and the header of its first nonzero's fibre.
#include <algorithm>

#include "plan.cuh"

namespace spm {
namespace {

constexpr int FIB_TILE = 2048;  // nonzeros per block of the scans
constexpr int FIB_THREADS = 256;
constexpr int FIB_PER_THREAD = FIB_TILE / FIB_THREADS;

__device__ __forceinline__ uint32_t fibre_start(const int4* __restrict__ rec, int64_t k) {
  if (k == 0) return 1u;
  const int4 a = __ldg(rec + k - 1), b = __ldg(rec + k);
  return (a.x != b.x || a.y != b.y) ? 1u : 0u;
}

// Inclusive scan of one value per thread over the block (FIB_THREADS).
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t* wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(SPM_FULL_MASK, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < FIB_THREADS / 32 ? wsum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(SPM_FULL_MASK, w, o);
      if (lane >= o) w += t;
    }
    if (lane < FIB_THREADS / 32) wsum[lane] = w;
  }
  __syncthreads();
  return v + (warp > 0 ? wsum[warp - 1] : 0u);
}

// Block b: number of fibre starts among nonzeros [b*FIB_TILE, (b+1)*FIB_TILE).
__global__ void __launch_bounds__(FIB_THREADS)
    fibre_count_kernel(const int4* __restrict__ rec, int64_t n, uint32_t* __restrict__ bcnt) {
  __shared__ uint32_t wsum[FIB_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * FIB_TILE + (int64_t)threadIdx.x * FIB_PER_THREAD;
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < FIB_PER_THREAD; ++i)
    if (base + i < n) c += fibre_start(rec, base + i);
  const uint32_t tot = block_inclusive_scan(c, wsum);
  if (threadIdx.x == FIB_THREADS - 1) bcnt[blockIdx.x] = tot;
}

// Exclusive prefix sums of a[0..m) in place, one block of 1024 threads
// (each thread a contiguous chunk, then a scan of the chunk sums).
__global__ void __launch_bounds__(1024) exclusive_scan_kernel(uint32_t* __restrict__ a, int64_t m) {
  __shared__ uint32_t part[1024];
  const int64_t per = (m + 1023) / 1024;
  const int64_t i0 = (int64_t)threadIdx.x * per, i1 = std::min<int64_t>(m, i0 + per);
  uint32_t s = 0;
  for (int64_t i = i0; i < i1; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t t = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += t;
    __syncthreads();
  }
  uint32_t run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0u;
  for (int64_t i = i0; i < i1; ++i) {
    const uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
}

// fidx[k] = index of the fibre that holds nonzero k (starts so far - 1).
__global__ void __launch_bounds__(FIB_THREADS)
    fibre_index_kernel(const int4* __restrict__ rec, int64_t n, const uint32_t* __restrict__ bpre,
                       int32_t* __restrict__ fidx) {
  __shared__ uint32_t wsum[FIB_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * FIB_TILE + (int64_t)threadIdx.x * FIB_PER_THREAD;
  uint32_t st[FIB_PER_THREAD];
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < FIB_PER_THREAD; ++i) {
    st[i] = base + i < n ? fibre_start(rec, base + i) : 0u;
    c += st[i];
  }
  uint32_t run = block_inclusive_scan(c, wsum) - c + bpre[blockIdx.x];
#pragma unroll
  for (int i = 0; i < FIB_PER_THREAD; ++i) {
    run += st[i];
    if (base + i < n) fidx[base + i] = (int32_t)run - 1;
  }
}

// Stream entries: nonzero k at k + fidx[k] + 1, its fibre's header just
// before it when k starts the fibre.
__global__ void fibre_stream_kernel(const int4* __restrict__ rec, const int32_t* __restrict__ fidx,
                                    int64_t n, int2* __restrict__ stream) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int4 r = __ldg(rec + k);
    const int64_t sp = k + fidx[k] + 1;
    stream[sp] = make_int2(r.z, r.w);
    if (fibre_start(rec, k)) stream[sp - 1] = make_int2(r.y | (int)0x80000000u, r.x);
  }
}

// Work unit q: stream range from its first nonzero to its last, the header
// of its first nonzero's fibre, and the row of the nonzero before its end.
__global__ void fibre_units_kernel(const int4* __restrict__ rec, const int32_t* __restrict__ fidx,
                                   const int64_t* __restrict__ woff, int64_t P, int64_t n,
                                   FibreUnit* __restrict__ units) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k0 = woff[q], k1 = woff[q + 1];
    FibreUnit u{};
    u.pad = 0;
    if (n > 0) {
      const int64_t kf = k0 < n ? k0 : n - 1;
      const int4 rf = __ldg(rec + kf);
      u.cd_first = rf.x;
      u.ca_first = rf.y;
      u.cd_last = k1 > 0 ? __ldg(rec + k1 - 1).x : -1;
    } else {
      u.cd_first = u.ca_first = u.cd_last = -1;
    }
    if (k1 > k0) {
      u.sbeg = k0 + fidx[k0] + 1;
      u.send = (k1 - 1) + fidx[k1 - 1] + 2;
    } else {
      u.sbeg = u.send = 0;
    }
    units[q] = u;
  }
}

int grid_n(int64_t n, int threads) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div<int64_t>(n, threads), 152 * 32));
}

}  // namespace

// Convert every (3-mode) record copy of plan p into the fibre layout; the
// record copies are released.  Synchronises `s` (the stream sizes depend on
// the fibre counts).
spm_status build_fibre_copies(spmttkrp_plan_s* p, cudaStream_t s) {
  const int64_t n = p->nnz;
  const int64_t P = (int64_t)p->kappa * p->nu;
  const int64_t nb = std::max<int64_t>(1, ceil_div<int64_t>(n, FIB_TILE));
  uint32_t* bcnt = nullptr;
  int32_t* fidx = nullptr;
  SPM_CUDA_TRY(cudaMallocAsync((void**)&bcnt, sizeof(uint32_t) * nb, s));
  SPM_CUDA_TRY(cudaMallocAsync((void**)&fidx, sizeof(int32_t) * std::max<int64_t>(1, n), s));
  spm_status st = SPM_OK;
  for (int d = 0; d < p->N && st == SPM_OK; ++d) {
    spm_mode_copy& c = p->mode[d];
    int64_t nfib = 0;
    if (n > 0) {
      fibre_count_kernel<<<(int)nb, FIB_THREADS, 0, s>>>(c.rec, n, bcnt);
      exclusive_scan_kernel<<<1, 1024, 0, s>>>(bcnt, nb);
      fibre_index_kernel<<<(int)nb, FIB_THREADS, 0, s>>>(c.rec, n, bcnt, fidx);
      int32_t last = 0;
      SPM_CUDA_TRY(cudaMemcpyAsync(&last, fidx + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      SPM_CUDA_TRY(cudaStreamSynchronize(s));
      nfib = (int64_t)last + 1;
    }
    // two entries of padding: 16-byte-aligned bulk copies of any range stay inside
    st = plan_alloc(p, (void**)&c.fstream, sizeof(int2) * (size_t)(n + nfib + 2));
    if (st == SPM_OK) st = plan_alloc(p, (void**)&c.funits, sizeof(FibreUnit) * (size_t)P);
    if (st != SPM_OK) break;
    SPM_CUDA_TRY(cudaMemsetAsync(c.fstream, 0, sizeof(int2) * (size_t)(n + nfib + 2), s));
    if (n > 0) fibre_stream_kernel<<<grid_n(n, 256), 256, 0, s>>>(c.rec, fidx, n, c.fstream);
    fibre_units_kernel<<<grid_n(P, 256), 256, 0, s>>>(c.rec, fidx, c.woff, P, n, c.funits);
    SPM_CUDA_TRY(cudaGetLastError());
    c.nfib = nfib;
  }
  SPM_CUDA_TRY(cudaFreeAsync(bcnt, s));
  SPM_CUDA_TRY(cudaFreeAsync(fidx, s));
  SPM_CUDA_TRY(cudaStreamSynchronize(s));
  if (st != SPM_OK) return st;
  for (int d = 0; d < p->N; ++d) plan_free(p, (void**)&p->mode[d].rec);
  return SPM_OK;
}

}  // namespace spm
