// ksdf_sort.cu -- device-wide exclusive scan and stable LSD radix sort used by the fit and the query
// grouping.  Written for one GPU; every launch is stream ordered and allocation free once `tmp` is large
// enough.
#include "ksdf_internal.cuh"

namespace ksdf {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// exclusive scan of one value per thread over a 256-thread block; returns the block total in *total
__device__ inline int64_t block_exscan(int64_t v, int64_t* smem_warp, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < (kScanThreads / 32) ? smem_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (kScanThreads / 32)) smem_warp[lane] = w;  // inclusive warp prefix
  }
  __syncthreads();
  int64_t warp_base = warp ? smem_warp[warp - 1] : 0;
  *total = smem_warp[kScanThreads / 32 - 1];
  __syncthreads();
  return warp_base + x - v;
}

// n_dev (may be NULL): the scan covers min(n, *n_dev) elements, a count known only on the device
__device__ __forceinline__ int64_t scan_len(int64_t n, const int64_t* n_dev) {
  return n_dev ? (*n_dev < n ? *n_dev : n) : n;
}

__global__ void k_scan_reduce(const int64_t* in, int64_t n, const int64_t* n_dev, int64_t* sums) {
  __shared__ int64_t sw[kScanThreads / 32];
  n = scan_len(n, n_dev);
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  int64_t tot;
  block_exscan(s, sw, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t* sums, int64_t nb, int64_t* total) {
  __shared__ int64_t sw[kScanThreads / 32];
  int64_t carry = 0;
  for (int64_t c0 = 0; c0 < nb; c0 += kScanThreads) {
    int64_t i = c0 + threadIdx.x;
    int64_t v = i < nb ? sums[i] : 0;
    int64_t tot;
    int64_t ex = block_exscan(v, sw, &tot);
    if (i < nb) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_apply(const int64_t* in, int64_t* out, int64_t n, const int64_t* n_dev, const int64_t* sums) {
  __shared__ int64_t sw[kScanThreads / 32];
  n = scan_len(n, n_dev);
  if ((int64_t)blockIdx.x * kScanTile >= n) return;  // the whole block is past the end (uniform)
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  int64_t tot;
  int64_t ex = block_exscan(s, sw, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += v[i];
  }
}

// small arrays: the whole exclusive scan in one 1024-thread block (one launch instead of three); each
// thread owns a contiguous run of up to kScanSingleItems elements
constexpr int kScanSingleThreads = 1024;
constexpr int kScanSingleItems = 64;

__global__ void __launch_bounds__(kScanSingleThreads) k_scan_single(const int64_t* in, int64_t* out, int64_t n,
                                                                     const int64_t* n_dev, int64_t* total) {
  __shared__ int64_t sw[kScanSingleThreads / 32];
  n = scan_len(n, n_dev);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t per = (n + kScanSingleThreads - 1) / kScanSingleThreads;
  const int64_t b = (int64_t)threadIdx.x * per, e = b + per < n ? b + per : n;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += in[i];
  int64_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sw[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = sw[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sw[lane] = w;  // inclusive prefix over the warps
  }
  __syncthreads();
  int64_t run = (warp ? sw[warp - 1] : 0) + x - s;
  for (int64_t i = b; i < e; ++i) {
    const int64_t v = in[i];
    out[i] = run;
    run += v;
  }
  if (threadIdx.x == kScanSingleThreads - 1 && total) *total = sw[31];
}

// ---- radix sort ----
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsChunks = 8;  // chunks of 256 elements per tile
constexpr int kRsTile = kRsThreads * kRsChunks;

__global__ void k_rs_hist(const uint64_t* keys, int64_t n, int shift, int64_t* hist, int nblocks) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll
  for (int c = 0; c < kRsChunks; ++c) {
    int64_t i = base + c * kRsThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// stable scatter: elements of a chunk are ranked by (warp, lane) order; chunks in order; blocks in order
__global__ void k_rs_scatter(const uint64_t* keys, const uint32_t* vals, uint64_t* okeys, uint32_t* ovals, int64_t n,
                             int shift, const int64_t* offs, int nblocks) {
  __shared__ int64_t running[256];
  __shared__ int64_t wcnt[kRsWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  running[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  int64_t base = (int64_t)blockIdx.x * kRsTile;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int c = 0; c < kRsChunks; ++c) {
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    int64_t i = base + c * kRsThreads + threadIdx.x;
    bool valid = i < n;
    uint64_t k = valid ? keys[i] : 0;
    uint32_t v = valid ? vals[i] : 0;
    int d = valid ? (int)((k >> shift) & 0xFF) : 256;  // 256: no element
    unsigned m = __match_any_sync(0xffffffffu, d);
    int rank = __popc(m & lt_mask);
    if (valid && rank == 0) wcnt[warp][d] = __popc(m);
    __syncthreads();
    {
      int64_t r = running[threadIdx.x];
#pragma unroll
      for (int w = 0; w < kRsWarps; ++w) {
        int64_t t = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = r;
        r += t;
      }
      running[threadIdx.x] = r;
    }
    __syncthreads();
    if (valid) {
      int64_t pos = wcnt[warp][d] + rank;
      okeys[pos] = k;
      ovals[pos] = v;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, DevBuf& tmp, cudaStream_t st,
                     const int64_t* n_dev) {
  if (n <= 0) {
    if (total) return cudaMemsetAsync(total, 0, sizeof(int64_t), st);
    return cudaSuccess;
  }
  if (n <= (int64_t)kScanSingleThreads * kScanSingleItems) {
    launch(k_scan_single, 1, kScanSingleThreads, 0, st, in, out, n, n_dev, total);
    return cudaGetLastError();
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  cudaError_t e = ensure(tmp, sizeof(int64_t) * (size_t)(nb + 1));
  if (e != cudaSuccess) return e;
  int64_t* sums = ptr<int64_t>(tmp);
  launch(k_scan_reduce, (unsigned)nb, kScanThreads, 0, st, in, n, n_dev, sums);
  launch(k_scan_sums, 1, kScanThreads, 0, st, sums, nb, total);
  launch(k_scan_apply, (unsigned)nb, kScanThreads, 0, st, in, out, n, n_dev, sums);
  return cudaGetLastError();
}

cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int bits, DevBuf& tmp, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int passes = (bits + 7) / 8;
  const int nblocks = (int)((n + kRsTile - 1) / kRsTile);
  const int64_t nh = 256LL * nblocks;
  const int64_t nb_scan = (nh + kScanTile - 1) / kScanTile;
  size_t need = sizeof(uint64_t) * n + sizeof(uint32_t) * n + sizeof(int64_t) * (size_t)(nh + nb_scan + 2) + 64;
  cudaError_t e = ensure(tmp, need);
  if (e != cudaSuccess) return e;
  char* b = static_cast<char*>(tmp.p);
  uint64_t* k2 = reinterpret_cast<uint64_t*>(b);
  b += sizeof(uint64_t) * n;
  uint32_t* v2 = reinterpret_cast<uint32_t*>(b);
  b += sizeof(uint32_t) * n;
  b = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(b) + 15) & ~uintptr_t(15));
  int64_t* hist = reinterpret_cast<int64_t*>(b);
  int64_t* sums = hist + nh;
  uint64_t *ki = keys, *ko = k2;
  uint32_t *vi = vals, *vo = v2;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    launch(k_rs_hist, nblocks, kRsThreads, 0, st, ki, n, shift, hist, nblocks);
    if (nh <= (int64_t)kScanSingleThreads * kScanSingleItems) {
      launch(k_scan_single, 1, kScanSingleThreads, 0, st, hist, hist, nh, (const int64_t*)nullptr, (int64_t*)nullptr);
    } else {
      launch(k_scan_reduce, (unsigned)nb_scan, kScanThreads, 0, st, hist, nh, (const int64_t*)nullptr, sums);
      launch(k_scan_sums, 1, kScanThreads, 0, st, sums, nb_scan, (int64_t*)nullptr);
      launch(k_scan_apply, (unsigned)nb_scan, kScanThreads, 0, st, hist, hist, nh, (const int64_t*)nullptr, sums);
    }
    launch(k_rs_scatter, nblocks, kRsThreads, 0, st, ki, vi, ko, vo, n, shift, hist, nblocks);
    uint64_t* tk = ki; ki = ko; ko = tk;
    uint32_t* tv = vi; vi = vo; vo = tv;
  }
  if (ki != keys) {
    e = cudaMemcpyAsync(keys, ki, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(vals, vi, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace ksdf
