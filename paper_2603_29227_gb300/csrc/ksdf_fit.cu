// ksdf_fit.cu -- the fit of Kernel-SDF's local GPs on the GPU (Sec. IV-B.1 of arXiv 2603.29227).
//
//   1. bin every sample: c = floor((x - o) / h) in IEEE binary64 with no contraction (bit-exact);
//   2. stable radix sort of the samples by cell, distinct cells numbered in ascending (cz, cy, cx) order,
//      and an open-addressing hash table key -> cell id;
//   3. training sets: one CTA per cell gathers the samples of the neighbouring cells that fall in its
//      collection box [o + c h - mu, o + (c+1) h + mu) (binary64 compares), sorts them by global id in
//      shared memory and keeps ranks floor(j cnt / n_max) when there are more than n_max;
//   4. the FP64 fit: A = K + diag(sigma^2) with K_ij = exp(-lambda |x_i - x_j|^2), A = L L^T, alpha =
//      A^{-1} 1 (all labels are 1), and L^{-1} by forward substitution on I.  Persistent CTAs take the
//      cells in descending size order; the packed matrix lives in shared memory up to N = 128 and in a
//      per-CTA global scratch slot above that.
#include "ksdf_internal.cuh"

#include <cstdarg>
#include <vector>

namespace ksdf {

namespace {

constexpr int kFitThreads = 256;
constexpr int kFitSmemN = 128;  // packed matrix in shared memory up to this N

__global__ void k_bin_samples(const double* x, const float* var, int64_t S, Params p, uint64_t* keys, uint32_t* vals,
                              int* bbox, uint32_t* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int c[3] = {0, 0, 0};
  bool ok = true, live = i < S;
  if (live) {
    for (int j = 0; j < p.dim; ++j) ok &= bin_coord(x[i * p.dim + j], p.o[j], p.h, c[j]);
    if (var) {
      float v = var[i];
      ok &= (v >= 0.f) && isfinite(v);
    }
    if (!ok) atomicOr(status, ST_NONFINITE);
    keys[i] = ok ? pack_key(c[0], c[1], c[2]) : 0;
    vals[i] = (uint32_t)i;
  }
  // bounding box of the cell coordinates (warp reduce, then one atomic per warp)
  int mn[3], mx[3];
  for (int j = 0; j < 3; ++j) {
    mn[j] = (live && ok) ? c[j] : INT32_MAX;
    mx[j] = (live && ok) ? c[j] : INT32_MIN;
  }
  for (int o = 16; o; o >>= 1)
    for (int j = 0; j < 3; ++j) {
      mn[j] = min(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], o));
      mx[j] = max(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], o));
    }
  if ((threadIdx.x & 31) == 0)
    for (int j = 0; j < 3; ++j) {
      if (mn[j] != INT32_MAX) atomicMin(&bbox[j], mn[j]);
      if (mx[j] != INT32_MIN) atomicMax(&bbox[3 + j], mx[j]);
    }
}

__global__ void k_linear_keys(uint64_t* keys, int64_t S, int x0, int y0, int z0, int64_t nx, int64_t ny) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S) return;
  int cx, cy, cz;
  unpack_key(keys[i], cx, cy, cz);
  keys[i] = ((uint64_t)(cz - z0) * (uint64_t)ny + (uint64_t)(cy - y0)) * (uint64_t)nx + (uint64_t)(cx - x0);
}

__global__ void k_flags(const uint64_t* lin, int64_t S, int64_t* flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < S) flag[i] = (i == 0 || lin[i] != lin[i - 1]) ? 1 : 0;
}

__global__ void k_cells(const uint64_t* lin, const int64_t* flag_scan, int64_t S, int x0, int y0, int z0, int64_t nx,
                        int64_t ny, uint64_t* cell_key, int64_t* own_off) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S) return;
  if (i == 0 || lin[i] != lin[i - 1]) {
    int64_t g = flag_scan[i];
    uint64_t l = lin[i];
    int64_t cx = (int64_t)(l % (uint64_t)nx) + x0;
    int64_t r = (int64_t)(l / (uint64_t)nx);
    int64_t cy = r % ny + y0;
    int64_t cz = r / ny + z0;
    cell_key[g] = pack_key(cx, cy, cz);
    own_off[g] = i;
  }
}

__global__ void k_fill_u64(uint64_t* a, int64_t n, uint64_t v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

__global__ void k_hash_insert(const uint64_t* cell_key, int64_t G, uint64_t* hk, int32_t* hv, uint64_t cap) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  uint64_t k = cell_key[g];
  uint64_t s = mix64(k) & (cap - 1);
  for (uint64_t probe = 0; probe < cap; ++probe) {
    unsigned long long prev = atomicCAS((unsigned long long*)&hk[s], (unsigned long long)kEmptyKey,
                                        (unsigned long long)k);
    if (prev == kEmptyKey || prev == k) {
      hv[s] = (int32_t)g;
      return;
    }
    s = (s + 1) & (cap - 1);
  }
}

// bitonic sort of n (power of two) ints in shared memory, ascending
__device__ void smem_bitonic(int* a, int n) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          int ai = a[i], aj = a[ixj];
          bool up = (i & k) == 0;
          if ((ai > aj) == up) {
            a[i] = aj;
            a[ixj] = ai;
          }
        }
      }
      __syncthreads();
    }
  }
}

// training set of one cell per CTA: collection-box members, ascending global id, rank-selected cap
__global__ void __launch_bounds__(512) k_assemble(const uint64_t* cell_key, int64_t G, const int64_t* own_off,
                                                  const uint32_t* own_id, const double* x, Params p, int R,
                                                  const uint64_t* hk, const int32_t* hv, uint64_t hcap,
                                                  int32_t* mpad, int64_t* n_out, int32_t* status, int* max_n,
                                                  uint32_t* st) {
  __shared__ int ids[kMaxPre];
  __shared__ int cnt;
  const int64_t g = blockIdx.x;
  if (g >= G) return;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c[3];
  unpack_key(cell_key[g], c[0], c[1], c[2]);
  double lo[3], hi[3];
  for (int j = 0; j < 3; ++j) {
    lo[j] = __dsub_rn(cell_base(p.o[j], c[j], p.h), p.mu);
    hi[j] = __dadd_rn(cell_base(p.o[j], c[j] + 1, p.h), p.mu);
  }
  const int zr = p.dim == 3 ? R : 0;
  for (int dz = -zr; dz <= zr; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        int64_t nb[3] = {(int64_t)c[0] + dx, (int64_t)c[1] + dy, (int64_t)c[2] + dz};
        bool inr = true;
        for (int j = 0; j < 3; ++j) inr &= nb[j] >= -kBias && nb[j] < kBias;
        if (!inr) continue;
        int h = hash_find(hk, hv, hcap, pack_key(nb[0], nb[1], nb[2]));
        if (h < 0) continue;
        for (int64_t t = own_off[h] + threadIdx.x; t < own_off[h + 1]; t += blockDim.x) {
          uint32_t id = own_id[t];
          const double* xi = x + (int64_t)id * p.dim;
          bool in = true;
          for (int j = 0; j < p.dim; ++j) in &= (xi[j] >= lo[j]) && (xi[j] < hi[j]);
          if (in) {
            int pos = atomicAdd(&cnt, 1);
            if (pos < kMaxPre) ids[pos] = (int)id;
          }
        }
      }
  __syncthreads();
  int n = cnt;
  if (n > kMaxPre) {
    if (threadIdx.x == 0) {
      atomicOr(st, ST_CAPACITY);
      n_out[g] = 0;
      status[g] = KSDF_CELL_EMPTY;
    }
    return;
  }
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (int i = n + threadIdx.x; i < np2; i += blockDim.x) ids[i] = INT32_MAX;
  __syncthreads();
  smem_bitonic(ids, np2);
  int keep = n > p.n_max ? p.n_max : n;
  for (int j = threadIdx.x; j < keep; j += blockDim.x) {
    int src = n > p.n_max ? (int)(((int64_t)j * n) / p.n_max) : j;
    mpad[g * p.n_max + j] = ids[src];
  }
  if (threadIdx.x == 0) {
    n_out[g] = keep;
    status[g] = keep > 0 ? KSDF_CELL_OK : KSDF_CELL_EMPTY;
    atomicMax(max_n, keep);
  }
}

__global__ void k_tri_sizes(const int64_t* n, int64_t G, int64_t* tri, int32_t* n32) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  tri[g] = n[g] * (n[g] + 1) / 2;
  n32[g] = (int32_t)n[g];
}

__global__ void k_order_keys(const int32_t* n32, int64_t G, int n_max, uint64_t* keys, uint32_t* vals) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  keys[g] = (uint64_t)(n_max - n32[g]);  // descending size
  vals[g] = (uint32_t)g;
}

// members: global id, cell-local FP64/FP32 coordinates, variance, normal
__global__ void k_gather_members(const uint64_t* cell_key, const int32_t* n32, const int64_t* ts_off,
                                 const int32_t* mpad, int64_t G, Params p, const double* x, const float* var,
                                 const float* nrm, int32_t* mgid, D4* md4, float4* mf4, float* mvar,
                                 float4* mnrm) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t g = t / p.n_max;
  int j = (int)(t % p.n_max);
  if (g >= G || j >= n32[g]) return;
  int id = mpad[g * p.n_max + j];
  int64_t m = ts_off[g] + j;
  int c[3];
  unpack_key(cell_key[g], c[0], c[1], c[2]);
  double l[3] = {0, 0, 0};
  for (int d = 0; d < p.dim; ++d) l[d] = __dsub_rn(x[(int64_t)id * p.dim + d], cell_base(p.o[d], c[d], p.h));
  mgid[m] = id;
  md4[m] = D4make(l[0], l[1], l[2], 0.0);
  mf4[m] = make_float4((float)l[0], (float)l[1], (float)l[2], 0.f);
  mvar[m] = var ? var[id] : 0.f;
  if (nrm) {
    float nv[3] = {0, 0, 0};
    for (int d = 0; d < p.dim; ++d) nv[d] = nrm[(int64_t)id * p.dim + d];
    mnrm[m] = make_float4(nv[0], nv[1], nv[2], 0.f);
  }
}

__host__ __device__ inline int64_t tri(int i) { return (int64_t)i * (i + 1) / 2; }

// FP64 fit of one cell per CTA iteration (persistent, dynamic work counter)
__global__ void __launch_bounds__(kFitThreads) k_fit(const uint32_t* order, int64_t G, const int32_t* n32,
                                                     const int64_t* ts_off, const int64_t* linv_off, Params p,
                                                     D4* md4, float4* mf4, const float* mvar, double* linv64,
                                                     float* linv32, float* linv32lo, int32_t* status,
                                                     double* scratch, int64_t scratch_stride, int* counter,
                                                     int* n_not_pd, uint32_t* st) {
  extern __shared__ double sm[];
  __shared__ int s_cell, s_fail;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  // shared layout: [xyz: 3 * n_max][b: n_max][A packed: tri(kFitSmemN) if used]
  double* sx = sm;
  double* sb = sx + 3 * p.n_max;
  double* sA = sb + p.n_max;
  for (;;) {
    if (tid == 0) {
      int w = atomicAdd(counter, 1);
      s_cell = w < G ? (int)order[w] : -1;
      s_fail = 0;
    }
    __syncthreads();
    const int g = s_cell;
    if (g < 0) break;
    const int N = n32[g];
    if (N == 0) {
      __syncthreads();
      continue;
    }
    const int64_t m0 = ts_off[g];
    double* A = N <= kFitSmemN ? sA : scratch + (int64_t)blockIdx.x * scratch_stride;
    for (int i = tid; i < N; i += nthr) {
      D4 v = md4[m0 + i];
      sx[3 * i] = v.x;
      sx[3 * i + 1] = v.y;
      sx[3 * i + 2] = v.z;
    }
    __syncthreads();
    // A = K + diag(sigma^2), lower triangle, rows by warps
    for (int i = warp; i < N; i += nwarp)
      for (int j = lane; j <= i; j += 32) {
        double dx = sx[3 * i] - sx[3 * j], dy = sx[3 * i + 1] - sx[3 * j + 1], dz = sx[3 * i + 2] - sx[3 * j + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        double a = exp(-p.lambda * r2);
        if (i == j) a += (double)mvar[m0 + i];
        A[tri(i) + j] = a;
      }
    __syncthreads();
    // Cholesky, right looking: column k scaled by the pivot, then the trailing update
    for (int k = 0; k < N; ++k) {
      if (tid == 0) {
        double piv = A[tri(k) + k];
        if (!(piv > 0.0)) s_fail = 1;
        else A[tri(k) + k] = sqrt(piv);
      }
      __syncthreads();
      if (s_fail) break;
      const double dkk = A[tri(k) + k];
      for (int i = k + 1 + tid; i < N; i += nthr) A[tri(i) + k] = A[tri(i) + k] / dkk;
      __syncthreads();
      for (int i = k + 1 + warp; i < N; i += nwarp) {
        const double lik = A[tri(i) + k];
        for (int j = k + 1 + lane; j <= i; j += 32) A[tri(i) + j] = fma(-lik, A[tri(j) + k], A[tri(i) + j]);
      }
      __syncthreads();
    }
    if (s_fail) {
      if (tid == 0) {
        status[g] = KSDF_CELL_NOT_PD;
        atomicAdd(n_not_pd, 1);
      }
      for (int i = tid; i < N; i += nthr) {
        md4[m0 + i].w = 0.0;
        mf4[m0 + i].w = 0.f;
      }
      __syncthreads();
      continue;
    }
    // alpha: L y = 1, then L^T alpha = y
    for (int i = tid; i < N; i += nthr) sb[i] = 1.0;
    __syncthreads();
    for (int k = 0; k < N; ++k) {
      if (tid == 0) sb[k] = sb[k] / A[tri(k) + k];
      __syncthreads();
      const double bk = sb[k];
      for (int i = k + 1 + tid; i < N; i += nthr) sb[i] = fma(-A[tri(i) + k], bk, sb[i]);
      __syncthreads();
    }
    for (int k = N - 1; k >= 0; --k) {
      if (tid == 0) sb[k] = sb[k] / A[tri(k) + k];
      __syncthreads();
      const double bk = sb[k];
      for (int i = tid; i < k; i += nthr) sb[i] = fma(-A[tri(k) + i], bk, sb[i]);
      __syncthreads();
    }
    for (int i = tid; i < N; i += nthr) {
      md4[m0 + i].w = sb[i];
      mf4[m0 + i].w = (float)sb[i];
    }
    // L^{-1}: X = I, row k divided by L_kk, then rows below updated (right looking); X lives in the output
    double* X = linv64 + linv_off[g];
    for (int i = warp; i < N; i += nwarp)
      for (int j = lane; j <= i; j += 32) X[tri(i) + j] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < N; ++k) {
      const double dkk = A[tri(k) + k];
      for (int j = tid; j <= k; j += nthr) X[tri(k) + j] = X[tri(k) + j] / dkk;
      __syncthreads();
      for (int i = k + 1 + warp; i < N; i += nwarp) {
        const double lik = A[tri(i) + k];
        for (int j = lane; j <= k; j += 32) X[tri(i) + j] = fma(-lik, X[tri(k) + j], X[tri(i) + j]);
      }
      __syncthreads();
    }
    for (int64_t e = tid; e < tri(N); e += nthr) {
      double v = X[e];
      float hi = (float)v;
      linv32[linv_off[g] + e] = hi;
      linv32lo[linv_off[g] + e] = (float)(v - (double)hi);
    }
    __syncthreads();
  }
}

}  // namespace

static int bits_for(uint64_t v) {
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

ksdf_status fit_model(ksdf_ctx* c, const double* x, const float* var, const float* nrm, int64_t S) {
  cudaStream_t st = c->stream;
  const Params& p = c->p;
  Model& m = c->m;
  c->fitted = false;
  if (S <= 0) return set_err(c, KSDF_ERR_ARG, "ksdf_fit: S must be positive");
  if (S >= (1LL << 31)) return set_err(c, KSDF_ERR_CAPACITY, "ksdf_fit: S must be < 2^31");
  uint32_t* stw = ptr<uint32_t>(c->status_word);
  cudaEvent_t e_fit = prof_begin(c), e0 = prof_begin(c);
  // 1. bin
  KSDF_CUDA(c, ensure(c->ws[WS_A], sizeof(uint64_t) * S));
  KSDF_CUDA(c, ensure(c->ws[WS_B], sizeof(uint32_t) * S));
  KSDF_CUDA(c, ensure(c->ws[WS_C], sizeof(int) * 8));
  uint64_t* keys = ptr<uint64_t>(c->ws[WS_A]);
  uint32_t* vals = ptr<uint32_t>(c->ws[WS_B]);
  int* bbox = ptr<int>(c->ws[WS_C]);
  int hb[8] = {INT32_MAX, INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN, INT32_MIN, 0, 0};
  KSDF_CUDA(c, cudaMemcpyAsync(bbox, hb, sizeof(hb), cudaMemcpyHostToDevice, st));
  KSDF_CUDA(c, cudaMemsetAsync(stw, 0, sizeof(uint32_t), st));
  launch(k_bin_samples, ceil_div(S, 256), 256, 0, st, x, var, S, p, keys, vals, bbox, stw);
  uint32_t hst = 0;
  KSDF_CUDA(c, cudaMemcpyAsync(hb, bbox, sizeof(int) * 6, cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaMemcpyAsync(&hst, stw, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaStreamSynchronize(st));
  if (hst & ST_NONFINITE)
    return set_err(c, KSDF_ERR_NONFINITE, "ksdf_fit: NaN/Inf or out-of-grid sample, or invalid variance");
  const int x0 = hb[0], y0 = hb[1], z0 = hb[2];
  for (int j = 0; j < 6; ++j) c->bb[j] = hb[j];
  const int64_t nx = (int64_t)hb[3] - x0 + 1, ny = (int64_t)hb[4] - y0 + 1, nz = (int64_t)hb[5] - z0 + 1;
  const uint64_t vol = (uint64_t)nx * (uint64_t)ny * (uint64_t)nz;
  // 2. sort by linear cell index (ascending (cz, cy, cx)), stable in sample id
  launch(k_linear_keys, ceil_div(S, 256), 256, 0, st, keys, S, x0, y0, z0, nx, ny);
  KSDF_CUDA(c, radix_sort_u64(keys, vals, S, bits_for(vol - 1), c->ws[WS_SORT], st));
  KSDF_CUDA(c, ensure(c->ws[WS_D], sizeof(int64_t) * (S + 1)));
  int64_t* flag = ptr<int64_t>(c->ws[WS_D]);
  launch(k_flags, ceil_div(S, 256), 256, 0, st, keys, S, flag);
  KSDF_CUDA(c, ensure(c->ws[WS_E], sizeof(int64_t) * 4));
  int64_t* dtot = ptr<int64_t>(c->ws[WS_E]);
  KSDF_CUDA(c, scan_i64(flag, flag, S, dtot, c->ws[WS_SCAN], st));
  int64_t G = 0;
  KSDF_CUDA(c, cudaMemcpyAsync(&G, dtot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaStreamSynchronize(st));
  m.G = G;
  m.S = S;
  KSDF_CUDA(c, ensure(m.key, sizeof(uint64_t) * G));
  KSDF_CUDA(c, ensure(c->ws[WS_F], sizeof(int64_t) * (G + 1)));
  int64_t* own_off = ptr<int64_t>(c->ws[WS_F]);
  launch(k_cells, ceil_div(S, 256), 256, 0, st, keys, flag, S, x0, y0, z0, nx, ny, ptr<uint64_t>(m.key), own_off);
  KSDF_CUDA(c, cudaMemcpyAsync(own_off + G, &S, sizeof(int64_t), cudaMemcpyHostToDevice, st));
  // hash table key -> cell id
  uint64_t cap = 64;
  while (cap < 2 * (uint64_t)G) cap <<= 1;
  m.hcap = cap;
  KSDF_CUDA(c, ensure(m.hkeys, sizeof(uint64_t) * cap));
  KSDF_CUDA(c, ensure(m.hvals, sizeof(int32_t) * cap));
  launch(k_fill_u64, ceil_div(cap, 256), 256, 0, st, ptr<uint64_t>(m.hkeys), cap, kEmptyKey);
  launch(k_hash_insert, ceil_div(G, 256), 256, 0, st, ptr<uint64_t>(m.key), G, ptr<uint64_t>(m.hkeys),
                                                   ptr<int32_t>(m.hvals), cap);
  prof_end(c, e0, "fit.index");
  e0 = prof_begin(c);
  // 3. training sets
  const int R = (int)floor(p.mu / p.h + 1e-6) + 1;
  KSDF_CUDA(c, ensure(m.mpad, sizeof(int32_t) * (size_t)G * p.n_max));
  KSDF_CUDA(c, ensure(m.status, sizeof(int32_t) * G));
  KSDF_CUDA(c, ensure(m.n, sizeof(int32_t) * G));
  KSDF_CUDA(c, ensure(m.ts_off, sizeof(int64_t) * (G + 1)));
  KSDF_CUDA(c, ensure(m.linv_off, sizeof(int64_t) * (G + 1)));
  KSDF_CUDA(c, ensure(c->ws[WS_D], sizeof(int64_t) * (2 * G + 2)));
  int64_t* n64 = ptr<int64_t>(c->ws[WS_D]);
  int64_t* tri64 = n64 + (G + 1);
  int* dmax = bbox + 6;
  KSDF_CUDA(c, cudaMemsetAsync(dmax, 0, sizeof(int) * 2, st));
  launch(k_assemble, (unsigned)G, 512, 0, st, ptr<uint64_t>(m.key), G, own_off, vals, x, p, R, ptr<uint64_t>(m.hkeys),
                                          ptr<int32_t>(m.hvals), cap, ptr<int32_t>(m.mpad), n64,
                                          ptr<int32_t>(m.status), dmax, stw);
  launch(k_tri_sizes, ceil_div(G, 256), 256, 0, st, n64, G, tri64, ptr<int32_t>(m.n));
  KSDF_CUDA(c, scan_i64(n64, ptr<int64_t>(m.ts_off), G, dtot, c->ws[WS_SCAN], st));
  KSDF_CUDA(c, scan_i64(tri64, ptr<int64_t>(m.linv_off), G, dtot + 1, c->ws[WS_SCAN], st));
  int64_t tots[2];
  int hmax[2];
  KSDF_CUDA(c, cudaMemcpyAsync(tots, dtot, sizeof(tots), cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaMemcpyAsync(hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaMemcpyAsync(&hst, stw, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaStreamSynchronize(st));
  if (hst & ST_CAPACITY)
    return set_err(c, KSDF_ERR_CAPACITY, "ksdf_fit: a collection box holds more than %d samples", kMaxPre);
  m.M = tots[0];
  m.linv_total = tots[1];
  m.max_n = hmax[0];
  KSDF_CUDA(c, cudaMemcpyAsync(ptr<int64_t>(m.ts_off) + G, &tots[0], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  KSDF_CUDA(c, cudaMemcpyAsync(ptr<int64_t>(m.linv_off) + G, &tots[1], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  prof_end(c, e0, "fit.assemble");
  // 4. member arrays
  const int64_t M = m.M;
  m.has_normals = nrm != nullptr;
  KSDF_CUDA(c, ensure(m.mgid, sizeof(int32_t) * (M + 1)));
  KSDF_CUDA(c, ensure(m.md4, sizeof(D4) * (M + 1)));
  KSDF_CUDA(c, ensure(m.mf4, sizeof(float4) * (M + 1)));
  KSDF_CUDA(c, ensure(m.mvar, sizeof(float) * (M + 1)));
  if (nrm) KSDF_CUDA(c, ensure(m.mnrm, sizeof(float4) * (M + 1)));
  KSDF_CUDA(c, ensure(m.linv64, sizeof(double) * (m.linv_total + 1)));
  KSDF_CUDA(c, ensure(m.linv32, sizeof(float) * (m.linv_total + 1)));
  KSDF_CUDA(c, ensure(m.linv32lo, sizeof(float) * (m.linv_total + 1)));
  launch(k_gather_members, ceil_div(G * p.n_max, 256), 256, 0, st, 
      ptr<uint64_t>(m.key), ptr<int32_t>(m.n), ptr<int64_t>(m.ts_off), ptr<int32_t>(m.mpad), G, p, x, var, nrm,
      ptr<int32_t>(m.mgid), ptr<D4>(m.md4), ptr<float4>(m.mf4), ptr<float>(m.mvar),
      nrm ? ptr<float4>(m.mnrm) : nullptr);
  // 5. FP64 fit, largest cells first
  KSDF_CUDA(c, ensure(c->ws[WS_A], sizeof(uint64_t) * (G + 1)));
  KSDF_CUDA(c, ensure(m.cell_order, sizeof(uint32_t) * (G + 1)));
  uint64_t* okeys = ptr<uint64_t>(c->ws[WS_A]);
  uint32_t* order = ptr<uint32_t>(m.cell_order);
  launch(k_order_keys, ceil_div(G, 256), 256, 0, st, ptr<int32_t>(m.n), G, p.n_max, okeys, order);
  KSDF_CUDA(c, radix_sort_u64(okeys, order, G, bits_for((uint64_t)p.n_max), c->ws[WS_SORT], st));
  const int nblk = (int)std::min<int64_t>(G, 2LL * c->num_sms);
  const int64_t stride = (m.max_n > kFitSmemN) ? tri(m.max_n) : 0;
  KSDF_CUDA(c, ensure(c->ws[WS_FITSCR], sizeof(double) * (size_t)(stride * nblk + 1)));
  const size_t smem = sizeof(double) * (4 * (size_t)p.n_max + tri(kFitSmemN));
  KSDF_CUDA(c, cudaFuncSetAttribute(k_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  KSDF_CUDA(c, cudaMemsetAsync(dmax, 0, sizeof(int) * 2, st));
  e0 = prof_begin(c);
  launch(k_fit, nblk, kFitThreads, smem, st, order, G, ptr<int32_t>(m.n), ptr<int64_t>(m.ts_off),
                                         ptr<int64_t>(m.linv_off), p, ptr<D4>(m.md4), ptr<float4>(m.mf4),
                                         ptr<float>(m.mvar), ptr<double>(m.linv64), ptr<float>(m.linv32),
                                         ptr<float>(m.linv32lo), ptr<int32_t>(m.status),
                                         ptr<double>(c->ws[WS_FITSCR]), stride, dmax, dmax + 1, stw);
  KSDF_CUDA(c, cudaGetLastError());
  prof_end(c, e0, "fit.cholesky");
  KSDF_CUDA(c, cudaMemcpyAsync(hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaStreamSynchronize(st));
  m.n_not_pd = hmax[1];
  // keep the sample positions for the adjoint's per-cell recomputation
  KSDF_CUDA(c, ensure(m.x, sizeof(double) * S * p.dim));
  KSDF_CUDA(c, cudaMemcpyAsync(m.x.p, x, sizeof(double) * S * p.dim, cudaMemcpyDeviceToDevice, st));
  prof_end(c, e_fit, "fit");
  c->fitted = true;
  if (m.n_not_pd > 0)
    return set_err(c, KSDF_ERR_NOT_PD, "ksdf_fit: %d cell(s) not positive definite in FP64 (excluded)", m.n_not_pd);
  return KSDF_OK;
}

namespace {
__global__ void k_bin_keys(const double* x, int64_t n, Params p, uint64_t* keys, uint32_t* st) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3] = {0, 0, 0};
  bool ok = true;
  for (int j = 0; j < p.dim; ++j) ok &= bin_coord(x[i * p.dim + j], p.o[j], p.h, c[j]);
  if (!ok) atomicOr(st, ST_NONFINITE);
  keys[i] = ok ? pack_key(c[0], c[1], c[2]) : kEmptyKey;
}
}  // namespace

ksdf_status bin_points(ksdf_ctx* c, const double* x, int64_t n, uint64_t* keys) {
  if (n <= 0) return KSDF_OK;
  launch(k_bin_keys, ceil_div(n, 256), 256, 0, c->stream, x, n, c->p, keys, ptr<uint32_t>(c->status_word));
  KSDF_CUDA(c, cudaGetLastError());
  return KSDF_OK;
}

}  // namespace ksdf
