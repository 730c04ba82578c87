// ksdf_fit.cu -- the fit of Kernel-SDF's local GPs on the GPU (Sec. IV-B.1 of arXiv 2603.29227).
//
//   1. bin every sample: c = floor((x - o) / h) in IEEE binary64 with no contraction (bit-exact);
//   2. stable radix sort of the samples by cell, distinct cells numbered in ascending (cz, cy, cx) order,
//      and an open-addressing hash table key -> cell id;
//   3. training sets: one CTA per cell gathers the samples of the neighbouring cells that fall in its
//      collection box [o + c h - mu, o + (c+1) h + mu) (binary64 compares), sorts them by global id in
//      shared memory and keeps ranks floor(j cnt / n_max) when there are more than n_max;
//   4. the fit: A = K + diag(sigma^2) with K_ij = exp(-lambda |x_i - x_j|^2) in FP64, the FP64 Cholesky
//      factor A = L L^T (blocked, right looking) and alpha = A^{-1} 1 by two FP64 triangular solves (all
//      labels are 1); L^{-1} for the variance contraction in FP32, from L rounded to FP32.  Persistent
//      CTAs take the cells in descending size order, in four size classes launched concurrently: the
//      packed matrix lives in shared memory up to N = 218 and in a per-CTA global scratch slot above that.
#include "ksdf_exp.cuh"
#include "ksdf_internal.cuh"

#include <cstdarg>
#include <vector>

namespace ksdf {

namespace {

constexpr int kPanel = 16;    // Cholesky panel width
constexpr int kClassS = 96;   // size classes: the packed FP64 matrix in shared memory up to N = 218
constexpr int kClassM = 160;
constexpr int kClassL = 218;
constexpr int kClassXL = kMaxNmax;

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
  // neighbour cells are spread over the warps (their hash lookups and member scans overlap)
  const int side = 2 * R + 1, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int nnb = p.dim == 3 ? side * side * side : side * side;
  for (int v = threadIdx.x >> 5; v < nnb; v += nwarps) {
    const int dx = v % side - R, dy = (v / side) % side - R, dz = p.dim == 3 ? v / (side * side) - R : 0;
    int64_t nb[3] = {(int64_t)c[0] + dx, (int64_t)c[1] + dy, (int64_t)c[2] + dz};
    bool inr = true;
    for (int j = 0; j < 3; ++j) inr &= nb[j] >= -kBias && nb[j] < kBias;
    if (!inr) continue;
    const int h = hash_find(hk, hv, hcap, pack_key(nb[0], nb[1], nb[2]));
    if (h < 0) continue;
    for (int64_t t = own_off[h] + lane; t < own_off[h + 1]; t += 32) {
      const uint32_t id = own_id[t];
      const double* xi = x + (int64_t)id * p.dim;
      bool in = true;
      for (int j = 0; j < p.dim; ++j) in &= (xi[j] >= lo[j]) && (xi[j] < hi[j]);
      if (in) {
        const int pos = atomicAdd(&cnt, 1);
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

__global__ void k_sizes(const int64_t* n, int64_t G, int64_t* tri, int64_t* lb, int32_t* n32) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  tri[g] = tri_sz(n[g]);
  lb[g] = linv_blocked_size(n[g]);
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
                                 const float* nrm, int32_t* mgid, D4* md4, float4* mf4, float* mvar, float4* mnrm) {
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

struct FitArgs {
  const uint32_t* order;  // cells by descending N; this launch takes order[first .. first + count)
  int64_t first, count;
  const int32_t* n32;
  const int64_t* ts_off;
  const int64_t* chol_off;
  const int64_t* linv_off;
  D4* md4;
  float4* mf4;
  const float* mvar;
  double* chol64;
  float* linv32;
  int32_t* status;
  double* gscr;     // per-CTA global slot (largest class): tri(np) doubles
  int64_t gstride;  // doubles per slot
  int np;           // largest N of this class
  int smem_mat;     // 1: the matrix lives in shared memory
  int* counter;
  int* n_not_pd;
};

__device__ __forceinline__ int64_t P(int i, int j) { return tri_sz(i) + j; }

// row of the packed lower-triangle entry t (t = i (i+1)/2 + j, j <= i)
__device__ __forceinline__ int tri_row(int64_t t) {
  int i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while (tri_sz(i + 1) <= t) ++i;
  while (tri_sz(i) > t) --i;
  return i;
}

__device__ __forceinline__ double kernel_entry(const double* sx, int i, int j, double lam, const double* tab) {
  const double dx = sx[3 * i] - sx[3 * j], dy = sx[3 * i + 1] - sx[3 * j + 1], dz = sx[3 * i + 2] - sx[3 * j + 2];
  const double e = lam * (dx * dx + dy * dy + dz * dz);
  return e > 50.0 ? 0.0 : exp_neg64(-e, tab);  // entries below e^-50 ~ 2e-22 are zero
}

constexpr int kInvRows = 2;  // rows per thread in the FP32 inversion (N <= 2 * blockDim.x)

// One cell per iteration of a persistent CTA:
//   A = K + diag(sigma^2) (FP64, packed lower), blocked Cholesky (FP64: 16-column panels factored by warp 0
//   with rsqrt pivots, trailing updates in 2x2 register blocks by the whole CTA), alpha by two FP64
//   triangular solves (warp 0) while the other warps copy L out; then L is converted in place to FP32 and
//   inverted column by column (all threads), and L^{-1} is written in 8-row blocks.
__global__ void __launch_bounds__(256) k_fit(FitArgs a, Params p) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_cell, s_fail;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  double* tab = sm;
  double* dinv = tab + kExpTab;
  double* sx = dinv + a.np;
  double* sb = sx + 3 * a.np;
  double* A = a.smem_mat ? sb + a.np : a.gscr + (int64_t)blockIdx.x * a.gstride;
  float* X = reinterpret_cast<float*>(A);  // L^{-1} in FP32 overwrites the FP64 factor at the end
  for (int i = tid; i < kExpTab; i += nthr) tab[i] = kExp2FracTab[i];
  const double lam = p.lambda;
  for (;;) {
    if (tid == 0) {
      int w = atomicAdd(a.counter, 1);
      s_cell = w < a.count ? (int)a.order[a.first + w] : -1;
      s_fail = 0;
    }
    __syncthreads();
    const int g = s_cell;
    if (g < 0) break;
    const int N = a.n32[g];
    if (N == 0) {
      __syncthreads();
      continue;
    }
    const int64_t m0 = a.ts_off[g];
    const int64_t T = tri_sz(N);
    for (int i = tid; i < N; i += nthr) {
      const D4 v = a.md4[m0 + i];
      sx[3 * i] = v.x;
      sx[3 * i + 1] = v.y;
      sx[3 * i + 2] = v.z;
    }
    __syncthreads();
    // A = K + diag(sigma^2): two independent entries per thread and iteration
    for (int64_t t0 = tid; t0 < T; t0 += 2 * nthr) {
      const int64_t t1 = t0 + nthr;
      const int i0 = tri_row(t0), j0 = (int)(t0 - tri_sz(i0));
      const int i1 = t1 < T ? tri_row(t1) : i0, j1 = t1 < T ? (int)(t1 - tri_sz(i1)) : j0;
      double v0 = kernel_entry(sx, i0, j0, lam, tab);
      double v1 = kernel_entry(sx, i1, j1, lam, tab);
      if (i0 == j0) v0 += (double)a.mvar[m0 + i0];
      if (i1 == j1) v1 += (double)a.mvar[m0 + i1];
      A[t0] = v0;
      if (t1 < T) A[t1] = v1;
    }
    __syncthreads();
    for (int kb = 0; kb < N; kb += kPanel) {
      const int ke = min(kb + kPanel, N);
      if (warp == 0) {
        for (int k = kb; k < ke; ++k) {
          int bad = 0;
          double r = 0.0;
          if (lane == 0) {
            const double piv = A[P(k, k)];
            if (!(piv > 0.0)) {
              bad = 1;
            } else {
              r = rsqrt(piv);
              A[P(k, k)] = piv * r;
              dinv[k] = r;
            }
          }
          bad = __shfl_sync(0xffffffffu, bad, 0);
          r = __shfl_sync(0xffffffffu, r, 0);
          if (bad) {
            if (lane == 0) s_fail = 1;
            break;
          }
          for (int i = k + 1 + lane; i < N; i += 32) A[P(i, k)] *= r;
          __syncwarp();
          for (int i = k + 1 + lane; i < N; i += 32) {
            const double lik = A[P(i, k)];
            const int cmax = min(i, ke - 1);
            for (int c = k + 1; c <= cmax; ++c) A[P(i, c)] = fma(-lik, A[P(c, k)], A[P(i, c)]);
          }
          __syncwarp();
        }
      }
      __syncthreads();
      if (s_fail) break;
      // trailing update A[i][j] -= sum_{k in panel} L[i][k] L[j][k] for ke <= j <= i, in 2x2 blocks
      const int w = ke - kb, nbk = (N - ke + 1) >> 1;
      const int64_t nblk = tri_sz(nbk);
      for (int64_t t = tid; t < nblk; t += nthr) {
        const int I = tri_row(t), J = (int)(t - tri_sz(I));
        const int i0 = ke + 2 * I, j0 = ke + 2 * J, i1 = i0 + 1, j1 = j0 + 1;
        const bool vi1 = i1 < N, v01 = j1 <= i0, vj1 = j1 < N;
        const double* Li0 = A + P(i0, kb);
        const double* Li1 = vi1 ? A + P(i1, kb) : Li0;
        const double* Lj0 = A + P(j0, kb);
        const double* Lj1 = vj1 ? A + P(j1, kb) : Lj0;
        double a00 = A[P(i0, j0)];
        double a01 = v01 ? A[P(i0, j1)] : 0.0;
        double a10 = vi1 ? A[P(i1, j0)] : 0.0;
        double a11 = vi1 ? A[P(i1, j1)] : 0.0;
        for (int k = 0; k < w; ++k) {
          const double li0 = Li0[k], li1 = Li1[k], lj0 = Lj0[k], lj1 = Lj1[k];
          a00 = fma(-li0, lj0, a00);
          a01 = fma(-li0, lj1, a01);
          a10 = fma(-li1, lj0, a10);
          a11 = fma(-li1, lj1, a11);
        }
        A[P(i0, j0)] = a00;
        if (v01) A[P(i0, j1)] = a01;
        if (vi1) {
          A[P(i1, j0)] = a10;
          A[P(i1, j1)] = a11;
        }
      }
      __syncthreads();
    }
    if (s_fail) {
      if (tid == 0) {
        a.status[g] = KSDF_CELL_NOT_PD;
        atomicAdd(a.n_not_pd, 1);
      }
      for (int i = tid; i < N; i += nthr) {
        a.md4[m0 + i].w = 0.0;
        a.mf4[m0 + i].w = 0.f;
      }
      __syncthreads();
      continue;
    }
    if (warp == 0) {
      // alpha: L y = 1, then L^T alpha = y (FP64, reciprocal pivots)
      for (int i = lane; i < N; i += 32) sb[i] = 1.0;
      __syncwarp();
      for (int k = 0; k < N; ++k) {
        const double bk = sb[k] * dinv[k];
        for (int i = k + 1 + lane; i < N; i += 32) sb[i] = fma(-A[P(i, k)], bk, sb[i]);
        __syncwarp();
        if (lane == 0) sb[k] = bk;
        __syncwarp();
      }
      for (int k = N - 1; k >= 0; --k) {
        const double bk = sb[k] * dinv[k];
        for (int i = lane; i < k; i += 32) sb[i] = fma(-A[P(k, i)], bk, sb[i]);
        __syncwarp();
        if (lane == 0) sb[k] = bk;
        __syncwarp();
      }
    } else {
      double* Lout = a.chol64 + a.chol_off[g];
      for (int64_t e = tid - 32; e < T; e += nthr - 32) Lout[e] = A[e];
    }
    __syncthreads();
    for (int i = tid; i < N; i += nthr) {
      a.md4[m0 + i].w = sb[i];
      a.mf4[m0 + i].w = (float)sb[i];
    }
    // FP64 -> FP32 in place, in chunks: the writes of a chunk only touch FP64 entries already read
    for (int64_t c0 = 0; c0 < T; c0 += 8 * (int64_t)nthr) {
      float v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t e = c0 + tid + (int64_t)r * nthr;
        v[r] = e < T ? (float)A[e] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t e = c0 + tid + (int64_t)r * nthr;
        if (e < T) X[e] = v[r];
      }
      __syncthreads();
    }
    // X = L^{-1}: column j (from the last) becomes X[j][j] = 1/L_jj,
    // X[i][j] = -X[j][j] sum_{k=j+1..i} X[i][k] L[k][j] (i > j), reading finished columns k > j of X and
    // the untouched column j of L
    for (int j = N - 1; j >= 0; --j) {
      float tv[kInvRows];
#pragma unroll
      for (int r = 0; r < kInvRows; ++r) {
        const int i = j + 1 + tid + r * nthr;
        float acc = 0.f;
        if (i < N) {
          const float* Xi = X + P(i, 0);
          for (int k = j + 1; k <= i; ++k) acc = fmaf(Xi[k], X[P(k, j)], acc);
        }
        tv[r] = acc;
      }
      __syncthreads();
      const float xjj = (float)dinv[j];
#pragma unroll
      for (int r = 0; r < kInvRows; ++r) {
        const int i = j + 1 + tid + r * nthr;
        if (i < N) X[P(i, j)] = -xjj * tv[r];
      }
      if (tid == 0) X[P(j, j)] = xjj;
      __syncthreads();
    }
    float* Iout = a.linv32 + a.linv_off[g];
    const int64_t lsz = linv_blocked_size(N);
    for (int64_t e = tid; e < lsz; e += nthr) {
      int R = (int)((sqrtf(1.f + (float)e / 8.f) - 1.f) * 0.5f);
      while (linv_block_off(R + 1) <= e) ++R;
      while (linv_block_off(R) > e) --R;
      const int64_t q = e - linv_block_off(R);
      const int col = (int)(q >> 3), i = 8 * R + (int)(q & 7);
      Iout[e] = (i < N && col <= i) ? X[P(i, col)] : 0.f;
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

static size_t fit_smem(int np, bool smem_mat) {
  size_t d = kExpTab + 5 * (size_t)np;  // exp table, reciprocal pivots, coordinates, right-hand side
  if (smem_mat) d += (size_t)tri_sz(np);
  return d * sizeof(double);
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
  KSDF_CUDA(c, ensure(m.chol_off, sizeof(int64_t) * (G + 1)));
  KSDF_CUDA(c, ensure(m.linv_off, sizeof(int64_t) * (G + 1)));
  KSDF_CUDA(c, ensure(c->ws[WS_D], sizeof(int64_t) * (3 * G + 3)));
  int64_t* n64 = ptr<int64_t>(c->ws[WS_D]);
  int64_t* tri64 = n64 + (G + 1);
  int64_t* lb64 = tri64 + (G + 1);
  int* dmax = bbox + 6;
  KSDF_CUDA(c, cudaMemsetAsync(dmax, 0, sizeof(int) * 2, st));
  launch(k_assemble, (unsigned)G, 512, 0, st, ptr<uint64_t>(m.key), G, own_off, vals, x, p, R, ptr<uint64_t>(m.hkeys),
         ptr<int32_t>(m.hvals), cap, ptr<int32_t>(m.mpad), n64, ptr<int32_t>(m.status), dmax, stw);
  launch(k_sizes, ceil_div(G, 256), 256, 0, st, n64, G, tri64, lb64, ptr<int32_t>(m.n));
  KSDF_CUDA(c, scan_i64(n64, ptr<int64_t>(m.ts_off), G, dtot, c->ws[WS_SCAN], st));
  KSDF_CUDA(c, scan_i64(tri64, ptr<int64_t>(m.chol_off), G, dtot + 1, c->ws[WS_SCAN], st));
  KSDF_CUDA(c, scan_i64(lb64, ptr<int64_t>(m.linv_off), G, dtot + 2, c->ws[WS_SCAN], st));
  int64_t tots[3];
  int hmax[2];
  KSDF_CUDA(c, cudaMemcpyAsync(tots, dtot, sizeof(tots), cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaMemcpyAsync(hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaMemcpyAsync(&hst, stw, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaStreamSynchronize(st));
  if (hst & ST_CAPACITY)
    return set_err(c, KSDF_ERR_CAPACITY, "ksdf_fit: a collection box holds more than %d samples", kMaxPre);
  m.M = tots[0];
  m.chol_total = tots[1];
  m.linv_total = tots[2];
  m.max_n = hmax[0];
  KSDF_CUDA(c, cudaMemcpyAsync(ptr<int64_t>(m.ts_off) + G, &tots[0], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  KSDF_CUDA(c, cudaMemcpyAsync(ptr<int64_t>(m.chol_off) + G, &tots[1], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  KSDF_CUDA(c, cudaMemcpyAsync(ptr<int64_t>(m.linv_off) + G, &tots[2], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  prof_end(c, e0, "fit.assemble");
  // 4. member arrays
  const int64_t M = m.M;
  m.has_normals = nrm != nullptr;
  KSDF_CUDA(c, ensure(m.mgid, sizeof(int32_t) * (M + 1)));
  KSDF_CUDA(c, ensure(m.md4, sizeof(D4) * (M + 1)));
  KSDF_CUDA(c, ensure(m.mf4, sizeof(float4) * (M + 1)));
  KSDF_CUDA(c, ensure(m.mvar, sizeof(float) * (M + 1)));
  if (nrm) KSDF_CUDA(c, ensure(m.mnrm, sizeof(float4) * (M + 1)));
  KSDF_CUDA(c, ensure(m.chol64, sizeof(double) * (m.chol_total + 1)));
  KSDF_CUDA(c, ensure(m.linv32, sizeof(float) * (m.linv_total + 4)));
  launch(k_gather_members, ceil_div(G * p.n_max, 256), 256, 0, st, ptr<uint64_t>(m.key), ptr<int32_t>(m.n),
         ptr<int64_t>(m.ts_off), ptr<int32_t>(m.mpad), G, p, x, var, nrm, ptr<int32_t>(m.mgid), ptr<D4>(m.md4),
         ptr<float4>(m.mf4), ptr<float>(m.mvar), nrm ? ptr<float4>(m.mnrm) : nullptr);
  // 5. the fit, largest cells first, three size classes on three streams
  KSDF_CUDA(c, ensure(c->ws[WS_A], sizeof(uint64_t) * (G + 1)));
  KSDF_CUDA(c, ensure(m.cell_order, sizeof(uint32_t) * (G + 1)));
  uint64_t* okeys = ptr<uint64_t>(c->ws[WS_A]);
  uint32_t* order = ptr<uint32_t>(m.cell_order);
  launch(k_order_keys, ceil_div(G, 256), 256, 0, st, ptr<int32_t>(m.n), G, p.n_max, okeys, order);
  KSDF_CUDA(c, radix_sort_u64(okeys, order, G, bits_for((uint64_t)p.n_max), c->ws[WS_SORT], st));
  // size classes (host histogram): N <= 96 (128 threads), <= 160, <= 218 (256 threads, matrix in shared
  // memory), larger (256 threads, matrix in a per-CTA global slot); launched concurrently, largest first
  std::vector<int32_t> hn((size_t)G);
  KSDF_CUDA(c, cudaMemcpyAsync(hn.data(), m.n.p, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaStreamSynchronize(st));
  const int lim[4] = {kClassXL, kClassL, kClassM, kClassS};  // upper bounds, descending
  int64_t cnt[4] = {0, 0, 0, 0};
  for (int32_t v : hn) {
    if (v > kClassL) ++cnt[0];
    else if (v > kClassM) ++cnt[1];
    else if (v > kClassS) ++cnt[2];
    else ++cnt[3];
  }
  KSDF_CUDA(c, cudaMemsetAsync(dmax, 0, sizeof(int) * 2, st));
  KSDF_CUDA(c, ensure(c->ws[WS_E], sizeof(int64_t) * 4 + sizeof(int) * 8));
  int* ctr = reinterpret_cast<int*>(ptr<int64_t>(c->ws[WS_E]) + 4);
  KSDF_CUDA(c, cudaMemsetAsync(ctr, 0, sizeof(int) * 4, st));
  FitArgs fa;
  fa.order = order;
  fa.n32 = ptr<int32_t>(m.n);
  fa.ts_off = ptr<int64_t>(m.ts_off);
  fa.chol_off = ptr<int64_t>(m.chol_off);
  fa.linv_off = ptr<int64_t>(m.linv_off);
  fa.md4 = ptr<D4>(m.md4);
  fa.mf4 = ptr<float4>(m.mf4);
  fa.mvar = ptr<float>(m.mvar);
  fa.chol64 = ptr<double>(m.chol64);
  fa.linv32 = ptr<float>(m.linv32);
  fa.status = ptr<int32_t>(m.status);
  fa.n_not_pd = dmax + 1;
  fa.gscr = nullptr;
  fa.gstride = 0;
  KSDF_CUDA(c, cudaFuncSetAttribute(k_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fit_smem(kClassL, true)));
  e0 = prof_begin(c);
  KSDF_CUDA(c, fork_streams(c));
  int64_t first = 0;
  for (int cl = 0; cl < 4; ++cl) {
    if (cnt[cl] == 0) continue;
    FitArgs f = fa;
    f.first = first;
    f.count = cnt[cl];
    f.counter = ctr + cl;
    first += cnt[cl];
    const int threads = cl == 3 ? 128 : 256;
    f.smem_mat = cl > 0 ? 1 : 0;
    f.np = cl > 0 ? lim[cl] : std::max(m.max_n, 1);
    if (cl == 0) {
      const int nblk = (int)std::min<int64_t>(cnt[cl], c->num_sms);
      f.gstride = tri_sz(f.np);
      KSDF_CUDA(c, ensure(c->ws[WS_FITSCR], sizeof(double) * (size_t)(f.gstride * nblk + 1)));
      f.gscr = ptr<double>(c->ws[WS_FITSCR]);
    }
    const size_t smem = fit_smem(f.np, f.smem_mat != 0);
    int occ = 0;
    KSDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fit, threads, smem));
    const int nblk = (int)std::min<int64_t>(cnt[cl], (int64_t)std::max(1, occ) * c->num_sms);
    cudaStream_t s = cl == 3 ? st : c->aux[cl & 1];
    launch(k_fit, nblk, threads, smem, s, f, p);
  }
  KSDF_CUDA(c, cudaGetLastError());
  KSDF_CUDA(c, join_streams(c));
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
