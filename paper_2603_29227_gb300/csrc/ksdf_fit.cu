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

#include <cmath>
#include <cstdarg>
#include <vector>

namespace ksdf {

namespace {


__global__ void k_bin_samples(const double* x, const float* var, int64_t S, Params p, uint64_t* keys, uint32_t* vals,
                              int* bbox, uint32_t* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int c[3] = {0, 0, 0};
  bool ok = true, live = i < S;
  if (live) {
    for (int j = 0; j < p.dim; ++j) ok &= bin_coord(x[i * p.dim + j], p.o[j], p.h, p.rh, c[j]);
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

// integer key with the order of the binary64 values (non-NaN; -0 and +0 equal): x < y iff key(x) < key(y)
__device__ __forceinline__ long long f64_order_key(double v) {
  long long b = __double_as_longlong(v);
  if (b == (long long)0x8000000000000000ull) b = 0;
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
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

// training set of one cell per CTA: collection-box members, ascending global id, rank-selected cap.  128
// threads: the neighbour cells' scans spread over four warps, and a cell's candidates (tens to a few
// hundred) sort with few idle threads at the bitonic network's barriers
constexpr int kAssembleThreads = 128;
__global__ void __launch_bounds__(kAssembleThreads) k_assemble(const uint64_t* cell_key, int64_t G, const int64_t* own_off,
                                                  const uint32_t* own_id, const double* x, Params p, int R,
                                                  const uint64_t* hk, const int32_t* hv, uint64_t hcap,
                                                  int32_t* mpad, int64_t* n_out, int32_t* status, int* max_n,
                                                  uint32_t* st) {
  __shared__ int ids[kMaxPre];
  __shared__ int cnt;
  __shared__ long long s_lo[3], s_hi[3];
  const int64_t g = blockIdx.x;
  if (g >= G) return;
  int c[3];
  unpack_key(cell_key[g], c[0], c[1], c[2]);
  // the box [lo, hi) in binary64 (computed once), compared through order-preserving integer keys
  if (threadIdx.x == 0) {
    cnt = 0;
    for (int j = 0; j < 3; ++j) {
      s_lo[j] = f64_order_key(__dsub_rn(cell_base(p.o[j], c[j], p.h), p.mu));
      s_hi[j] = f64_order_key(__dadd_rn(cell_base(p.o[j], c[j] + 1, p.h), p.mu));
    }
  }
  __syncthreads();
  const long long lo[3] = {s_lo[0], s_lo[1], s_lo[2]}, hi[3] = {s_hi[0], s_hi[1], s_hi[2]};
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
      for (int j = 0; j < p.dim; ++j) {
        const long long k = f64_order_key(xi[j]);
        in &= (k >= lo[j]) && (k < hi[j]);
      }
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

__global__ void k_sizes(const int64_t* n, int64_t G, int64_t* tri, int64_t* lb, int64_t* tc, int32_t* n32) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  tri[g] = tri_sz(n[g]);
  lb[g] = linv_blocked_size(n[g]);
  tc[g] = ltc_size(n[g]);
  n32[g] = (int32_t)n[g];
}

// fit order: descending size; cells not to be fitted (touched == 0) sort after every other
// ---- refit scheduling (Sec. IV-C, App. G) ----
// Per cell g of the new model (a warp each): its previous cell (by key), whether its freshly assembled training
// set (mpad, n64) differs from the one the previous model was fitted on, the carried counters (c2 + 1 when it
// changed) and the priority key of the training queue: 0 for a cell that must be fitted (new, or previously not
// fitted), 1 + (2^32 - 1 - bits(s)) for a changed cell with score s = c2 (1 + eta c0) (FP32, rounded step by step,
// so larger scores come first), 2^40 for an unchanged cell.  Ties keep cell order (ascending key).
__global__ void k_sched_score(const uint64_t* key, const int64_t* n64, const int32_t* mpad, int64_t G, int n_max,
                              const uint64_t* ohk, const int32_t* ohv, uint64_t ohcap, const int32_t* on32,
                              const int64_t* ots_off, const int32_t* omgid, const int32_t* ostatus,
                              const int32_t* oc0, const int32_t* oc2, float eta, int32_t* c0, int32_t* c2,
                              int32_t* oid, int32_t* chg, uint64_t* skey, uint32_t* sval) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= G) return;
  const int o = hash_find(ohk, ohv, ohcap, key[g]);
  const int n = (int)n64[g];
  const bool fitted_before = o >= 0 && ostatus[o] == KSDF_CELL_OK;
  bool same = fitted_before && on32[o] == n && n > 0;
  if (same) {
    const int32_t* a = mpad + g * n_max;
    const int32_t* b = omgid + ots_off[o];
    bool eq = true;
    for (int i = lane; i < n; i += 32) eq &= a[i] == b[i];
    same = __all_sync(0xffffffffu, eq);
  }
  if (lane == 0) {
    const int q0 = o >= 0 ? oc0[o] : 0, q2 = (o >= 0 ? oc2[o] : 0) + (same ? 0 : 1);
    c0[g] = q0;
    c2[g] = q2;
    oid[g] = o;
    chg[g] = same ? 0 : 1;
    uint64_t k = 1ull << 40;
    if (!fitted_before) {
      k = 0;
    } else if (!same) {
      const float sc = __fmul_rn((float)q2, __fadd_rn(1.f, __fmul_rn(eta, (float)q0)));
      k = 1ull + (0xFFFFFFFFull - (uint64_t)__float_as_uint(sc));
    }
    skey[g] = k;
    sval[g] = (uint32_t)g;
  }
}

// the first `budget` cells in priority order are fitted (cells that must be fitted always are); the other changed
// cells are deferred
__global__ void k_sched_select(const uint64_t* skey, const uint32_t* sval, int64_t G, int64_t budget, int32_t* sel) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= G) return;
  const uint64_t k = skey[r];
  sel[sval[r]] = (k == 0 || (k < (1ull << 40) && r < budget)) ? 1 : 0;
}

// a deferred cell keeps the training set its previous fit was made on (a warp per cell)
__global__ void k_sched_defer(const int32_t* chg, const int32_t* sel, const int32_t* oid, int64_t G, int n_max,
                              const int32_t* on32, const int64_t* ots_off, const int32_t* omgid, int32_t* mpad,
                              int64_t* n64, int* max_n) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= G || !chg[g] || sel[g]) return;
  const int o = oid[g], n = on32[o];
  for (int i = lane; i < n; i += 32) mpad[g * n_max + i] = omgid[ots_off[o] + i];
  if (lane == 0) {
    n64[g] = n;
    atomicMax(max_n, n);
  }
}

// after the fit: the cells fitted now (all of them on a fresh fit) reset their training marks and halve their
// query counters
__global__ void k_sched_after(const int32_t* touched, int64_t G, int32_t* c0, int32_t* c2, int32_t* refit) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int r = touched ? touched[g] : 1;
  refit[g] = r;
  if (r) {
    c2[g] = 0;
    c0[g] >>= 1;
  }
}

__global__ void k_order_keys(const int32_t* n32, const int32_t* touched, int64_t G, int n_max, uint64_t* keys,
                             uint32_t* vals) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  keys[g] = (!touched || touched[g]) ? (uint64_t)(n_max - n32[g]) : (uint64_t)(n_max + 1);
  vals[g] = (uint32_t)g;
}

// update: touched[g] = 1 unless the previous model has a cell with the same key, an OK fit and the same
// training set (member ids in the same order); oid[g] = that cell's id (or -1).  One warp per cell.
__global__ void k_touched(const uint64_t* key, const int32_t* n32, const int64_t* ts_off, const int32_t* mgid,
                          int64_t G, const uint64_t* ohk, const int32_t* ohv, uint64_t ohcap, const int32_t* on32,
                          const int64_t* ots_off, const int32_t* omgid, const int32_t* ostatus, int32_t* touched,
                          int32_t* oid) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= G) return;
  const int o = hash_find(ohk, ohv, ohcap, key[g]);
  const int n = n32[g];
  bool same = o >= 0 && on32[o] == n && ostatus[o] == KSDF_CELL_OK && n > 0;
  if (same) {
    const int32_t* a = mgid + ts_off[g];
    const int32_t* b = omgid + ots_off[o];
    bool eq = true;
    for (int i = lane; i < n; i += 32) eq &= a[i] == b[i];
    same = __all_sync(0xffffffffu, eq);
  }
  if (lane == 0) {
    touched[g] = same ? 0 : 1;
    oid[g] = o;
  }
}

// update: an unchanged cell takes the previous model's fit (factor, L^-1 in both layouts, alpha, status)
struct CopyFitArgs {
  const int32_t *touched, *oid, *n32;
  int64_t G;
  const int64_t *ts_off, *chol_off, *linv_off, *ltc_off;
  const int64_t *ots_off, *ochol_off, *olinv_off, *oltc_off;
  const double* ochol64;
  const float *olinv32, *oltc;
  const D4* omd4;
  double* chol64;
  float *linv32, *ltc;
  D4* md4;
  float4* mf4;
  int32_t* status;
};

__global__ void k_copy_fit(CopyFitArgs a) {
  for (int64_t g = blockIdx.x; g < a.G; g += gridDim.x) {
    if (a.touched[g]) continue;
    const int o = a.oid[g], n = a.n32[g];
    const int64_t T = tri_sz(n), lb = linv_blocked_size(n), tc = ltc_size(n);
    const double* sc = a.ochol64 + a.ochol_off[o];
    double* dc = a.chol64 + a.chol_off[g];
    for (int64_t e = threadIdx.x; e < T; e += blockDim.x) dc[e] = sc[e];
    const float* sl = a.olinv32 + a.olinv_off[o];
    float* dl = a.linv32 + a.linv_off[g];
    for (int64_t e = threadIdx.x; e < lb; e += blockDim.x) dl[e] = sl[e];
    const float* st = a.oltc + a.oltc_off[o];
    float* dt = a.ltc + a.ltc_off[g];
    for (int64_t e = threadIdx.x; e < tc; e += blockDim.x) dt[e] = st[e];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double al = a.omd4[a.ots_off[o] + i].w;
      a.md4[a.ts_off[g] + i].w = al;
      a.mf4[a.ts_off[g] + i].w = d2f_bits(al);  // as the fit writes it
    }
    if (threadIdx.x == 0) a.status[g] = KSDF_CELL_OK;
  }
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
  double* gscr;     // per-CTA global slot (largest class): tri(np + 1) doubles
  int64_t gstride;  // doubles per slot
  int np;           // largest N of this class
  int* counter;
  int* n_not_pd;
};

// The kernel matrices of the cells order[0 .. count), each written (lower triangle with its diagonal) where
// the cell's Cholesky factor will go: k_fit reads it back from there.
struct KmatArgs {
  const uint32_t* order;  // this launch takes order[first .. first + count)
  int64_t first, count;
  int* counter;
  const int32_t* n32;
  const int64_t* ts_off;
  const int64_t* chol_off;
  const D4* md4;
  const float4* mf4;
  const float* mvar;
  double* chol64;
  int np;      // largest N
  double sc;   // sqrt(lambda 2^16 / ln2): coordinates scaled so that |s_i - s_j|^2 is exp2_neg_q16's argument
  float lamf;  // lambda in FP32 (the near/far screen)
  bool fixed;  // scaled coordinates below 2^21: exact fixed-point squared distances (else binary64)
};

// row of the packed lower-triangle entry t (t = i (i+1)/2 + j, j <= i)
__device__ __forceinline__ int tri_row(int64_t t) {
  int i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while (tri_sz(i + 1) <= t) ++i;
  while (tri_sz(i) > t) --i;
  return i;
}

constexpr int kB = 8;        // Cholesky panel width
constexpr float kNearE = 36.f;  // RBF: lambda r^2 below this: FP64 entry; above: FP32 (value < 2.4e-16)
constexpr float kNearM = 42.f;  // Matern 3/2: lambda r below this: FP64 entry; above: FP32 (value < 2.5e-17)

// The kernel entry from the scaled coordinates.  RBF: exp(-lambda r_ij^2), coordinates scaled by
// sqrt(lambda 2^16 / ln2), in fixed point (exact squared distance; the slots hold the coordinates as 64-bit
// integers s 2^40) or binary64.  Matern 3/2: (1 + lambda r) exp(-lambda r), coordinates scaled by
// lambda 2^16 / ln2 so that the scaled distance is exp2_neg_q16's argument (binary64, correctly rounded sqrt).
template <bool MATERN>
__device__ __forceinline__ double near_entry(const double* s, const long long* sfix, bool fixed, int i, int j) {
  if (MATERN) {
    const double ex = s[3 * i] - s[3 * j], ey = s[3 * i + 1] - s[3 * j + 1], ez = s[3 * i + 2] - s[3 * j + 2];
    const double e = sqrt(fma(ez, ez, fma(ey, ey, ex * ex)));
    return fma(e, 1.0 / kExpQ16PerNat, 1.0) * exp2_neg_q16(e);
  }
  if (fixed)
    return exp2_neg_fixed40(sqdiff40(sfix[3 * i], sfix[3 * j]) + sqdiff40(sfix[3 * i + 1], sfix[3 * j + 1]) +
                            sqdiff40(sfix[3 * i + 2], sfix[3 * j + 2]));
  const double ex = s[3 * i] - s[3 * j], ey = s[3 * i + 1] - s[3 * j + 1], ez = s[3 * i + 2] - s[3 * j + 2];
  return exp2_neg_q16(fma(ez, ez, fma(ey, ey, ex * ex)));
}

__device__ __forceinline__ bool pivot_ok(double d) {  // finite, positive and normal
  const long long b = __double_as_longlong(d);
  const int ex = (int)((b >> 52) & 0x7ff);
  return b > 0 && ex > 0 && ex < 2047;
}

__device__ __forceinline__ void fit_sync(int team) {
  if (team == 32) __syncwarp();
  else __syncthreads();
}

constexpr int kKmatWarps = 4;

// per-warp shared memory of k_kmat (doubles), with np rounded up to even so that every region starts on
// 16 bytes (the FP32 coordinates are read as float4): scaled coordinates 3 np (binary64 or fixed point) |
// FP32 coordinates 4 np floats | near-entry queue 64 ints
__host__ __device__ inline int kmat_np_even(int np) { return (np + 1) & ~1; }
__host__ __device__ inline int64_t kmat_warp_doubles(int np) { return 5 * (int64_t)kmat_np_even(np) + 32; }

// The kernel matrix A = K + diag(sigma^2) of one cell per warp (persistent over the cells to fit).  Each
// off-diagonal entry is screened in FP32: lambda r^2 >= 36 gives a value below 2.4e-16 that FP32 evaluates to
// far better than its absolute rounding; the others are queued and evaluated 32 at a time in FP64
// (exp2_neg_q16 on coordinates pre-scaled by sqrt(lambda 2^16 / ln2)).  The scaled coordinates are held in
// fixed point with 40 fractional bits, so that the squared distance comes out of exact integer arithmetic as
// exp2_neg_fixed40's argument: 4 FP64 operations per entry instead of 10 (the rounding of s to 2^-41 moves
// an entry by below 1e-13 of its value).  A separate, high-occupancy kernel: the factorisation's warps then
// spend their time in the FP64 factorisation alone.
template <bool MATERN>
__global__ void __launch_bounds__(32 * kKmatWarps) k_kmat(KmatArgs a) {
  extern __shared__ __align__(16) double smk[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int npe = kmat_np_even(a.np);
  double* s = smk + warp * kmat_warp_doubles(a.np);
  long long* sfix = reinterpret_cast<long long*>(s);  // the same slots, fixed point (a.fixed)
  float* xf = reinterpret_cast<float*>(s + 3 * npe);
  int* qw = reinterpret_cast<int*>(xf + 4 * npe);
  const unsigned lt_mask = (1u << lane) - 1u;
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(a.counter, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= a.count) break;
    const int g = (int)a.order[a.first + w];
    const int N = a.n32[g];
    const int64_t m0 = a.ts_off[g];
    double* Ag = a.chol64 + a.chol_off[g];
    for (int i = lane; i < N; i += 32) {
      const D4 v = a.md4[m0 + i];
      const double sv[3] = {a.sc * v.x, a.sc * v.y, a.sc * v.z};
      for (int d = 0; d < 3; ++d) {
        if (a.fixed) sfix[3 * i + d] = __double2ll_rn(sv[d] * 0x1p40);
        else s[3 * i + d] = sv[d];
      }
      const float4 f = a.mf4[m0 + i];
      xf[4 * i] = f.x;
      xf[4 * i + 1] = f.y;
      xf[4 * i + 2] = f.z;
      Ag[tri_sz(i) + i] = 1.0 + f2d_bits(a.mvar[m0 + i]);  // exp(0) + sigma_i^2
    }
    __syncwarp();
    // the strictly lower pairs flattened, t = i (i - 1) / 2 + j, 32 consecutive pairs per step (full warps
    // for every row length); a lane walks its (i, j) forward by 32 each step
    const int64_t npair = (int64_t)N * (N - 1) / 2;
    int i = 1, j = lane;
    while (j >= i) {
      j -= i;
      ++i;
    }
    int qn = 0;
    for (int64_t t0 = 0; t0 < npair; t0 += 32) {
      bool near = false;
      if (t0 + lane < npair) {
        const float4 pi = reinterpret_cast<const float4*>(xf)[i];
        const float4 pj = reinterpret_cast<const float4*>(xf)[j];
        const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        if (MATERN) {
          const float ef = a.lamf * sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
          if (ef < kNearM) near = true;
          else Ag[tri_sz(i) + j] = f2d_bits((1.f + ef) * exp2f(-1.44269504f * ef));
        } else {
          const float ef = a.lamf * fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          if (ef < kNearE) near = true;
          else Ag[tri_sz(i) + j] = f2d_bits(exp2f(-1.44269504f * ef));
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, near);
      if (near) qw[qn + __popc(mask & lt_mask)] = (i << 16) | j;
      qn += __popc(mask);
      if (qn >= 32) {
        __syncwarp();
        const int ij = qw[lane];
        Ag[tri_sz(ij >> 16) + (ij & 0xffff)] = near_entry<MATERN>(s, sfix, a.fixed, ij >> 16, ij & 0xffff);
        __syncwarp();
        if (lane < qn - 32) qw[lane] = qw[32 + lane];
        qn -= 32;
        __syncwarp();
      }
      j += 32;
      while (j >= i) {
        j -= i;
        ++i;
      }
    }
    __syncwarp();
    if (lane < qn) {
      const int ij = qw[lane];
      Ag[tri_sz(ij >> 16) + (ij & 0xffff)] = near_entry<MATERN>(s, sfix, a.fixed, ij >> 16, ij & 0xffff);
    }
    __syncwarp();
  }
}

// Shared-memory layout of one cell's fit (doubles): two column buffers 2 (np + 1) | reciprocal pivots np |
// the augmented packed matrix tri(np + 1) (when it lives here).
__host__ __device__ inline int64_t fit_smem_doubles(int np, bool smem_mat) {
  return 2 * ((int64_t)np + 1) + np + (smem_mat ? tri_sz(np + 1) : 0);
}

// Panel kb..ke-1 of the packed augmented matrix A (rows up to N) by one warp: per column the pivot (its
// reciprocal square root kept in dinv; the diagonal keeps d_k), the column scaled, and the updates inside the
// panel flattened over (row, column) pairs so that each warp instruction carries 32 of them.  Sets *fail on an
// unusable pivot.
__device__ __forceinline__ void fit_factor_panel(double* A, double* dinv, int N, int kb, int ke, int* fail) {
  const int lane = threadIdx.x & 31;
  for (int c = kb; c < ke; ++c) {
    const double d = A[tri_sz(c) + c];
    if (!pivot_ok(d)) {
      if (lane == 0) *fail = 1;
      break;
    }
    const double y = rsqrt_pivot(d);
    if (lane == 0) dinv[c] = y;
    for (int i = c + 1 + lane; i <= N; i += 32) A[tri_sz(i) + c] *= y;
    __syncwarp();
    const int nc = ke - 1 - c;
    if (nc > 0) {
      const unsigned mg = 0xFFFFFFFFu / (unsigned)nc + 1u;  // t / nc = umulhi(t, mg) for t < 2^29, nc > 1
      const unsigned nt = (unsigned)(N - c) * (unsigned)nc;
      for (unsigned t = lane; t < nt; t += 32) {
        const unsigned q = nc == 1 ? t : __umulhi(t, mg);
        const int i = c + 1 + (int)q, j = c + 1 + (int)(t - q * (unsigned)nc);
        if (j <= i) A[tri_sz(i) + j] = fma(-A[tri_sz(i) + c], A[tri_sz(j) + c], A[tri_sz(i) + j]);
      }
      __syncwarp();
    }
  }
}

// The update of the 2 x 2 block of entries (i0, j0), (i0, j0+1), (i0+1, j0), (i0+1, j0+1) -- those with
// j <= i, i <= N and j < cmax -- by the w factored columns kb .. kb+w-1: a_ij -= sum_k L_ik L_jk, k in order.
__device__ __forceinline__ void fit_update_block(double* A, int N, int kb, int w, int i0, int j0, int cmax) {
  const int i1 = i0 + 1, j1 = j0 + 1;
  const bool vi1 = i1 <= N, vj1 = j1 < cmax, v01 = vj1 && j1 <= i0;
  double* Ai0 = A + tri_sz(i0);
  double* Ai1 = vi1 ? A + tri_sz(i1) : Ai0;
  const double* Li0 = Ai0 + kb;
  const double* Li1 = Ai1 + kb;
  const double* Lj0 = A + tri_sz(j0) + kb;
  const double* Lj1 = vj1 ? A + tri_sz(j1) + kb : Lj0;
  double a00 = Ai0[j0];
  double a01 = v01 ? Ai0[j1] : 0.0;
  double a10 = vi1 ? Ai1[j0] : 0.0;
  double a11 = (vi1 && vj1) ? Ai1[j1] : 0.0;
#pragma unroll
  for (int k = 0; k < kB; ++k) {
    if (k < w) {
      const double li0 = Li0[k], li1 = Li1[k], lj0 = Lj0[k], lj1 = Lj1[k];
      a00 = fma(-li0, lj0, a00);
      a01 = fma(-li0, lj1, a01);
      a10 = fma(-li1, lj0, a10);
      a11 = fma(-li1, lj1, a11);
    }
  }
  Ai0[j0] = a00;
  if (v01) Ai0[j1] = a01;
  if (vi1) {
    Ai1[j0] = a10;
    if (vj1) Ai1[j1] = a11;
  }
}

// Right-looking Cholesky of the augmented matrix in shared memory with a one-panel look-ahead (teams of
// TEAM >= 64 threads).  Per panel kb..ke-1, once it is factored:
//   1. the whole team updates the next panel's columns ke..ken-1 (rows ke..N) by it;
//   2. warp 0 factors the next panel while the team updates the rest of the trailing triangle (rows and
//      columns ken..N) by the current one, in chunks of 32 2 x 2 blocks taken from a shared counter, so that
//      warp 0 joins in when its panel is done.
template <int TEAM>
__device__ void fit_lookahead(double* A, double* dinv, int N, int& s_fail, int& s_next) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int kb = 0, ke = min(kB, N);
  if (warp == 0) fit_factor_panel(A, dinv, N, kb, ke, &s_fail);
  __syncthreads();
  while (!s_fail && ke < N) {
    const int w = ke - kb;
    const int ken = min(ke + kB, N);
    // 1. the next panel's columns: 2 x 2 blocks (ke + 2I, ke + 2J), J < 4, J <= I
    {
      const int nI = (N + 2 - ke) >> 1;
      for (int t = tid; t < 4 * nI; t += TEAM) {
        const int I = t >> 2, J = t & 3;
        const int i0 = ke + 2 * I, j0 = ke + 2 * J;
        if (J <= I && j0 < ken) fit_update_block(A, N, kb, w, i0, j0, ken);
      }
    }
    if (tid == 0) s_next = 0;
    __syncthreads();
    // 2. warp 0: the next panel; everyone: the trailing triangle beyond it
    if (warp == 0) fit_factor_panel(A, dinv, N, ke, ken, &s_fail);
    {
      const int nbk = (N + 2 - ken) >> 1;  // 2-row blocks over rows ken..N
      const int64_t nblk = tri_sz(nbk);
      for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&s_next, 32);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if ((int64_t)base >= nblk) break;
        const int64_t t = base + lane;
        if (t < nblk) {
          const int I = tri_row(t), J = (int)(t - tri_sz(I));
          fit_update_block(A, N, kb, w, ken + 2 * I, ken + 2 * J, N + 1);
        }
      }
    }
    __syncthreads();
    kb = ke;
    ke = ken;
  }
}

// The fit of one cell per iteration of a persistent team (TEAM threads; one warp for the small classes).
// On GB300 an SM retires one FP64 warp instruction per ~20 cycles (one per ~68 per scheduler) whether 1 or
// 32 lanes are active, so every step keeps its FP64 work in full warps:
//   1. A = K + diag(sigma^2) (written by k_kmat where L goes) is read into the team's matrix and augmented
//      with a row of ones (the right-hand side of A alpha = 1).
//   2. Right-looking Cholesky of the augmented matrix in panels of kB columns: warp 0 factors a panel
//      (pivots by rsqrt_pivot, column scaling, updates inside the panel flattened over the lanes), then the
//      team updates the trailing triangle in 2 x 2 register blocks over the panel depth.  The augmented row
//      ends as y = L^{-1} 1.
//   3. alpha = L^{-T} y by backward substitution (warp 0) while the other warps write L out.
// L^{-1} in FP32 follows in k_linv.
template <int TEAM, bool GMAT>
__global__ void __launch_bounds__(TEAM, TEAM == 32 ? 12 : 256 / TEAM) k_fit(FitArgs a, Params p) {
  constexpr int W = TEAM / 32;
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_cell, s_fail, s_next;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = a.np;
  double* cb = sm;
  double* dinv = cb + 2 * (np + 1);
  double* A = GMAT ? a.gscr + (int64_t)blockIdx.x * a.gstride : sm + fit_smem_doubles(np, false);
  double* P = sm + fit_smem_doubles(np, false);  // GMAT: the current panel, (np + 1) x kB
  for (;;) {
    if (tid == 0) {
      const int w = atomicAdd(a.counter, 1);
      s_cell = w < a.count ? (int)a.order[a.first + w] : -1;
      s_fail = 0;
    }
    fit_sync(TEAM);
    const int g = s_cell;
    if (g < 0) break;
    const int N = a.n32[g];
    if (N == 0) {
      fit_sync(TEAM);
      continue;
    }
    const int64_t m0 = a.ts_off[g];
    const int64_t T = tri_sz(N);
    // 1. the kernel matrix (eight loads in flight per thread) and the augmented row
    {
      const double* Ag = a.chol64 + a.chol_off[g];
      for (int64_t e0 = tid; e0 < T; e0 += 8 * (int64_t)TEAM) {
        double v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t e = e0 + (int64_t)r * TEAM;
          v[r] = e < T ? Ag[e] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t e = e0 + (int64_t)r * TEAM;
          if (e < T) A[e] = v[r];
        }
      }
      for (int i = tid; i < N; i += TEAM) A[T + i] = 1.0;
      if (tid == 0) A[T + N] = 0.0;  // never used; kept finite
    }
    fit_sync(TEAM);
    // 2. Cholesky of the augmented matrix in panels of kB columns: warp 0 factors the panel (pivots,
    //    column scaling, updates inside the panel), then the team updates the trailing triangle (rows and
    //    columns ke..N, the augmented row included) in 2 x 2 register blocks over the panel depth.  The
    //    diagonal keeps the pivot d_k until the end (L_kk = d_k / sqrt(d_k) is applied in bulk).
    //    Teams of two or more warps with the matrix in shared memory look one panel ahead: once a panel is
    //    factored, the team first brings the next panel's columns up to date, then warp 0 factors that
    //    panel while the other warps (and warp 0, when it is done) take the rest of the trailing update in
    //    chunks of 32 blocks.  Every entry receives the same FMAs in the same order either way.
    if (W > 1 && !GMAT) {
      fit_lookahead<TEAM>(A, dinv, N, s_fail, s_next);
    } else
    for (int kb = 0; kb < N; kb += kB) {
      const int ke = min(kb + kB, N);
      // the panel's element (row i >= kb, column kb <= c < ke): in the matrix itself, or (GMAT: the matrix
      // in a global slot) in a shared-memory copy of the panel, so that the panel's factorisation and the
      // trailing update read it from shared memory
      auto PE = [&](int i, int c) -> double& { return GMAT ? P[(i - kb) * kB + (c - kb)] : A[tri_sz(i) + c]; };
      if (GMAT) {
        for (int t = tid; t < (N + 1 - kb) * kB; t += TEAM) {
          const int i = kb + (t >> 3), col = kb + (t & 7);
          P[t] = (col < ke && col <= i) ? A[tri_sz(i) + col] : 0.0;
        }
        fit_sync(TEAM);
      }
      if (warp == 0) {
        for (int c = kb; c < ke; ++c) {
          const double d = PE(c, c);
          if (!pivot_ok(d)) {
            if (lane == 0) s_fail = 1;
            break;
          }
          const double y = rsqrt_pivot(d);
          if (lane == 0) dinv[c] = y;
          for (int i = c + 1 + lane; i <= N; i += 32) PE(i, c) *= y;
          __syncwarp();
          const int nc = ke - 1 - c;
          if (nc > 0) {
            // the (row, column) pairs of the update flattened over the lanes, so that each warp
            // instruction carries 32 of them: t -> row c + 1 + t / nc, column c + 1 + t % nc
            const unsigned mg = 0xFFFFFFFFu / (unsigned)nc + 1u;  // t / nc = umulhi(t, mg) for t < 2^29, nc > 1
            const unsigned nt = (unsigned)(N - c) * (unsigned)nc;
            for (unsigned t = lane; t < nt; t += 32) {
              const unsigned q = nc == 1 ? t : __umulhi(t, mg);
              const int i = c + 1 + (int)q, j = c + 1 + (int)(t - q * (unsigned)nc);
              if (j <= i) PE(i, j) = fma(-PE(i, c), PE(j, c), PE(i, j));
            }
            __syncwarp();
          }
        }
      }
      fit_sync(TEAM);
      if (s_fail) break;
      if (GMAT)  // the factored panel back into the matrix (columns disjoint from the trailing update's)
        for (int t = tid; t < (N + 1 - kb) * kB; t += TEAM) {
          const int i = kb + (t >> 3), col = kb + (t & 7);
          if (col < ke && col <= i) A[tri_sz(i) + col] = P[t];
        }
      const int w = ke - kb;
      const int nbk = (N + 2 - ke) >> 1;  // 2-row blocks over rows ke..N
      const int64_t nblk = tri_sz(nbk);
      // full rounds of 2 x 2 blocks (every thread busy); the last, partial round is done as single entries
      // below (a warp instruction costs the same FP64 pipe time however few lanes it has)
      const int64_t nfull = (nblk / TEAM) * TEAM;
      // (GMAT: the matrix is in a global slot; each thread loads its next block's four entries before this
      // block's FMAs, so that the L2 latency overlaps the FP64 work)
      double n00 = 0.0, n01 = 0.0, n10 = 0.0, n11 = 0.0;
      auto load_block = [&](int64_t tt) {
        const int I = tri_row(tt), J = (int)(tt - tri_sz(I));
        const int i0 = ke + 2 * I, j0 = ke + 2 * J;
        const double* Ai0 = A + tri_sz(i0);
        n00 = Ai0[j0];
        n01 = j0 + 1 <= i0 ? Ai0[j0 + 1] : 0.0;
        if (i0 + 1 <= N) {
          const double* Ai1 = A + tri_sz(i0 + 1);
          n10 = Ai1[j0];
          n11 = Ai1[j0 + 1];
        } else {
          n10 = n11 = 0.0;
        }
      };
      if (GMAT && tid < nfull) load_block(tid);
      for (int64_t t = tid; t < nfull; t += TEAM) {
        const int I = tri_row(t), J = (int)(t - tri_sz(I));
        const int i0 = ke + 2 * I, j0 = ke + 2 * J, i1 = i0 + 1, j1 = j0 + 1;
        const bool vi1 = i1 <= N, v01 = j1 <= i0, vj1 = j1 <= N;
        double* Ai0 = A + tri_sz(i0);
        double* Ai1 = vi1 ? A + tri_sz(i1) : Ai0;
        const double* Li0 = GMAT ? P + (i0 - kb) * kB : Ai0 + kb;
        const double* Li1 = GMAT ? (vi1 ? P + (i1 - kb) * kB : Li0) : Ai1 + kb;
        const double* Lj0 = GMAT ? P + (j0 - kb) * kB : A + tri_sz(j0) + kb;
        const double* Lj1 = vj1 ? (GMAT ? P + (j1 - kb) * kB : A + tri_sz(j1) + kb) : Lj0;
        double a00, a01, a10, a11;
        if (GMAT) {
          a00 = n00;
          a01 = n01;
          a10 = n10;
          a11 = n11;
          if (t + TEAM < nfull) load_block(t + TEAM);
        } else {
          a00 = Ai0[j0];
          a01 = v01 ? Ai0[j1] : 0.0;
          a10 = vi1 ? Ai1[j0] : 0.0;
          a11 = vi1 ? Ai1[j1] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < kB; ++k) {
          if (k < w) {
            const double li0 = Li0[k], li1 = Li1[k], lj0 = Lj0[k], lj1 = Lj1[k];
            a00 = fma(-li0, lj0, a00);
            a01 = fma(-li0, lj1, a01);
            a10 = fma(-li1, lj0, a10);
            a11 = fma(-li1, lj1, a11);
          }
        }
        Ai0[j0] = a00;
        if (v01) Ai0[j1] = a01;
        if (vi1) {
          Ai1[j0] = a10;
          Ai1[j1] = a11;
        }
      }
      for (int64_t e = tid; e < 4 * (nblk - nfull); e += TEAM) {
        const int64_t t = nfull + (e >> 2);
        const int I = tri_row(t), J = (int)(t - tri_sz(I));
        const int i = ke + 2 * I + (int)((e >> 1) & 1), j = ke + 2 * J + (int)(e & 1);
        if (i <= N && j <= i) {
          double* Aij = A + tri_sz(i) + j;
          const double* Li = GMAT ? P + (i - kb) * kB : A + tri_sz(i) + kb;
          const double* Lj = GMAT ? P + (j - kb) * kB : A + tri_sz(j) + kb;
          double acc = *Aij;
#pragma unroll
          for (int k = 0; k < kB; ++k)
            if (k < w) acc = fma(-Li[k], Lj[k], acc);
          *Aij = acc;
        }
      }
      fit_sync(TEAM);
    }
    if (s_fail) {
      if (tid == 0) {
        a.status[g] = KSDF_CELL_NOT_PD;
        atomicAdd(a.n_not_pd, 1);
      }
      for (int i = tid; i < N; i += TEAM) {
        a.md4[m0 + i].w = 0.0;
        a.mf4[m0 + i].w = 0.f;
      }
      fit_sync(TEAM);
      continue;
    }
    for (int k = tid; k < N; k += TEAM) A[tri_sz(k) + k] *= dinv[k];  // L_kk = d_k / sqrt(d_k)
    fit_sync(TEAM);
    // 3. alpha = L^{-T} y (warp 0); the other warps write L out meanwhile
    double* yb = cb;
    double* Lout = a.chol64 + a.chol_off[g];
    if (warp == 0) {
      for (int i = lane; i < N; i += 32) yb[i] = A[T + i];
      __syncwarp();
      for (int k = N - 1; k >= 0; --k) {
        const double ak = yb[k] * dinv[k];
        const double* Lk = A + tri_sz(k);
        for (int i = lane; i < k; i += 32) yb[i] = fma(-Lk[i], ak, yb[i]);
        __syncwarp();
        if (lane == 0) yb[k] = ak;
      }
    } else {
      for (int64_t e = tid - 32; e < T; e += TEAM - 32) Lout[e] = A[e];
    }
    fit_sync(TEAM);
    if (W == 1)
      for (int64_t e = tid; e < T; e += TEAM) Lout[e] = A[e];
    for (int i = tid; i < N; i += TEAM) {
      a.md4[m0 + i].w = yb[i];
      a.mf4[m0 + i].w = d2f_bits(yb[i]);
    }
    fit_sync(TEAM);
  }
}

// L^{-1} in FP32 for the variance contraction, one team per cell (persistent over cells order[first ..
// first + count)).  L is rounded to FP32 (integer-bit conversion) into shared memory and each column of X =
// L^{-1} is the forward substitution L x = e_j: X[j][j] = 1/L_jj and X[i][j] = -(sum_{k=j..i-1} L_ik X_kj) /
// L_ii for i > j.  A lane owns a column and a warp a group of 32 consecutive columns, walking the rows
// four at a time so that every X_kj load feeds four FFMAs; no synchronisation beyond the warp.
//   INPLACE (one warp, small cells): the groups run in order and X overwrites L (a group only reads L in
//     its own and later columns, and a row's L entries until that row is finished);
//   otherwise one warp per group, all groups concurrently, each with its own buffer of (np - 32 g) rows.
// The group's columns are then written in the 8-row blocked layout.  A separate kernel so that the fit's
// warps keep the FP64 pipe busy; this one is FP32 only.
struct LinvArgs {
  const uint32_t* order;
  int64_t first, count;
  const int32_t* n32;
  const int32_t* status;
  const int64_t* chol_off;
  const int64_t* linv_off;
  const double* chol64;
  float* linv32;
  const int64_t* ltc_off;
  float* ltc;       // the cell's image at ltc + ltc_off[g]
  float* gscr;      // per-CTA global slot (largest class): linv_slot_floats(np, false)
  int64_t gstride;
  int np;
  int* counter;
};

// float offset of group g's buffer (after the reciprocal diagonal and L) and the slot size
__host__ __device__ inline int64_t linv_group_off(int np, int g) {
  return (((int64_t)np + 3) & ~3LL) + tri_sz(np) + 32LL * ((int64_t)g * np - 32LL * tri_sz(g - 1));
}
__host__ __device__ inline int64_t linv_slot_floats(int np, bool inplace) {
  return inplace ? (((int64_t)np + 3) & ~3LL) + tri_sz(np) : linv_group_off(np, (np + 31) / 32);
}

// L^{-1} of the cells with N <= 256, a CTA of W warps per cell (persistent).  Shared memory holds L in FP32
// with every row padded to a multiple of four floats (row i at lrow_off(i)), the reciprocal diagonal, and per
// warp the 32 columns of its current group of X = L^{-1}, one per lane, stored column-major (Xt[c xs + i] =
// X[i][base + c], xs = 4 mod 32 so that the lanes' 16-byte loads are conflict-free).  The 32-column groups
// are independent (each reads only L): with two warps they are dealt out so that the warps' work, which
// falls with the group's first row, balances (0, 3, 4, 7, ... and 1, 2, 5, 6, ...).  A lane computes its
// column by forward substitution four rows at a time, walking k four at a time with 16-byte loads: five
// loads feed sixteen FFMAs (the L rows are broadcasts).  The group's columns are then written in the 8-row
// blocked layout and as the tensor-core images (coalesced float4 stores along the rows).
__host__ __device__ inline int lrow_off(int i) {
  const int q = i >> 2, r = i & 3;
  return 4 * (2 * q * (q + 1) + r * (q + 1));
}
__host__ __device__ inline int linv_small_stride(int np) { return 32 * ((np + 31) / 32) + 4; }
__host__ __device__ inline int64_t linv_small_floats(int np, int warps) {
  return lrow_off(np) + ((np + 3) & ~3) + 32LL * warps * linv_small_stride(np);
}

template <int W>
__global__ void __launch_bounds__(32 * W) k_linv_small(LinvArgs a) {
  extern __shared__ __align__(16) float smf[];
  __shared__ int s_cell;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = a.np;
  float* L = smf;
  float* dg = smf + lrow_off(np);
  const int xs = linv_small_stride(np);
  float* Xt = dg + ((np + 3) & ~3) + (int64_t)warp * 32 * xs;  // this warp's group buffer
  float* xc = Xt + lane * xs;  // this lane's column of the current group
  for (;;) {
    if (tid == 0) {
      const int w = atomicAdd(a.counter, 1);
      s_cell = w < a.count ? (int)a.order[a.first + w] : -1;
    }
    __syncthreads();
    const int g = s_cell;
    if (g < 0) break;
    const int N = a.n32[g];
    if (N == 0 || a.status[g] != KSDF_CELL_OK) {
      __syncthreads();
      continue;
    }
    // L: binary64 packed rows -> FP32 padded rows, eight loads in flight per lane; a lane walks its (row,
    // column) forward by 32 entries per load
    {
      const int64_t T = tri_sz(N);
      const double* Ld = a.chol64 + a.chol_off[g];
      int ri = 0, rk = tid;
      while (rk > ri) {
        rk -= ri + 1;
        ++ri;
      }
      for (int64_t e0 = tid; e0 < T; e0 += 8 * 32 * W) {
        double v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t e = e0 + 32 * W * r;
          v[r] = e < T ? Ld[e] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          if (e0 + 32 * W * r < T) L[lrow_off(ri) + rk] = d2f_bits(v[r]);
          rk += 32 * W;
          while (rk > ri) {
            rk -= ri + 1;
            ++ri;
          }
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < N; i += 32 * W) dg[i] = 1.f / L[lrow_off(i) + i];
    __syncthreads();
    float* Iout = a.linv32 + a.linv_off[g];
    const int nR = (N + 7) >> 3;
    for (int base = 0; base < N; base += 32) {
      const int grp = base >> 5;
      if (W == 2 && (((grp >> 1) ^ grp) & 1) != warp) continue;  // the other warp's group
      const int j = base + lane;
      for (int i0 = base; i0 < N; i0 += 4) {
        const float* L0 = L + lrow_off(i0);
        const float* L1 = L + lrow_off(min(i0 + 1, N - 1));
        const float* L2 = L + lrow_off(min(i0 + 2, N - 1));
        const float* L3 = L + lrow_off(min(i0 + 3, N - 1));
        float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
#pragma unroll 2
        for (int k0 = base; k0 < i0; k0 += 4) {
          const float4 x = *reinterpret_cast<const float4*>(xc + k0);
          const float4 l0 = *reinterpret_cast<const float4*>(L0 + k0);
          const float4 l1 = *reinterpret_cast<const float4*>(L1 + k0);
          const float4 l2 = *reinterpret_cast<const float4*>(L2 + k0);
          const float4 l3 = *reinterpret_cast<const float4*>(L3 + k0);
          c0 = fmaf(l0.w, x.w, fmaf(l0.z, x.z, fmaf(l0.y, x.y, fmaf(l0.x, x.x, c0))));
          c1 = fmaf(l1.w, x.w, fmaf(l1.z, x.z, fmaf(l1.y, x.y, fmaf(l1.x, x.x, c1))));
          c2 = fmaf(l2.w, x.w, fmaf(l2.z, x.z, fmaf(l2.y, x.y, fmaf(l2.x, x.x, c2))));
          c3 = fmaf(l3.w, x.w, fmaf(l3.z, x.z, fmaf(l3.y, x.y, fmaf(l3.x, x.x, c3))));
        }
        // the 4 x 4 block on the diagonal, row by row
        float xv[4] = {0.f, 0.f, 0.f, 0.f};
        xv[0] = i0 > j ? -c0 * dg[i0] : (i0 == j ? dg[j] : 0.f);
        if (i0 + 1 < N) {
          c1 = fmaf(L1[i0], xv[0], c1);
          xv[1] = i0 + 1 > j ? -c1 * dg[i0 + 1] : (i0 + 1 == j ? dg[j] : 0.f);
          if (i0 + 2 < N) {
            c2 = fmaf(L2[i0 + 1], xv[1], fmaf(L2[i0], xv[0], c2));
            xv[2] = i0 + 2 > j ? -c2 * dg[i0 + 2] : (i0 + 2 == j ? dg[j] : 0.f);
            if (i0 + 3 < N) {
              c3 = fmaf(L3[i0 + 2], xv[2], fmaf(L3[i0 + 1], xv[1], fmaf(L3[i0], xv[0], c3)));
              xv[3] = i0 + 3 > j ? -c3 * dg[i0 + 3] : (i0 + 3 == j ? dg[j] : 0.f);
            }
          }
        }
        *reinterpret_cast<float4*>(xc + i0) = make_float4(xv[0], xv[1], xv[2], xv[3]);
      }
      __syncwarp();
      // blocked output: column j, blocks R >= j / 8 (rows above the diagonal, beyond N, or above this group's
      // first row read as zero)
      if (j < 8 * nR) {
        for (int R = j >> 3; R < nR; ++R) {
          const float4 u0 = *reinterpret_cast<const float4*>(xc + 8 * R);
          const float4 u1 = *reinterpret_cast<const float4*>(xc + 8 * R + 4);
          const float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
          float v[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int i = 8 * R + r;
            v[r] = (j < N && i < N && i >= j) ? u[r] : 0.f;
          }
          float4* dst = reinterpret_cast<float4*>(Iout + linv_block_off(R) + (int64_t)j * 8);
          dst[0] = make_float4(v[0], v[1], v[2], v[3]);
          dst[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
      }
      // tensor-core image: quads of this group's columns, all Np rows (FP32; the query splits it into TF32
      // hi and lo parts in shared memory)
      if (N <= kTcMaxN) {
        const int np16 = tc_np(N);
        const int q1 = min(base + 32, tc_kp(N)) >> 2;
        float* img = a.ltc + a.ltc_off[g];
        for (int q = base >> 2; q < q1; ++q) {
          for (int i = lane; i < np16; i += 32) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int col = 4 * q + u;
              v[u] = (col <= i && i < N) ? Xt[(col - base) * xs + i] : 0.f;
            }
            const int64_t o = ((int64_t)q * np16 + i) * 4;
            *reinterpret_cast<float4*>(img + o) = make_float4(v[0], v[1], v[2], v[3]);
          }
        }
      }
      __syncwarp();
    }
    __syncthreads();  // L and dg are reused by the next cell
  }
}

template <int TEAM, bool INPLACE, bool GMAT>
__global__ void __launch_bounds__(TEAM) k_linv(LinvArgs a) {
  extern __shared__ __align__(16) float smf[];
  __shared__ int s_cell;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = a.np;
  float* ws = GMAT ? a.gscr + (int64_t)blockIdx.x * a.gstride : smf;
  float* dg = ws;
  float* L = ws + ((np + 3) & ~3);
  for (;;) {
    if (tid == 0) {
      const int w = atomicAdd(a.counter, 1);
      s_cell = w < a.count ? (int)a.order[a.first + w] : -1;
    }
    fit_sync(TEAM);
    const int g = s_cell;
    if (g < 0) break;
    const int N = a.n32[g];
    if (N == 0 || a.status[g] != KSDF_CELL_OK) {
      fit_sync(TEAM);
      continue;
    }
    const int64_t T = tri_sz(N);
    const double* Ld = a.chol64 + a.chol_off[g];
    for (int64_t e0 = tid; e0 < T; e0 += 8 * (int64_t)TEAM) {  // eight loads in flight per thread
      double v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t e = e0 + (int64_t)r * TEAM;
        v[r] = e < T ? Ld[e] : 0.0;
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t e = e0 + (int64_t)r * TEAM;
        if (e < T) L[e] = d2f_bits(v[r]);
      }
    }
    fit_sync(TEAM);
    for (int j = tid; j < N; j += TEAM) dg[j] = 1.f / L[tri_sz(j) + j];
    fit_sync(TEAM);
    float* Iout = a.linv32 + a.linv_off[g];
    const int nR = (N + 7) >> 3;
    for (int gi = INPLACE ? 0 : warp; 32 * gi < N; gi += INPLACE ? 1 : TEAM / 32) {
      const int base = 32 * gi, j = base + lane;
      // X[k][j] lives at xs[k * ldx] (in place: L's packed row k; else the group's buffer)
      float* xcol = INPLACE ? L + j : ws + linv_group_off(np, gi) - (int64_t)base * 32 + lane;
      for (int i0 = base; i0 < N; i0 += 4) {
        const float* L0 = L + tri_sz(i0);
        const float* L1 = L + tri_sz(min(i0 + 1, N - 1));
        const float* L2 = L + tri_sz(min(i0 + 2, N - 1));
        const float* L3 = L + tri_sz(min(i0 + 3, N - 1));
        float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
#pragma unroll 4
        for (int k = base; k < i0; ++k) {
          float x;
          if (INPLACE) x = k >= j ? xcol[tri_sz(k)] : 0.f;  // X[k][j], zero above the diagonal
          else x = xcol[(int64_t)k * 32];
          c0 = fmaf(L0[k], x, c0);
          c1 = fmaf(L1[k], x, c1);
          c2 = fmaf(L2[k], x, c2);
          c3 = fmaf(L3[k], x, c3);
        }
        float xv[4];
        xv[0] = i0 > j ? -c0 * dg[i0] : (i0 == j ? dg[j] : 0.f);
        if (i0 + 1 < N) {
          c1 = fmaf(L1[i0], xv[0], c1);
          xv[1] = i0 + 1 > j ? -c1 * dg[i0 + 1] : (i0 + 1 == j ? dg[j] : 0.f);
          if (i0 + 2 < N) {
            c2 = fmaf(L2[i0 + 1], xv[1], fmaf(L2[i0], xv[0], c2));
            xv[2] = i0 + 2 > j ? -c2 * dg[i0 + 2] : (i0 + 2 == j ? dg[j] : 0.f);
            if (i0 + 3 < N) {
              c3 = fmaf(L3[i0 + 2], xv[2], fmaf(L3[i0 + 1], xv[1], fmaf(L3[i0], xv[0], c3)));
              xv[3] = i0 + 3 > j ? -c3 * dg[i0 + 3] : (i0 + 3 == j ? dg[j] : 0.f);
            }
          }
        }
        // rows i0.. are finished: store (in place: only on or below the diagonal and inside the matrix)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int i = i0 + r;
          if (i < N) {
            if (INPLACE) {
              if (j <= i) xcol[tri_sz(i)] = xv[r];
            } else {
              xcol[(int64_t)i * 32] = xv[r];
            }
          }
        }
        if (INPLACE) __syncwarp();  // rows of L read by other lanes' columns are overwritten in place
      }
      // blocked output of the group's columns (columns N .. 8 nR - 1 of the last block are zero)
      if (j < 8 * nR) {
        for (int R = j >> 3; R < nR; ++R) {
          float v[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int i = 8 * R + r;
            v[r] = (j < N && i < N && i >= j) ? (INPLACE ? xcol[tri_sz(i)] : xcol[(int64_t)i * 32]) : 0.f;
          }
          float4* dst = reinterpret_cast<float4*>(Iout + linv_block_off(R) + (int64_t)j * 8);
          dst[0] = make_float4(v[0], v[1], v[2], v[3]);
          dst[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
      }
      // the tensor-core image (column j of L^-1 is K index j of the B operand): all Np rows, zero padded, FP32
      if (N <= kTcMaxN && j < tc_kp(N)) {
        const int np16 = tc_np(N);
        float* col = a.ltc + a.ltc_off[g] + (int64_t)(j >> 2) * np16 * 4 + (j & 3);
        for (int i = 0; i < np16; ++i)
          col[(int64_t)i * 4] =
              (j < N && i < N && i >= j) ? (INPLACE ? xcol[tri_sz(i)] : xcol[(int64_t)i * 32]) : 0.f;
      }
      if (INPLACE) __syncwarp();
    }
    fit_sync(TEAM);
  }
}

}  // namespace

static int bits_for(uint64_t v) {
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

// persistent launches of one size class: as many teams as fit on the GPU (at most one per cell)
template <class K, class Args, class... Extra>
static cudaError_t launch_persistent(ksdf_ctx* c, K kern, int team, const Args& f, size_t smem, bool gslot,
                                     cudaStream_t s, const Extra&... extra) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, team, smem);
  if (e != cudaSuccess) return e;
  int64_t nblk = std::min<int64_t>(f.count, (int64_t)std::max(1, occ) * c->num_sms);
  if (gslot) nblk = std::min<int64_t>(nblk, c->num_sms);  // one global slot per CTA
  launch(kern, (unsigned)nblk, team, smem, s, f, extra...);
  return cudaSuccess;
}

__global__ void k_device_math(int fn, const double* x, int64_t n, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  double r = __longlong_as_double(0x7ff8000000000000ll);
  if (fn == 0 && v >= 0.0 && v < 0x1p22) r = exp2_neg_q16(v);
  if (fn == 1 && v >= 0.0 && v < 0x1p22) r = exp2_neg_fixed40((unsigned long long)(v * 0x1p40));
  if (fn == 2 && pivot_ok(v)) r = rsqrt_pivot(v);
  y[i] = r;
}

// brick of an OK cell (index (bz nby + by) nbx + bx over the cell bounding box); -1 for other cells
__device__ __forceinline__ int64_t cell_brick(uint64_t key, int lx, int ly, int lz, int nbx, int nby) {
  int cx, cy, cz;
  unpack_key(key, cx, cy, cz);
  return ((int64_t)((cz - lz) >> kBrickShift) * nby + ((cy - ly) >> kBrickShift)) * nbx + ((cx - lx) >> kBrickShift);
}

// per-brick counts of OK cells, and each cell's rank within its brick
__global__ void k_brick_count(const uint64_t* cell_key, const int32_t* status, int64_t G, int lx, int ly, int lz,
                              int nbx, int nby, int64_t* bcnt, int32_t* rank) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  if (status[g] != KSDF_CELL_OK) {
    rank[g] = -1;
    return;
  }
  const int64_t b = cell_brick(cell_key[g], lx, ly, lz, nbx, nby);
  rank[g] = (int32_t)atomicAdd((unsigned long long*)&bcnt[b], 1ull);
}

__global__ void k_brick_fill(const uint64_t* cell_key, const int32_t* rank, int64_t G, int lx, int ly, int lz,
                             int nbx, int nby, const int64_t* boff, int32_t* cells) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G || rank[g] < 0) return;
  cells[boff[cell_brick(cell_key[g], lx, ly, lz, nbx, nby)] + rank[g]] = (int32_t)g;
}

ksdf_status fit_model(ksdf_ctx* c, const double* x, const float* var, const float* nrm, int64_t S, const Model* prev,
                      int64_t* n_refit) {
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
  KSDF_CUDA(c, ensure(m.ltc_off, sizeof(int64_t) * (G + 1)));
  KSDF_CUDA(c, ensure(c->ws[WS_D], sizeof(int64_t) * (4 * G + 4)));
  int64_t* n64 = ptr<int64_t>(c->ws[WS_D]);
  int64_t* tri64 = n64 + (G + 1);
  int64_t* lb64 = tri64 + (G + 1);
  int64_t* tc64 = lb64 + (G + 1);
  int* dmax = bbox + 6;
  KSDF_CUDA(c, cudaMemsetAsync(dmax, 0, sizeof(int) * 2, st));
  launch(k_assemble, (unsigned)G, kAssembleThreads, 0, st, ptr<uint64_t>(m.key), G, own_off, vals, x, p, R, ptr<uint64_t>(m.hkeys),
         ptr<int32_t>(m.hvals), cap, ptr<int32_t>(m.mpad), n64, ptr<int32_t>(m.status), dmax, stw);
  // refit scheduling: carried counters; with a budget, the changed cells beyond it keep their previous training
  // set (and, below, their previous fit)
  KSDF_CUDA(c, ensure(m.qc0, sizeof(int32_t) * (G + 1)));
  KSDF_CUDA(c, ensure(m.qc2, sizeof(int32_t) * (G + 1)));
  KSDF_CUDA(c, ensure(m.refit, sizeof(int32_t) * (G + 1)));
  if (!prev) {
    KSDF_CUDA(c, cudaMemsetAsync(m.qc0.p, 0, sizeof(int32_t) * G, st));
    KSDF_CUDA(c, cudaMemsetAsync(m.qc2.p, 0, sizeof(int32_t) * G, st));
  } else {
    Model& o = const_cast<Model&>(*prev);
    KSDF_CUDA(c, ensure(c->ws[WS_SCHED], (sizeof(uint64_t) + 4 * sizeof(int32_t)) * (size_t)(G + 1)));
    uint64_t* skey = ptr<uint64_t>(c->ws[WS_SCHED]);
    uint32_t* sval = reinterpret_cast<uint32_t*>(skey + (G + 1));
    int32_t* chg = reinterpret_cast<int32_t*>(sval + (G + 1));
    int32_t* soid = chg + (G + 1);
    int32_t* sel = soid + (G + 1);
    launch(k_sched_score, ceil_div(G * 32, 256), 256, 0, st, ptr<uint64_t>(m.key), n64, ptr<int32_t>(m.mpad), G,
           p.n_max, ptr<uint64_t>(o.hkeys), ptr<int32_t>(o.hvals), o.hcap, ptr<int32_t>(o.n), ptr<int64_t>(o.ts_off),
           ptr<int32_t>(o.mgid), ptr<int32_t>(o.status), ptr<int32_t>(o.qc0), ptr<int32_t>(o.qc2), c->sched_eta,
           ptr<int32_t>(m.qc0), ptr<int32_t>(m.qc2), soid, chg, skey, sval);
    if (c->sched_max > 0) {
      KSDF_CUDA(c, radix_sort_u64(skey, sval, G, 41, c->ws[WS_SORT], st));
      launch(k_sched_select, ceil_div(G, 256), 256, 0, st, skey, sval, G, c->sched_max, sel);
      launch(k_sched_defer, ceil_div(G * 32, 256), 256, 0, st, chg, sel, soid, G, p.n_max, ptr<int32_t>(o.n),
             ptr<int64_t>(o.ts_off), ptr<int32_t>(o.mgid), ptr<int32_t>(m.mpad), n64, dmax);
    }
  }
  launch(k_sizes, ceil_div(G, 256), 256, 0, st, n64, G, tri64, lb64, tc64, ptr<int32_t>(m.n));
  KSDF_CUDA(c, scan_i64(n64, ptr<int64_t>(m.ts_off), G, dtot, c->ws[WS_SCAN], st));
  KSDF_CUDA(c, scan_i64(tri64, ptr<int64_t>(m.chol_off), G, dtot + 1, c->ws[WS_SCAN], st));
  KSDF_CUDA(c, scan_i64(lb64, ptr<int64_t>(m.linv_off), G, dtot + 2, c->ws[WS_SCAN], st));
  KSDF_CUDA(c, scan_i64(tc64, ptr<int64_t>(m.ltc_off), G, dtot + 3, c->ws[WS_SCAN], st));
  int64_t tots[4];
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
  m.ltc_total = tots[3];
  m.max_n = hmax[0];
  KSDF_CUDA(c, cudaMemcpyAsync(ptr<int64_t>(m.ts_off) + G, &tots[0], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  KSDF_CUDA(c, cudaMemcpyAsync(ptr<int64_t>(m.chol_off) + G, &tots[1], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  KSDF_CUDA(c, cudaMemcpyAsync(ptr<int64_t>(m.linv_off) + G, &tots[2], sizeof(int64_t), cudaMemcpyHostToDevice, st));
  KSDF_CUDA(c, cudaMemcpyAsync(ptr<int64_t>(m.ltc_off) + G, &tots[3], sizeof(int64_t), cudaMemcpyHostToDevice, st));
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
  KSDF_CUDA(c, ensure(m.ltc, sizeof(float) * (m.ltc_total + 4)));
  launch(k_gather_members, ceil_div(G * p.n_max, 256), 256, 0, st, ptr<uint64_t>(m.key), ptr<int32_t>(m.n),
         ptr<int64_t>(m.ts_off), ptr<int32_t>(m.mpad), G, p, x, var, nrm, ptr<int32_t>(m.mgid), ptr<D4>(m.md4),
         ptr<float4>(m.mf4), ptr<float>(m.mvar), nrm ? ptr<float4>(m.mnrm) : nullptr);
  // 5. the fit, largest cells first, three size classes on three streams
  KSDF_CUDA(c, ensure(c->ws[WS_A], sizeof(uint64_t) * (G + 1)));
  KSDF_CUDA(c, ensure(m.cell_order, sizeof(uint32_t) * (G + 1)));
  uint64_t* okeys = ptr<uint64_t>(c->ws[WS_A]);
  uint32_t* order = ptr<uint32_t>(m.cell_order);
  // update: which cells need a fit (training set changed), the others copy the previous model's later
  int32_t* touched = nullptr;
  int32_t* oid = nullptr;
  if (prev) {
    KSDF_CUDA(c, ensure(c->ws[WS_TOUCH], sizeof(int32_t) * 2 * (G + 1)));
    touched = ptr<int32_t>(c->ws[WS_TOUCH]);
    oid = touched + (G + 1);
    Model& o = const_cast<Model&>(*prev);
    launch(k_touched, ceil_div(G * 32, 256), 256, 0, st, ptr<uint64_t>(m.key), ptr<int32_t>(m.n),
           ptr<int64_t>(m.ts_off), ptr<int32_t>(m.mgid), G, ptr<uint64_t>(o.hkeys), ptr<int32_t>(o.hvals), o.hcap,
           ptr<int32_t>(o.n), ptr<int64_t>(o.ts_off), ptr<int32_t>(o.mgid), ptr<int32_t>(o.status), touched, oid);
  }
  launch(k_order_keys, ceil_div(G, 256), 256, 0, st, ptr<int32_t>(m.n), touched, G, p.n_max, okeys, order);
  KSDF_CUDA(c, radix_sort_u64(okeys, order, G, bits_for((uint64_t)p.n_max + 1), c->ws[WS_SORT], st));
  // size classes (host histogram of the cells to fit), launched concurrently, largest first; each class has
  // its team size
  std::vector<int32_t> hn((size_t)G), ht;
  KSDF_CUDA(c, cudaMemcpyAsync(hn.data(), m.n.p, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, st));
  if (prev) {
    ht.resize((size_t)G);
    KSDF_CUDA(c, cudaMemcpyAsync(ht.data(), touched, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, st));
  }
  KSDF_CUDA(c, cudaStreamSynchronize(st));
  int64_t nfit = 0;
  for (int64_t g = 0; g < G; ++g) {
    if (prev && !ht[(size_t)g]) hn[(size_t)g] = -1;  // not fitted: out of every class
    else ++nfit;
  }
  if (n_refit) *n_refit = nfit;
  using FitClass = FitClassCfg;
  const std::vector<FitClassCfg>& cls = c->fit_cls.empty() ? fit_table(0) : c->fit_cls;
  const int kNumClass = (int)cls.size();
  std::vector<int64_t> cnt((size_t)kNumClass, 0);
  for (int32_t v : hn) {
    if (v < 0) continue;
    int cl = kNumClass - 1;
    while (cl > 0 && v > cls[cl].np) --cl;
    ++cnt[cl];
  }
  KSDF_CUDA(c, cudaMemsetAsync(dmax, 0, sizeof(int) * 2, st));
  KSDF_CUDA(c, ensure(c->ws[WS_E], sizeof(int64_t) * 4 + sizeof(int) * 32));  // counters: fit and L^-1 classes
  int* ctr = reinterpret_cast<int*>(ptr<int64_t>(c->ws[WS_E]) + 4);
  KSDF_CUDA(c, cudaMemsetAsync(ctr, 0, sizeof(int) * 32, st));
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
  // kernel matrices of the cells to fit (largest first), into the factor's place
  e0 = prof_begin(c);
  if (nfit > 0) {
    KmatArgs ka;
    ka.order = order;
    ka.first = 0;
    ka.count = nfit;
    ka.counter = ctr + 24;
    ka.n32 = ptr<int32_t>(m.n);
    ka.ts_off = ptr<int64_t>(m.ts_off);
    ka.chol_off = ptr<int64_t>(m.chol_off);
    ka.md4 = ptr<D4>(m.md4);
    ka.mf4 = ptr<float4>(m.mf4);
    ka.mvar = ptr<float>(m.mvar);
    ka.chol64 = ptr<double>(m.chol64);
    ka.np = std::max(m.max_n, 1);
    const bool matern = p.kernel == KSDF_KERNEL_MATERN32;
    ka.sc = matern ? p.lambda * kExpQ16PerNat : std::sqrt(p.lambda * kExpQ16PerNat);
    ka.lamf = (float)p.lambda;
    // members lie within the margin of their cell: |local coordinate| <= h + mu
    ka.fixed = !matern && ka.sc * (p.h + p.mu) < 0x1p21;
    const size_t ksm = sizeof(double) * (size_t)kmat_warp_doubles(ka.np) * kKmatWarps;
    auto kern = matern ? k_kmat<true> : k_kmat<false>;
    KSDF_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ksm));
    int occ = 0;
    KSDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * kKmatWarps, ksm));
    const int64_t nblk = std::min<int64_t>(ceil_div(nfit, kKmatWarps), (int64_t)std::max(1, occ) * c->num_sms);
    launch(kern, (unsigned)nblk, 32 * kKmatWarps, ksm, st, ka);
  }
  prof_end(c, e0, "fit.kmat");
  e0 = prof_begin(c);
  KSDF_CUDA(c, fork_streams(c));
  int64_t first = 0;
  int launched = 0;
  for (int cl = 0; cl < kNumClass; ++cl) {
    if (cnt[cl] == 0) continue;
    FitArgs f = fa;
    f.first = first;
    f.count = cnt[cl];
    f.counter = ctr + cl;
    first += cnt[cl];
    const int team = cls[cl].team;
    f.np = cls[cl].gmat ? std::max(m.max_n, 1) : cls[cl].np;
    const size_t smem = sizeof(double) * (size_t)(fit_smem_doubles(f.np, !cls[cl].gmat) +
                                                  (cls[cl].gmat ? (int64_t)(f.np + 1) * kB : 0));
    const int si = launched % ksdf_ctx::kNumAux;  // auxiliary streams only: the main stream marks the stage end
    cudaStream_t s = c->aux[si];
    ++launched;
    if (cls[cl].gmat) {
      f.gstride = tri_sz(f.np + 1);
      const int64_t slots = std::min<int64_t>(cnt[cl], c->num_sms);
      KSDF_CUDA(c, ensure(c->ws[WS_FITSCR], sizeof(double) * (size_t)(f.gstride * slots + 1)));
      f.gscr = ptr<double>(c->ws[WS_FITSCR]);
    }
    cudaError_t le = cudaSuccess;
    switch (team) {
      case 256: le = cls[cl].gmat ? launch_persistent(c, k_fit<256, true>, 256, f, smem, true, s, p)
                                  : launch_persistent(c, k_fit<256, false>, 256, f, smem, false, s, p); break;
      case 128: le = launch_persistent(c, k_fit<128, false>, 128, f, smem, false, s, p); break;
      case 64: le = launch_persistent(c, k_fit<64, false>, 64, f, smem, false, s, p); break;
      default: le = launch_persistent(c, k_fit<32, false>, 32, f, smem, false, s, p); break;
    }
    KSDF_CUDA(c, le);
    KSDF_CUDA(c, cudaEventRecord(c->ev_mid[si], s));
    // L^{-1} in FP32 of the same cells, behind their factorisation, on a high-priority stream: its blocks take
    // the SM resources this class's factorisation frees ahead of the pending blocks of the other classes'
    // factorisations, so that its FP32 work overlaps their FP64 work instead of trailing it
    {
      const cudaStream_t sh = c->aux_hi[si];
      KSDF_CUDA(c, cudaStreamWaitEvent(sh, c->ev_mid[si], 0));
      LinvArgs la;
      la.order = order;
      la.first = f.first;
      la.count = f.count;
      la.counter = ctr + 16 + cl;
      la.n32 = ptr<int32_t>(m.n);
      la.status = ptr<int32_t>(m.status);
      la.chol_off = ptr<int64_t>(m.chol_off);
      la.linv_off = ptr<int64_t>(m.linv_off);
      la.chol64 = ptr<double>(m.chol64);
      la.linv32 = ptr<float>(m.linv32);
      la.ltc_off = ptr<int64_t>(m.ltc_off);
      la.ltc = ptr<float>(m.ltc);
      la.gscr = nullptr;
      la.gstride = 0;
      la.np = f.np;
      if (f.np <= 96) {
        le = launch_persistent(c, k_linv_small<1>, 32, la, sizeof(float) * (size_t)linv_small_floats(f.np, 1), false,
                               sh);
      } else if (f.np <= kTcMaxN) {
        le = launch_persistent(c, k_linv_small<2>, 64, la, sizeof(float) * (size_t)linv_small_floats(f.np, 2), false,
                               sh);
      } else {
        la.gstride = (linv_slot_floats(f.np, false) + 3) & ~3LL;
        const int64_t slots = std::min<int64_t>(f.count, c->num_sms);
        KSDF_CUDA(c, ensure(c->ws[WS_LINVSCR], sizeof(float) * (size_t)(la.gstride * slots + 4)));
        la.gscr = ptr<float>(c->ws[WS_LINVSCR]);
        le = launch_persistent(c, k_linv<512, false, true>, 512, la, 0, true, sh);
      }
      KSDF_CUDA(c, le);
    }
  }
  // the factorisations are done when every class stream has passed its k_fit
  for (int i = 0; i < std::min(launched, ksdf_ctx::kNumAux); ++i) KSDF_CUDA(c, cudaStreamWaitEvent(st, c->ev_mid[i], 0));
  KSDF_CUDA(c, cudaGetLastError());
  prof_end(c, e0, "fit.cholesky");
  // the rest of the L^{-1} kernels
  e0 = prof_begin(c);
  KSDF_CUDA(c, join_streams(c));
  prof_end(c, e0, "fit.linv");
  if (prev && nfit < G) {
    Model& o = const_cast<Model&>(*prev);
    CopyFitArgs ca;
    ca.touched = touched;
    ca.oid = oid;
    ca.n32 = ptr<int32_t>(m.n);
    ca.G = G;
    ca.ts_off = ptr<int64_t>(m.ts_off);
    ca.chol_off = ptr<int64_t>(m.chol_off);
    ca.linv_off = ptr<int64_t>(m.linv_off);
    ca.ltc_off = ptr<int64_t>(m.ltc_off);
    ca.ots_off = ptr<int64_t>(o.ts_off);
    ca.ochol_off = ptr<int64_t>(o.chol_off);
    ca.olinv_off = ptr<int64_t>(o.linv_off);
    ca.oltc_off = ptr<int64_t>(o.ltc_off);
    ca.ochol64 = ptr<double>(o.chol64);
    ca.olinv32 = ptr<float>(o.linv32);
    ca.oltc = ptr<float>(o.ltc);
    ca.omd4 = ptr<D4>(o.md4);
    ca.chol64 = ptr<double>(m.chol64);
    ca.linv32 = ptr<float>(m.linv32);
    ca.ltc = ptr<float>(m.ltc);
    ca.md4 = ptr<D4>(m.md4);
    ca.mf4 = ptr<float4>(m.mf4);
    ca.status = ptr<int32_t>(m.status);
    launch(k_copy_fit, (unsigned)std::min<int64_t>(G, 8 * c->num_sms), 256, 0, st, ca);
  }
  launch(k_sched_after, ceil_div(G, 256), 256, 0, st, (const int32_t*)touched, G, ptr<int32_t>(m.qc0),
         ptr<int32_t>(m.qc2), ptr<int32_t>(m.refit));
  // bricks over the cell bounding box for the candidate search (OK cells only; statuses are final here)
  {
    int64_t nbk[3];
    for (int j = 0; j < 3; ++j) {
      nbk[j] = (((int64_t)hb[3 + j] - hb[j]) >> kBrickShift) + 1;
      m.bk_lo[j] = hb[j];
    }
    const int64_t nb = nbk[0] * nbk[1] * nbk[2];
    m.nbricks = 0;
    if (nb <= 4 * G + 4096) {
      for (int j = 0; j < 3; ++j) m.bk_n[j] = (int)nbk[j];
      m.nbricks = nb;
      KSDF_CUDA(c, ensure(m.bk_off, sizeof(int64_t) * (nb + 1)));
      KSDF_CUDA(c, ensure(m.bk_cells, sizeof(int32_t) * G));
      KSDF_CUDA(c, ensure(c->ws[WS_BRICK], sizeof(int32_t) * G));
      int64_t* boff = ptr<int64_t>(m.bk_off);
      int32_t* rank = ptr<int32_t>(c->ws[WS_BRICK]);
      KSDF_CUDA(c, cudaMemsetAsync(boff, 0, sizeof(int64_t) * (nb + 1), st));
      launch(k_brick_count, ceil_div(G, 256), 256, 0, st, ptr<uint64_t>(m.key), ptr<int32_t>(m.status), G, hb[0],
             hb[1], hb[2], m.bk_n[0], m.bk_n[1], boff, rank);
      KSDF_CUDA(c, scan_i64(boff, boff, nb, boff + nb, c->ws[WS_SCAN], st));
      launch(k_brick_fill, ceil_div(G, 256), 256, 0, st, ptr<uint64_t>(m.key), rank, G, hb[0], hb[1], hb[2],
             m.bk_n[0], m.bk_n[1], boff, ptr<int32_t>(m.bk_cells));
    }
  }
  KSDF_CUDA(c, cudaMemcpyAsync(hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, st));
  KSDF_CUDA(c, cudaStreamSynchronize(st));
  m.n_not_pd = hmax[1];
  // keep the samples: positions for the adjoint's per-cell recomputation; all three for later updates
  m.S = S;
  KSDF_CUDA(c, ensure(m.x, sizeof(double) * S * p.dim));
  KSDF_CUDA(c, cudaMemcpyAsync(m.x.p, x, sizeof(double) * S * p.dim, cudaMemcpyDeviceToDevice, st));
  KSDF_CUDA(c, ensure(m.var_all, sizeof(float) * S));
  if (var) KSDF_CUDA(c, cudaMemcpyAsync(m.var_all.p, var, sizeof(float) * S, cudaMemcpyDeviceToDevice, st));
  else KSDF_CUDA(c, cudaMemsetAsync(m.var_all.p, 0, sizeof(float) * S, st));
  if (nrm) {
    KSDF_CUDA(c, ensure(m.nrm_all, sizeof(float) * S * p.dim));
    KSDF_CUDA(c, cudaMemcpyAsync(m.nrm_all.p, nrm, sizeof(float) * S * p.dim, cudaMemcpyDeviceToDevice, st));
  }
  prof_end(c, e_fit, "fit");
  c->fitted = true;
  if (m.n_not_pd > 0)
    return set_err(c, KSDF_ERR_NOT_PD, "ksdf_fit: %d cell(s) not positive definite in FP64 (excluded)", m.n_not_pd);
  return KSDF_OK;
}

// candidate size-class tables of the fit (largest class first; the first entry keeps its matrices in a
// global slot).  Table 0 is the default; ksdf_autotune times them all on the model's own cells.  The result
// of a fit does not depend on the table (each cell's arithmetic is the same whatever the team size).
ksdf_status device_math(ksdf_ctx* c, int fn, const double* x, int64_t n, double* y) {
  if (n > 0) launch(k_device_math, ceil_div(n, 256), 256, 0, c->stream, fn, x, n, y);
  KSDF_CUDA(c, cudaGetLastError());
  return KSDF_OK;
}

static const std::vector<std::vector<FitClassCfg>> kFitTables = {
    // one warp up to 80, two up to 96, four up to 156, eight up to 218
    {{kMaxNmax, 256, true}, {218, 256, false}, {156, 128, false}, {128, 128, false}, {96, 64, false},
     {80, 32, false}, {64, 32, false}},
    // one warp up to 96, two up to 128
    {{kMaxNmax, 256, true}, {218, 256, false}, {156, 128, false}, {128, 64, false}, {96, 32, false},
     {80, 32, false}, {64, 32, false}},
    // one warp up to 64, two up to 128
    {{kMaxNmax, 256, true}, {218, 256, false}, {156, 128, false}, {128, 64, false}, {96, 64, false},
     {80, 64, false}, {64, 32, false}, {48, 32, false}},
    // one warp up to 80, two up to 128, four up to 218
    {{kMaxNmax, 256, true}, {218, 128, false}, {156, 128, false}, {128, 64, false}, {96, 64, false},
     {80, 32, false}, {64, 32, false}},
    // one warp up to 64, two up to 112, four up to 180, finer classes
    {{kMaxNmax, 256, true}, {218, 256, false}, {180, 128, false}, {140, 128, false}, {112, 64, false},
     {96, 64, false}, {80, 64, false}, {64, 32, false}},
    // one warp up to 72, two up to 156, four up to 218
    {{kMaxNmax, 256, true}, {218, 128, false}, {156, 64, false}, {128, 64, false}, {96, 64, false},
     {72, 32, false}, {56, 32, false}, {40, 32, false}},
};

int fit_table_count() { return (int)kFitTables.size(); }
const std::vector<FitClassCfg>& fit_table(int i) { return kFitTables[(size_t)i]; }

// time every candidate table on the fitted model (each fit run twice, the second timed with CUDA events on
// the context stream), keep the fastest in the context, and refit with it; the model is unchanged
ksdf_status autotune_fit(ksdf_ctx* c, int* chosen, double* ms) {
  if (!c->fitted) return set_err(c, KSDF_ERR_NOT_FITTED, "ksdf_autotune: no model (call ksdf_fit first)");
  Model& m = c->m;
  const int dim = c->p.dim;
  const int64_t S = m.S;
  cudaStream_t st = c->stream;
  KSDF_CUDA(c, ensure(c->ws[WS_UX], sizeof(double) * S * dim));
  KSDF_CUDA(c, ensure(c->ws[WS_UV], sizeof(float) * S));
  double* ux = ptr<double>(c->ws[WS_UX]);
  float* uv = ptr<float>(c->ws[WS_UV]);
  float* un = nullptr;
  KSDF_CUDA(c, cudaMemcpyAsync(ux, m.x.p, sizeof(double) * S * dim, cudaMemcpyDeviceToDevice, st));
  KSDF_CUDA(c, cudaMemcpyAsync(uv, m.var_all.p, sizeof(float) * S, cudaMemcpyDeviceToDevice, st));
  if (m.has_normals) {
    KSDF_CUDA(c, ensure(c->ws[WS_UN], sizeof(float) * S * dim));
    un = ptr<float>(c->ws[WS_UN]);
    KSDF_CUDA(c, cudaMemcpyAsync(un, m.nrm_all.p, sizeof(float) * S * dim, cudaMemcpyDeviceToDevice, st));
  }
  const bool prof = c->prof;
  c->prof = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KSDF_CUDA(c, cudaEventCreate(&e0));
  KSDF_CUDA(c, cudaEventCreate(&e1));
  int best = 0;
  double best_ms = 1e300;
  ksdf_status rs = KSDF_OK;
  for (int t = 0; t < fit_table_count() && rs == KSDF_OK; ++t) {
    c->fit_cls = fit_table(t);
    float tms = 0.f;
    for (int rep = 0; rep < 2 && rs == KSDF_OK; ++rep) {
      cudaEventRecord(e0, st);
      rs = fit_model(c, ux, uv, un, S);
      cudaEventRecord(e1, st);
      if (rs == KSDF_ERR_NOT_PD) rs = KSDF_OK;
    }
    if (rs != KSDF_OK) break;
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&tms, e0, e1);
    if (ms) ms[t] = tms;
    if (tms < best_ms) {
      best_ms = tms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->prof = prof;
  if (rs != KSDF_OK) return rs;
  c->fit_cls = fit_table(best);
  if (chosen) *chosen = best;
  rs = fit_model(c, ux, uv, un, S);
  return rs == KSDF_ERR_NOT_PD ? KSDF_OK : rs;
}

namespace {
__global__ void k_bin_keys(const double* x, int64_t n, Params p, uint64_t* keys, uint32_t* st) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3] = {0, 0, 0};
  bool ok = true;
  for (int j = 0; j < p.dim; ++j) ok &= bin_coord(x[i * p.dim + j], p.o[j], p.h, p.rh, c[j]);
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
