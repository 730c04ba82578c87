// ksdf_bhm.cu -- the Bayesian Hilbert map front-end of Kernel-SDF (Sec. IV-A, App. A, App. B) on one GPU: a device
// hash table of hinge blocks, the samples of each ray, the diagonal-covariance variational EM, the online threshold,
// prediction (log-odds, sign, gradient, probit occupancy) and the surface points of the marked marching cells.
// C ABI in include/ksdf_bhm.h, which also states the definitions every kernel here follows.
//
// Data layout in HBM (one map):
//   W[slot * NW + i]  float4 {mu, P, B, A} per weight (NW = n_h^3 + 1, the bias last): mean and precision of the map
//                     before the running update, and the update's two accumulators -- B = sum (t - 1/2) phi and
//                     A = sum c(xi) phi^2 of odd EM rounds; PB[slot * NW + i] holds A of even rounds
//   hash table        block key -> slot (open addressing, linear probing), 4x the block capacity
//   per block         packed key, active flag, the frame stamps of the touched / marked lists, its marked-cell index
//   masks             one bit per marching cell of each marked block ((n_h m)^3 bits)
// Every EM round is one launch over the rays (one thread per ray walks its samples; blocks without a hit are
// skipped a whole block at a time), so no sample is ever stored.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <string>

#include "ksdf_internal.cuh"
#include "../../include/ksdf_bhm.h"

namespace ksdf {
namespace {

constexpr int kQ = 20;                   // fixed-point bits of a lattice fraction
constexpr double kLatMax = 65000.0;      // |u| bound (marching nodes stay within the 20-bit edge-key fields)
constexpr int64_t kEdgeBias = 1LL << 19;
constexpr int kT = 256;
constexpr int kGridStride = 152 * 4;     // CTAs of the grid-stride kernels: four per SM

struct BhmState {
  int32_t n_blocks, n_new, n_touched, n_marked;
  int32_t n_out, pad0, pad1, pad2;
  unsigned long long n_samples;
  double lsum;
  double tau;
  uint32_t status;
  uint32_t pad3;
};

struct BhmDev {
  double o[3], h, p[3], up[3];
  double fstep, fgap;
  double tau_a, tau_b;      // tau <- tau_a tau + tau_b sum_k l(x_k)
  double inv_m;             // 1 / march_sub (exact: a power of two)
  float gh2, g2h;           // gamma h^2 and -2 gamma h (binary32)
  float prior_prec, xi0, beta;
  long long r2q;
  int nh, nw, msub, cdim, mask_words;
  int frame, max_blocks, max_marked;
  int bias;
  uint64_t hcap;
  uint64_t* hkeys;
  int32_t* hvals;
  uint64_t* bkey;
  uint8_t* active;
  int32_t *stamp_touch, *stamp_mark, *mark_idx;
  int32_t *new_list, *touched, *marked;
  float4* W;
  float* PB;
  uint32_t* masks;
  BhmState* st;
};

__device__ __forceinline__ double lat(double x, double o, double h) { return __ddiv_rn(__dsub_rn(x, o), h); }
__device__ __forceinline__ bool lat_ok(double u) { return u > -kLatMax && u < kLatMax; }
__host__ __device__ __forceinline__ int fdiv(int a, int b) {  // floor(a / b), b > 0
  int q = a / b;
  return (a < 0 && q * b != a) ? q - 1 : q;
}

__device__ __forceinline__ void set_status(BhmState* st, uint32_t bit) { atomicOr(&st->status, bit); }

__device__ int hash_insert(uint64_t* keys, uint64_t cap, uint64_t k, uint64_t* pos) {
  uint64_t s = mix64(k) & (cap - 1);
  for (uint64_t probe = 0; probe < cap; ++probe) {
    unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(&keys[s]),
                                       (unsigned long long)kEmptyKey, (unsigned long long)k);
    if (old == kEmptyKey) {
      *pos = s;
      return 1;
    }
    if (old == k) {
      *pos = s;
      return 0;
    }
    s = (s + 1) & (cap - 1);
  }
  return -1;
}

__device__ __forceinline__ int find_block(const BhmDev& d, int bx, int by, int bz) {
  return hash_find(d.hkeys, d.hvals, d.hcap, pack_key(bx, by, bz));
}

// the c(xi) of the E-step, (sigmoid(xi) - 1/2) / xi = tanh(xi / 2) / (2 xi); its Taylor series 1/4 - xi^2/48 near 0
__device__ __forceinline__ float jj_coef(float xi) {
  if (xi < 1e-3f) return 0.25f - xi * xi * (1.0f / 48.0f);
  return tanhf(0.5f * xi) / (2.0f * xi);
}

// ---- the feature window of one point -----------------------------------------------------------------------
// A point with lattice coordinate u (g0 = floor(u), fraction f = u - g0) reaches the hinges g0 + delta,
// delta in [-RW, RW + 1]^3; they lie in at most two blocks per axis, the 2 x 2 x 2 blocks from lo.
struct Win {
  int lo[3];
  int s[8];  // slot of block lo + (bx, by, bz) at s[bz * 4 + by * 2 + bx], -1 if not allocated
};

template <bool TOUCH>
__device__ void win_load(const BhmDev& d, Win& w, int lx, int ly, int lz) {
  w.lo[0] = lx;
  w.lo[1] = ly;
  w.lo[2] = lz;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int s = find_block(d, lx + (i & 1), ly + ((i >> 1) & 1), lz + (i >> 2));
    w.s[i] = s;
    if (TOUCH && s >= 0 && d.stamp_touch[s] != d.frame) {
      if (atomicExch(&d.stamp_touch[s], d.frame) != d.frame) d.touched[atomicAdd(&d.st->n_touched, 1)] = s;
    }
  }
}

struct Point {
  int g0[3];
  int base[3];  // g0 - n_h lo (local coordinate in block lo of the hinge at delta = 0)
  long long q[3];
  float f[3];
};

template <int RW, bool TOUCH>
__device__ __forceinline__ void point_setup(const BhmDev& d, Win& w, const double u[3], Point& pt) {
  int lo[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double fl = floor(u[a]);
    pt.g0[a] = (int)fl;
    const double fr = __dsub_rn(u[a], fl);  // exact
    pt.q[a] = (long long)__dmul_rn(fr, (double)(1 << kQ));  // exact scaling, truncation = floor (fr >= 0)
    pt.f[a] = (float)fr;
    lo[a] = fdiv(pt.g0[a] - RW, d.nh);
    pt.base[a] = pt.g0[a] - d.nh * lo[a];
  }
  if (lo[0] != w.lo[0] || lo[1] != w.lo[1] || lo[2] != w.lo[2]) win_load<TOUCH>(d, w, lo[0], lo[1], lo[2]);
}

// fn(index of the weight, phi, f - delta per axis) for every kept hinge feature with an allocated weight.  The x and
// y factors are tabulated (unrolled, in registers); the z offsets are a plain loop that forms its own factor.
template <int RW, class F>
__device__ __forceinline__ void for_features(const BhmDev& d, const Win& w, const Point& pt, F&& fn) {
  constexpr int NO = 2 * RW + 2;
  float e[2][NO], df[2][NO];
  long long dq[2][NO];
  int bit[2][NO], loc[2][NO];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
#pragma unroll
    for (int i = 0; i < NO; ++i) {
      const int delta = i - RW;
      const long long t = pt.q[a] - ((long long)delta << kQ);
      dq[a][i] = t * t;
      df[a][i] = pt.f[a] - (float)delta;
      e[a][i] = expf(-d.gh2 * df[a][i] * df[a][i]);
      const int l = pt.base[a] + delta;
      bit[a][i] = l >= d.nh;
      loc[a][i] = l - (l >= d.nh ? d.nh : 0);
    }
  }
  const long long R2 = d.r2q;
#pragma unroll 1
  for (int dz = -RW; dz <= RW + 1; ++dz) {
    const long long tz = pt.q[2] - ((long long)dz << kQ);
    const long long dqz = tz * tz;
    if (dqz > R2) continue;
    const float dfz = pt.f[2] - (float)dz;
    const float ez = expf(-d.gh2 * dfz * dfz);
    const int lz = pt.base[2] + dz;
    const int bz = lz >= d.nh;
    const int locz = lz - (bz ? d.nh : 0);
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      const long long dzy = dqz + dq[1][j];
      if (dzy > R2) continue;
      const float ezy = ez * e[1][j];
      const int s0 = bz ? (bit[1][j] ? w.s[6] : w.s[4]) : (bit[1][j] ? w.s[2] : w.s[0]);
      const int s1 = bz ? (bit[1][j] ? w.s[7] : w.s[5]) : (bit[1][j] ? w.s[3] : w.s[1]);
      const int lzy = (locz * d.nh + loc[1][j]) * d.nh;
#pragma unroll
      for (int i = 0; i < NO; ++i) {
        if (dzy + dq[0][i] > R2) continue;
        const int s = bit[0][i] ? s1 : s0;
        if (s < 0) continue;
        fn((int64_t)s * d.nw + lzy + loc[0][i], ezy * e[0][i], df[0][i], df[1][j], dfz);
      }
    }
  }
}

// index of the bias weight of the point's own block, or -1
__device__ __forceinline__ int64_t bias_index(const BhmDev& d, const Win& w, const Point& pt) {
  if (!d.bias) return -1;
  const int s = w.s[(pt.base[2] >= d.nh) * 4 + (pt.base[1] >= d.nh) * 2 + (pt.base[0] >= d.nh)];
  return s < 0 ? -1 : (int64_t)s * d.nw + d.nw - 1;
}

// l(u), and optionally grad l (per metre) and phi^T Sigma phi, from the committed weights
template <int RW, bool GRAD, bool VAR>
__device__ void bhm_eval(const BhmDev& d, Win& w, const double u[3], float& l, float3& g, float& v) {
  Point pt;
  point_setup<RW, false>(d, w, u, pt);
  float sl = 0.f, gx = 0.f, gy = 0.f, gz = 0.f, sv = 0.f;
  for_features<RW>(d, w, pt, [&](int64_t idx, float phi, float dx, float dy, float dz) {
    const float2 r = *reinterpret_cast<const float2*>(&d.W[idx]);
    const float mp = r.x * phi;
    sl += mp;
    if (GRAD) {
      gx = fmaf(mp, dx, gx);
      gy = fmaf(mp, dy, gy);
      gz = fmaf(mp, dz, gz);
    }
    if (VAR) sv += phi * phi / r.y;
  });
  const int64_t b = bias_index(d, w, pt);
  if (b >= 0) {
    const float2 r = *reinterpret_cast<const float2*>(&d.W[b]);
    sl += r.x;
    if (VAR) sv += 1.0f / r.y;
  }
  l = sl;
  g = make_float3(d.g2h * gx, d.g2h * gy, d.g2h * gz);
  v = sv;
}

// ---- update kernels --------------------------------------------------------------------------------------

__device__ __forceinline__ bool hit_lattice(const BhmDev& d, const double* hits, int64_t r, double u[3]) {
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u[a] = lat(hits[3 * r + a], d.o[a], d.h);
    ok = ok && lat_ok(u[a]);
  }
  return ok;
}

__global__ void k_bhm_insert(BhmDev d, const double* __restrict__ hits, int64_t R) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double u[3];
  if (!hit_lattice(d, hits, r, u)) {
    set_status(d.st, ST_NONFINITE);
    return;
  }
  const int bx = fdiv((int)floor(u[0]), d.nh), by = fdiv((int)floor(u[1]), d.nh), bz = fdiv((int)floor(u[2]), d.nh);
  for (int i = 0; i < 27; ++i) {
    uint64_t pos;
    const int rc = hash_insert(d.hkeys, d.hcap, pack_key(bx + i % 3 - 1, by + (i / 3) % 3 - 1, bz + i / 9 - 1), &pos);
    if (rc < 0) {
      set_status(d.st, ST_CAPACITY);
    } else if (rc == 1) {
      const int k = atomicAdd(&d.st->n_new, 1);
      d.new_list[k] = (int32_t)pos;  // table positions: at most one insertion per key
    }
  }
}

// give every key inserted by this update a slot (in list order after the existing blocks) and the prior weights
__global__ void k_bhm_assign(BhmDev d) {
  const int nb = d.st->n_blocks, nn = d.st->n_new;
  for (int i = blockIdx.x; i < nn; i += gridDim.x) {
    const uint64_t pos = (uint64_t)d.new_list[i];
    const int id = nb + i;
    if (id >= d.max_blocks) {
      if (threadIdx.x == 0) set_status(d.st, ST_CAPACITY);
      continue;  // the key stays in the table with no slot: lookups treat it as absent
    }
    if (threadIdx.x == 0) {
      d.hvals[pos] = id;
      d.bkey[id] = d.hkeys[pos];
      d.active[id] = 0;
      d.stamp_touch[id] = -1;
      d.stamp_mark[id] = -1;
      d.mark_idx[id] = -1;
    }
    for (int k = threadIdx.x; k < d.nw; k += blockDim.x) {
      d.W[(int64_t)id * d.nw + k] = make_float4(0.f, d.prior_prec, 0.f, 0.f);
      d.PB[(int64_t)id * d.nw + k] = 0.f;
    }
  }
}

__global__ void k_bhm_counts(BhmDev d) {
  BhmState* st = d.st;
  const int nb = st->n_blocks + st->n_new;
  st->n_blocks = nb < d.max_blocks ? nb : d.max_blocks;
  st->n_new = 0;
  st->n_touched = 0;
  st->n_marked = 0;
  st->n_samples = 0ull;
  st->lsum = 0.0;
}

__global__ void k_bhm_activate(BhmDev d, const double* __restrict__ hits, int64_t R) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double u[3];
  if (!hit_lattice(d, hits, r, u)) return;
  const int s = find_block(d, fdiv((int)floor(u[0]), d.nh), fdiv((int)floor(u[1]), d.nh), fdiv((int)floor(u[2]), d.nh));
  if (s >= 0) d.active[s] = 1;
}

// One EM round over every ray's samples.  FIRST: xi = xi_init, accumulates B and A into W (and builds the
// touched-block list).  Otherwise: the M-step for each sample from the previous round's accumulators (src: 0 = A
// in W, 1 = PB), then the E-step statistic c(xi) phi^2 into dst.
template <int RW, bool FIRST>
__device__ __forceinline__ void em_sample(const BhmDev& d, Win& w, const double u[3], float tlab, int src, int dst) {
  Point pt;
  point_setup<RW, FIRST>(d, w, u, pt);
  const int64_t bidx = bias_index(d, w, pt);
  float xi = d.xi0;
  if (!FIRST) {
    float vs = 0.f, ms = 0.f;
    auto mstep = [&](int64_t idx, float phi) {
      const float4 r = d.W[idx];
      const float a = src ? d.PB[idx] : r.w;
      const float P = r.y + a;
      const float mu = fmaf(r.y, r.x, r.z) / P;
      vs = fmaf(phi * phi, 1.0f / P, vs);
      ms = fmaf(mu, phi, ms);
    };
    for_features<RW>(d, w, pt, [&](int64_t idx, float phi, float, float, float) { mstep(idx, phi); });
    if (bidx >= 0) mstep(bidx, 1.0f);
    xi = sqrtf(fmaf(ms, ms, vs));
  }
  const float c = jj_coef(xi);
  const float tb = tlab - 0.5f;
  auto estep = [&](int64_t idx, float phi) {
    float* acc = dst ? &d.PB[idx] : &d.W[idx].w;
    atomicAdd(acc, c * phi * phi);
    if (FIRST) atomicAdd(&d.W[idx].z, tb * phi);
  };
  for_features<RW>(d, w, pt, [&](int64_t idx, float phi, float, float, float) { estep(idx, phi); });
  if (bidx >= 0) estep(bidx, 1.0f);
}

template <int RW, bool FIRST>
__global__ void __launch_bounds__(kT) k_bhm_em(BhmDev d, const double* __restrict__ hits, int64_t R, int src, int dst) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double ux[3];
  if (!hit_lattice(d, hits, r, ux)) return;
  const double dx = __dsub_rn(hits[3 * r], d.p[0]), dy = __dsub_rn(hits[3 * r + 1], d.p[1]),
               dz = __dsub_rn(hits[3 * r + 2], d.p[2]);
  const double L = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
  long long jmax = 0;
  double sig = 0.0;
  if (L > 0.0) {
    const double t = floor(__ddiv_rn(__dsub_rn(L, d.fgap), d.fstep));
    jmax = t > 0.0 ? (long long)t : 0;
    sig = __ddiv_rn(d.fstep, L);
  }
  double du[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) du[a] = __dsub_rn(ux[a], d.up[a]);
  Win w;
  w.lo[0] = w.lo[1] = w.lo[2] = INT_MIN;
  int cb[3] = {INT_MIN, INT_MIN, INT_MIN};
  bool cact = false;
  unsigned long long count = 0;
  for (long long j = 1; j <= jmax; ++j) {
    const double s = __dmul_rn((double)j, sig);
    double u[3];
    int b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      u[a] = __dadd_rn(d.up[a], __dmul_rn(s, du[a]));
      b[a] = fdiv((int)floor(u[a]), d.nh);
    }
    if (b[0] != cb[0] || b[1] != cb[1] || b[2] != cb[2]) {
      cb[0] = b[0];
      cb[1] = b[1];
      cb[2] = b[2];
      const int sl = find_block(d, b[0], b[1], b[2]);
      cact = sl >= 0 && d.active[sl];
    }
    if (!cact) {
      // every sample up to one step before the ray leaves this block is in it: jump there
      double sx = 1e300;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (du[a] != 0.0) {
          const double bnd = (double)(d.nh * (du[a] > 0.0 ? b[a] + 1 : b[a]));
          sx = fmin(sx, (bnd - d.up[a]) / du[a]);
        }
      }
      const double jn = floor(sx / sig) - 1.0;
      if (jn > (double)j) j = jn < (double)jmax ? (long long)jn : jmax;
      continue;
    }
    em_sample<RW, FIRST>(d, w, u, 0.0f, src, dst);
    ++count;
  }
  em_sample<RW, FIRST>(d, w, ux, 1.0f, src, dst);
  ++count;
  if (FIRST) atomicAdd(&d.st->n_samples, count);
}

// zero one accumulator of every touched block (between EM rounds three and four)
__global__ void k_bhm_zero_acc(BhmDev d, int which) {
  const int n = d.st->n_touched;
  for (int b = blockIdx.x; b < n; b += gridDim.x) {
    const int64_t base = (int64_t)d.touched[b] * d.nw;
    for (int k = threadIdx.x; k < d.nw; k += blockDim.x) {
      if (which) d.PB[base + k] = 0.f;
      else d.W[base + k].w = 0.f;
    }
  }
}

// the last E-step's posterior becomes the map: P = P_prev + A, mu = (P_prev mu_prev + B) / P; accumulators cleared
__global__ void k_bhm_commit(BhmDev d, int last) {
  const int n = d.st->n_touched;
  for (int b = blockIdx.x; b < n; b += gridDim.x) {
    const int64_t base = (int64_t)d.touched[b] * d.nw;
    for (int k = threadIdx.x; k < d.nw; k += blockDim.x) {
      float4 r = d.W[base + k];
      const float a = last ? d.PB[base + k] : r.w;
      if (a != 0.f) {
        const float P = r.y + a;
        r.x = fmaf(r.y, r.x, r.z) / P;
        r.y = P;
      }
      r.z = 0.f;
      r.w = 0.f;
      d.W[base + k] = r;
      d.PB[base + k] = 0.f;
    }
  }
}

template <int RW>
__global__ void k_bhm_tau_sum(BhmDev d, const double* __restrict__ hits, int64_t R) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (r < R) {
    double u[3];
    if (hit_lattice(d, hits, r, u)) {
      Win w;
      w.lo[0] = w.lo[1] = w.lo[2] = INT_MIN;
      float lf, v;
      float3 g;
      bhm_eval<RW, false, false>(d, w, u, lf, g, v);
      l = (double)lf;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(&d.st->lsum, l);
}

__global__ void k_bhm_tau_fin(BhmDev d) {
  BhmState* st = d.st;
  st->tau = __dadd_rn(__dmul_rn(d.tau_a, st->tau), __dmul_rn(d.tau_b, st->lsum));
  st->lsum = 0.0;
}

// marching cells: nu = floor(m u); block of a cell = floor(nu / (n_h m))
__device__ __forceinline__ bool hit_cell(const BhmDev& d, const double* hits, int64_t r, int c[3]) {
  double u[3];
  if (!hit_lattice(d, hits, r, u)) return false;
#pragma unroll
  for (int a = 0; a < 3; ++a) c[a] = (int)floor(__dmul_rn(u[a], (double)d.msub));
  return true;
}

// claim a mask for every block holding a node of a marked cell (cells c - 1 .. c + 1 of each hit cell c, so nodes
// c - 1 .. c + 2): the march walks the nodes of claimed blocks
__global__ void k_bhm_mark_claim(BhmDev d, const double* __restrict__ hits, int64_t R) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  int c[3];
  if (!hit_cell(d, hits, r, c)) return;
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = fdiv(c[a] - 1, d.cdim);
    hi[a] = fdiv(c[a] + 2, d.cdim);
  }
  for (int bz = lo[2]; bz <= hi[2]; ++bz)
    for (int by = lo[1]; by <= hi[1]; ++by)
      for (int bx = lo[0]; bx <= hi[0]; ++bx) {
        const int s = find_block(d, bx, by, bz);
        if (s < 0 || d.stamp_mark[s] == d.frame) continue;
        if (atomicExch(&d.stamp_mark[s], d.frame) != d.frame) {
          const int k = atomicAdd(&d.st->n_marked, 1);
          if (k < d.max_marked) {
            d.mark_idx[s] = k;
            d.marked[k] = s;
          } else {
            d.mark_idx[s] = -1;
            set_status(d.st, ST_CAPACITY);
          }
        }
      }
}

__global__ void k_bhm_mask_zero(BhmDev d) {
  const int n = min(d.st->n_marked, d.max_marked);
  for (int b = blockIdx.x; b < n; b += gridDim.x)
    for (int k = threadIdx.x; k < d.mask_words; k += blockDim.x) d.masks[(int64_t)b * d.mask_words + k] = 0u;
}

__global__ void k_bhm_mark_set(BhmDev d, const double* __restrict__ hits, int64_t R) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  int c[3];
  if (!hit_cell(d, hits, r, c)) return;
  for (int i = 0; i < 27; ++i) {
    const int cx = c[0] + i % 3 - 1, cy = c[1] + (i / 3) % 3 - 1, cz = c[2] + i / 9 - 1;
    const int bx = fdiv(cx, d.cdim), by = fdiv(cy, d.cdim), bz = fdiv(cz, d.cdim);
    const int s = find_block(d, bx, by, bz);
    if (s < 0) continue;
    const int k = d.mark_idx[s];
    if (k < 0) continue;
    const int bitn = ((cz - bz * d.cdim) * d.cdim + (cy - by * d.cdim)) * d.cdim + (cx - bx * d.cdim);
    atomicOr(&d.masks[(int64_t)k * d.mask_words + (bitn >> 5)], 1u << (bitn & 31));
  }
}

// ---- surface points ------------------------------------------------------------------------------------------

struct MarchOut {
  uint64_t* key;
  uint32_t* val;
  double* x;
  float* var;
  float* nrm;
  int64_t cap;
};

template <int RW>
__global__ void __launch_bounds__(kT) k_bhm_march(BhmDev d, MarchOut mo) {
  __shared__ int nbr[27];  // mark index of the 27 blocks around (only the lower seven are read), -1 if unmarked
  const int nmk = min(d.st->n_marked, d.max_marked);
  const double tau = d.st->tau;
  const int C = d.cdim;
  for (int mb = blockIdx.x; mb < nmk; mb += gridDim.x) {
    const int slot = d.marked[mb];
    int bx, by, bz;
    unpack_key(d.bkey[slot], bx, by, bz);
    __syncthreads();
    if (threadIdx.x < 27) {
      const int s = find_block(d, bx + threadIdx.x % 3 - 1, by + (threadIdx.x / 3) % 3 - 1, bz + threadIdx.x / 9 - 1);
      nbr[threadIdx.x] = (s >= 0 && d.stamp_mark[s] == d.frame) ? d.mark_idx[s] : -1;
    }
    __syncthreads();
    // is local cell (cx, cy, cz), each in [-1, C), marked?
    auto marked = [&](int cx, int cy, int cz) -> bool {
      const int k = nbr[(cz < 0 ? 0 : 1) * 9 + (cy < 0 ? 0 : 1) * 3 + (cx < 0 ? 0 : 1)];
      if (k < 0) return false;
      const int lx = cx < 0 ? C - 1 : cx, ly = cy < 0 ? C - 1 : cy, lz = cz < 0 ? C - 1 : cz;
      const int bitn = (lz * C + ly) * C + lx;
      return (d.masks[(int64_t)k * d.mask_words + (bitn >> 5)] >> (bitn & 31)) & 1u;
    };
    Win w;
    w.lo[0] = w.lo[1] = w.lo[2] = INT_MIN;
    const int nn = C * C * C;
    for (int n = threadIdx.x; n < nn; n += blockDim.x) {
      const int lx = n % C, ly = (n / C) % C, lz = n / (C * C);
      const int l3[3] = {lx, ly, lz};
      bool doit[3];
      bool any = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
        bool m = false;
#pragma unroll
        for (int ib = 0; ib < 2; ++ib)
#pragma unroll
          for (int ic = 0; ic < 2; ++ic) {
            int cc[3] = {l3[0], l3[1], l3[2]};
            cc[b] -= ib;
            cc[c] -= ic;
            m = m || marked(cc[0], cc[1], cc[2]);
          }
        doit[a] = m;
        any = any || m;
      }
      if (!any) continue;
      const int nu[3] = {bx * C + lx, by * C + ly, bz * C + lz};
      double u0[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) u0[a] = __dmul_rn((double)nu[a], d.inv_m);
      float la, lb, lv, vv;
      float3 g;
      bhm_eval<RW, false, false>(d, w, u0, la, g, vv);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (!doit[a]) continue;
        double u1[3] = {u0[0], u0[1], u0[2]};
        u1[a] = __dmul_rn((double)(nu[a] + 1), d.inv_m);
        bhm_eval<RW, false, false>(d, w, u1, lb, g, vv);
        if (((double)la >= tau) == ((double)lb >= tau)) continue;
        const double t = ((tau - (double)la) / ((double)lb - (double)la));
        double ui[3] = {u0[0], u0[1], u0[2]};
        ui[a] = __dmul_rn(__dadd_rn((double)nu[a], t), d.inv_m);
        bhm_eval<RW, true, false>(d, w, ui, lv, g, vv);
        const float g2 = g.x * g.x + g.y * g.y + g.z * g.z;
        if (!(g2 > 0.f)) continue;
        const int64_t k = atomicAdd(&d.st->n_out, 1);
        if (k >= mo.cap) continue;
        const float dl = (float)(tau - (double)lv);
        const float ig = rsqrtf(g2);
        mo.key[k] = ((uint64_t)(nu[2] + kEdgeBias) << 42) | ((uint64_t)(nu[1] + kEdgeBias) << 22) |
                    ((uint64_t)(nu[0] + kEdgeBias) << 2) | (uint64_t)a;
        mo.val[k] = (uint32_t)k;
#pragma unroll
        for (int e = 0; e < 3; ++e) mo.x[3 * k + e] = __dadd_rn(d.o[e], __dmul_rn(ui[e], d.h));
        mo.var[k] = d.beta * dl * dl / g2;
        mo.nrm[3 * k] = -g.x * ig;
        mo.nrm[3 * k + 1] = -g.y * ig;
        mo.nrm[3 * k + 2] = -g.z * ig;
      }
    }
  }
}

__global__ void k_bhm_gather(MarchOut mo, int64_t n, double* x, float* var, float* nrm, uint64_t* keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t j = mo.val[i];
  if (x)
    for (int e = 0; e < 3; ++e) x[3 * i + e] = mo.x[3 * j + e];
  if (var) var[i] = mo.var[j];
  if (nrm)
    for (int e = 0; e < 3; ++e) nrm[3 * i + e] = mo.nrm[3 * j + e];
  if (keys) keys[i] = mo.key[i];
}

// ---- prediction --------------------------------------------------------------------------------------------

template <int RW>
__global__ void k_bhm_query(BhmDev d, const float* __restrict__ xq, int64_t Q, uint32_t mask, float* lo, int8_t* sg,
                            float* gr, float* pr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Q) return;
  double u[3];
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u[a] = lat((double)xq[3 * i + a], d.o[a], d.h);
    ok = ok && lat_ok(u[a]);
  }
  float l, v;
  float3 g;
  if (!ok) {
    set_status(d.st, ST_NONFINITE);
    l = v = __int_as_float(0x7fc00000);
    g = make_float3(l, l, l);
  } else {
    Win w;
    w.lo[0] = w.lo[1] = w.lo[2] = INT_MIN;
    if (mask & (KSDF_BHM_GRAD | KSDF_BHM_PROB)) bhm_eval<RW, true, true>(d, w, u, l, g, v);
    else bhm_eval<RW, false, false>(d, w, u, l, g, v);
  }
  if (mask & KSDF_BHM_LOGODDS) lo[i] = l;
  if (mask & KSDF_BHM_SIGN) sg[i] = (ok && (double)l < d.st->tau) || !ok ? (int8_t)1 : (int8_t)-1;
  if (mask & KSDF_BHM_GRAD) {
    gr[3 * i] = g.x;
    gr[3 * i + 1] = g.y;
    gr[3 * i + 2] = g.z;
  }
  if (mask & KSDF_BHM_PROB) pr[i] = 1.0f / (1.0f + expf(-l / sqrtf(1.0f + 0.39269908169872414f * v)));
}

}  // namespace
}  // namespace ksdf

// ============================================================================================================
// the map object and the C ABI

using namespace ksdf;

struct ksdf_bhm {
  ksdf_bhm_params p{};
  cudaStream_t stream = nullptr;
  std::string err;
  int rw = 0, nh = 0, nw = 0, cdim = 0, mask_words = 0, frame = -1;
  long long r2q = 0;
  int64_t max_blocks = 0, max_marked = 0;
  uint64_t hcap = 0;
  DevBuf hkeys, hvals, bkey, active, stamps, lists, W, PB, masks, state;
  DevBuf stage_hits, mkey, mval, mx, mvar, mnrm, sort_tmp, out_stage[4], q_stage[5];
  int64_t mcap = 0;
  double up[3] = {0, 0, 0}, p_last[3] = {0, 0, 0};
};

namespace {

ksdf_status berr(ksdf_bhm* m, ksdf_status s, const char* fmt, ...) {
  if (m) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    m->err = buf;
  }
  return s;
}

#define BHM_CUDA(m, call)                                                                                \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return berr(m, KSDF_ERR_CUDA, "CUDA error %d (%s) in %s", (int)e_, cudaGetErrorString(e_), #call); \
  } while (0)

bool dev_ptr(const void* p) {
  if (!p) return true;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

BhmDev dev_view(ksdf_bhm* m) {
  BhmDev d{};
  for (int a = 0; a < 3; ++a) {
    d.o[a] = m->p.origin[a];
    d.p[a] = m->p_last[a];
    d.up[a] = m->up[a];
  }
  d.h = m->p.hinge_spacing;
  d.fstep = m->p.free_step;
  d.fgap = m->p.free_gap;
  d.inv_m = 1.0 / m->p.march_sub;
  d.gh2 = (float)(m->p.gamma * m->p.hinge_spacing * m->p.hinge_spacing);
  d.g2h = (float)(-2.0 * m->p.gamma * m->p.hinge_spacing);
  d.prior_prec = (float)(1.0 / m->p.prior_var);
  d.xi0 = (float)m->p.xi_init;
  d.beta = (float)m->p.beta;
  d.r2q = m->r2q;
  d.nh = m->nh;
  d.nw = m->nw;
  d.msub = m->p.march_sub;
  d.cdim = m->cdim;
  d.mask_words = m->mask_words;
  d.frame = m->frame;
  d.max_blocks = (int)m->max_blocks;
  d.max_marked = (int)m->max_marked;
  d.bias = m->p.bias_feature;
  d.hcap = m->hcap;
  d.hkeys = ptr<uint64_t>(m->hkeys);
  d.hvals = ptr<int32_t>(m->hvals);
  d.bkey = ptr<uint64_t>(m->bkey);
  d.active = ptr<uint8_t>(m->active);
  int32_t* st = ptr<int32_t>(m->stamps);
  d.stamp_touch = st;
  d.stamp_mark = st + m->max_blocks;
  d.mark_idx = st + 2 * m->max_blocks;
  int32_t* li = ptr<int32_t>(m->lists);
  d.new_list = li;
  d.touched = li + m->hcap;
  d.marked = li + m->hcap + m->max_blocks;
  d.W = ptr<float4>(m->W);
  d.PB = ptr<float>(m->PB);
  d.masks = ptr<uint32_t>(m->masks);
  d.st = ptr<BhmState>(m->state);
  return d;
}

unsigned nblk(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

}  // namespace

extern "C" {

ksdf_status ksdf_bhm_create(const ksdf_bhm_params* prm, int64_t max_blocks, int64_t max_marked, void* stream,
                            ksdf_bhm** out) {
  if (!prm || !out) return KSDF_ERR_ARG;
  *out = nullptr;
  const ksdf_bhm_params& p = *prm;
  bool ok = std::isfinite(p.hinge_spacing) && p.hinge_spacing > 0 && p.block_hinges >= 4 && p.block_hinges <= 16 &&
            std::isfinite(p.gamma) && p.gamma > 0 && p.phi_min > 0 && p.phi_min < 1 && std::isfinite(p.prior_var) &&
            p.prior_var > 0 && p.em_iters >= 1 && p.em_iters <= 4 && std::isfinite(p.xi_init) && p.xi_init >= 0 &&
            std::isfinite(p.free_step) && p.free_step > 0 && std::isfinite(p.free_gap) && p.free_gap >= 0 &&
            p.tau_alpha > 0 && p.tau_alpha <= 1 && std::isfinite(p.tau_init) && std::isfinite(p.beta) && p.beta > 0 &&
            (p.march_sub == 1 || p.march_sub == 2 || p.march_sub == 4 || p.march_sub == 8) &&
            (p.bias_feature == 0 || p.bias_feature == 1) && max_blocks >= 1 &&
            max_blocks <= (1LL << 24) && max_marked >= 0;
  for (int a = 0; a < 3; ++a) ok = ok && std::isfinite(p.origin[a]);
  if (!ok) return KSDF_ERR_ARG;
  const double r2 = std::log(1.0 / p.phi_min) / (p.gamma * p.hinge_spacing * p.hinge_spacing) * 1099511627776.0;
  if (!(r2 >= 0 && r2 < 9.0e18)) return KSDF_ERR_ARG;
  const long long r2q = (long long)std::floor(r2);
  long long rt = (long long)std::sqrt((double)r2q);  // integer square root
  while (rt * rt > r2q) --rt;
  while ((rt + 1) * (rt + 1) <= r2q) ++rt;
  const int rw = (int)(rt >> kQ);
  if (rw > 2 || 2 * rw + 1 > p.block_hinges) return KSDF_ERR_ARG;
  const int cdim = p.block_hinges * p.march_sub;
  if (cdim > 64) return KSDF_ERR_ARG;

  ksdf_bhm* m = new ksdf_bhm();
  m->p = p;
  m->stream = (cudaStream_t)stream;
  m->rw = rw;
  m->r2q = r2q;
  m->nh = p.block_hinges;
  m->nw = p.block_hinges * p.block_hinges * p.block_hinges + 1;
  m->cdim = cdim;
  m->mask_words = (cdim * cdim * cdim + 31) / 32;
  m->max_blocks = max_blocks;
  m->max_marked = max_marked ? std::min(max_marked, max_blocks) : max_blocks;
  uint64_t cap = 1024;
  while (cap < 4ull * (uint64_t)max_blocks) cap <<= 1;
  m->hcap = cap;
  cudaError_t e = cudaSuccess;
  auto al = [&](DevBuf& b, size_t bytes) {
    if (e == cudaSuccess) e = ensure(b, bytes);
  };
  al(m->hkeys, 8 * cap);
  al(m->hvals, 4 * cap);
  al(m->bkey, 8 * (size_t)max_blocks);
  al(m->active, (size_t)max_blocks);
  al(m->stamps, 12 * (size_t)max_blocks);
  al(m->lists, 4 * (cap + 2 * (size_t)max_blocks));  // new-key list (one per table position), touched, marked
  al(m->W, 16 * (size_t)max_blocks * m->nw);
  al(m->PB, 4 * (size_t)max_blocks * m->nw);
  al(m->masks, 4 * (size_t)m->max_marked * m->mask_words);
  al(m->state, sizeof(BhmState));
  if (e == cudaSuccess) e = cudaMemsetAsync(m->hkeys.p, 0xff, 8 * cap, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->hvals.p, 0xff, 4 * cap, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->state.p, 0, sizeof(BhmState), m->stream);
  if (e == cudaSuccess) {
    const double tau = p.tau_init;
    e = cudaMemcpyAsync(reinterpret_cast<char*>(m->state.p) + offsetof(BhmState, tau), &tau, sizeof(double),
                        cudaMemcpyHostToDevice, m->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    ksdf_bhm_destroy(m);
    return KSDF_ERR_CUDA;
  }
  *out = m;
  return KSDF_OK;
}

ksdf_status ksdf_bhm_destroy(ksdf_bhm* m) {
  if (!m) return KSDF_OK;
  DevBuf* bufs[] = {&m->hkeys, &m->hvals, &m->bkey, &m->active, &m->stamps, &m->lists, &m->W, &m->PB,
                    &m->masks, &m->state, &m->stage_hits, &m->mkey, &m->mval, &m->mx, &m->mvar, &m->mnrm,
                    &m->sort_tmp};
  for (DevBuf* b : bufs) release(*b);
  for (DevBuf& b : m->out_stage) release(b);
  for (DevBuf& b : m->q_stage) release(b);
  delete m;
  return KSDF_OK;
}

ksdf_status ksdf_bhm_set_stream(ksdf_bhm* m, void* stream) {
  if (!m) return KSDF_ERR_ARG;
  m->stream = (cudaStream_t)stream;
  return KSDF_OK;
}

ksdf_status ksdf_bhm_update(ksdf_bhm* m, const double* p, const double* hits, int64_t R) {
  if (!m) return KSDF_ERR_ARG;
  if (!p || R < 0 || (R > 0 && !hits)) return berr(m, KSDF_ERR_ARG, "ksdf_bhm_update: need p and R >= 0 hits");
  if (R >= (1LL << 31)) return berr(m, KSDF_ERR_CAPACITY, "ksdf_bhm_update: R must be < 2^31");
  for (int a = 0; a < 3; ++a) {
    const double u = (p[a] - m->p.origin[a]) / m->p.hinge_spacing;
    if (!(u > -kLatMax && u < kLatMax)) return berr(m, KSDF_ERR_ARG, "ksdf_bhm_update: sensor position out of range");
    m->up[a] = u;
    m->p_last[a] = p[a];
  }
  const double* dh = hits;
  if (R > 0 && !dev_ptr(hits)) {
    BHM_CUDA(m, ensure(m->stage_hits, sizeof(double) * 3 * R));
    BHM_CUDA(m, cudaMemcpyAsync(m->stage_hits.p, hits, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, m->stream));
    dh = ptr<double>(m->stage_hits);
  }
  ++m->frame;
  BhmDev d = dev_view(m);
  d.tau_a = 1.0 - m->p.tau_alpha;
  d.tau_b = R > 0 ? m->p.tau_alpha / (double)R : 0.0;
  cudaStream_t st = m->stream;
  const unsigned g = nblk(R);
  if (R > 0) launch(k_bhm_insert, g, kT, 0, st, d, dh, R);
  launch(k_bhm_assign, kGridStride, kT, 0, st, d);
  launch(k_bhm_counts, 1, 1, 0, st, d);
  if (R > 0) {
    launch(k_bhm_activate, g, kT, 0, st, d, dh, R);
    const int iters = m->p.em_iters;
    for (int it = 1; it <= iters; ++it) {
      const int dst = (it - 1) & 1, src = it >= 2 ? (it - 2) & 1 : 0;
      if (it >= 3) launch(k_bhm_zero_acc, kGridStride, kT, 0, st, d, dst);
      switch (m->rw) {
#define EM_CASE(RWV)                                                                   \
  case RWV:                                                                            \
    if (it == 1) launch(k_bhm_em<RWV, true>, g, kT, 0, st, d, dh, R, src, dst);        \
    else launch(k_bhm_em<RWV, false>, g, kT, 0, st, d, dh, R, src, dst);               \
    break;
        EM_CASE(0)
        EM_CASE(1)
        EM_CASE(2)
#undef EM_CASE
      }
    }
    launch(k_bhm_commit, kGridStride, kT, 0, st, d, (iters - 1) & 1);
    switch (m->rw) {
      case 0: launch(k_bhm_tau_sum<0>, g, kT, 0, st, d, dh, R); break;
      case 1: launch(k_bhm_tau_sum<1>, g, kT, 0, st, d, dh, R); break;
      default: launch(k_bhm_tau_sum<2>, g, kT, 0, st, d, dh, R); break;
    }
    launch(k_bhm_tau_fin, 1, 1, 0, st, d);
    launch(k_bhm_mark_claim, g, kT, 0, st, d, dh, R);
    launch(k_bhm_mask_zero, kGridStride, kT, 0, st, d);
    launch(k_bhm_mark_set, g, kT, 0, st, d, dh, R);
  }
  BHM_CUDA(m, cudaGetLastError());
  return KSDF_OK;
}

ksdf_status ksdf_bhm_march(ksdf_bhm* m, int64_t cap, double* x, float* var, float* normals, uint64_t* keys,
                           int64_t* n_out) {
  if (!m) return KSDF_ERR_ARG;
  if (cap < 0 || !n_out) return berr(m, KSDF_ERR_ARG, "ksdf_bhm_march: need cap >= 0 and n_out");
  *n_out = 0;
  cudaStream_t st = m->stream;
  if (m->frame < 0) return KSDF_OK;
  BhmDev d = dev_view(m);
  int32_t n = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (m->mcap == 0 || (attempt == 1)) {
      const int64_t want = std::max<int64_t>(1 << 16, (int64_t)n + (n >> 3));
      BHM_CUDA(m, ensure(m->mkey, 8 * want));
      BHM_CUDA(m, ensure(m->mval, 4 * want));
      BHM_CUDA(m, ensure(m->mx, 24 * want));
      BHM_CUDA(m, ensure(m->mvar, 4 * want));
      BHM_CUDA(m, ensure(m->mnrm, 12 * want));
      m->mcap = want;
    }
    MarchOut mo{ptr<uint64_t>(m->mkey), ptr<uint32_t>(m->mval), ptr<double>(m->mx), ptr<float>(m->mvar),
                ptr<float>(m->mnrm), m->mcap};
    BHM_CUDA(m, cudaMemsetAsync(reinterpret_cast<char*>(m->state.p) + offsetof(BhmState, n_out), 0, 4, st));
    switch (m->rw) {
      case 0: launch(k_bhm_march<0>, kGridStride, kT, 0, st, d, mo); break;
      case 1: launch(k_bhm_march<1>, kGridStride, kT, 0, st, d, mo); break;
      default: launch(k_bhm_march<2>, kGridStride, kT, 0, st, d, mo); break;
    }
    BHM_CUDA(m, cudaGetLastError());
    BHM_CUDA(m, cudaMemcpyAsync(&n, reinterpret_cast<char*>(m->state.p) + offsetof(BhmState, n_out), 4,
                                cudaMemcpyDeviceToHost, st));
    BHM_CUDA(m, cudaStreamSynchronize(st));
    if (n <= m->mcap) break;
  }
  *n_out = n;
  if (n > cap) return berr(m, KSDF_ERR_CAPACITY, "ksdf_bhm_march: %d points, cap %lld", n, (long long)cap);
  if (n == 0) return KSDF_OK;
  MarchOut mo{ptr<uint64_t>(m->mkey), ptr<uint32_t>(m->mval), ptr<double>(m->mx), ptr<float>(m->mvar),
              ptr<float>(m->mnrm), m->mcap};
  BHM_CUDA(m, radix_sort_u64(mo.key, mo.val, n, 62, m->sort_tmp, st));
  void* outs[4] = {x, var, normals, keys};
  const size_t bytes[4] = {24 * (size_t)n, 4 * (size_t)n, 12 * (size_t)n, 8 * (size_t)n};
  void* dv[4];
  for (int i = 0; i < 4; ++i) {
    dv[i] = outs[i];
    if (outs[i] && !dev_ptr(outs[i])) {
      BHM_CUDA(m, ensure(m->out_stage[i], bytes[i]));
      dv[i] = m->out_stage[i].p;
    }
  }
  launch(k_bhm_gather, nblk(n), kT, 0, st, mo, (int64_t)n, (double*)dv[0], (float*)dv[1], (float*)dv[2],
         (uint64_t*)dv[3]);
  BHM_CUDA(m, cudaGetLastError());
  for (int i = 0; i < 4; ++i)
    if (outs[i] && dv[i] != outs[i])
      BHM_CUDA(m, cudaMemcpyAsync(outs[i], dv[i], bytes[i], cudaMemcpyDeviceToHost, st));
  BHM_CUDA(m, cudaStreamSynchronize(st));
  return KSDF_OK;
}

ksdf_status ksdf_bhm_query(ksdf_bhm* m, const float* xq, int64_t Q, uint32_t out_mask, float* logodds, int8_t* sign,
                           float* grad, float* prob) {
  if (!m) return KSDF_ERR_ARG;
  if (Q < 0 || (Q > 0 && !xq)) return berr(m, KSDF_ERR_ARG, "ksdf_bhm_query: bad Q or NULL points");
  if (Q >= (1LL << 31)) return berr(m, KSDF_ERR_CAPACITY, "ksdf_bhm_query: Q must be < 2^31");
  if (((out_mask & KSDF_BHM_LOGODDS) && !logodds) || ((out_mask & KSDF_BHM_SIGN) && !sign) ||
      ((out_mask & KSDF_BHM_GRAD) && !grad) || ((out_mask & KSDF_BHM_PROB) && !prob))
    return berr(m, KSDF_ERR_ARG, "ksdf_bhm_query: an output selected by out_mask is NULL");
  if (Q == 0) return KSDF_OK;
  cudaStream_t st = m->stream;
  const float* dq = xq;
  if (!dev_ptr(xq)) {
    BHM_CUDA(m, ensure(m->q_stage[0], 12 * (size_t)Q));
    BHM_CUDA(m, cudaMemcpyAsync(m->q_stage[0].p, xq, 12 * (size_t)Q, cudaMemcpyHostToDevice, st));
    dq = ptr<float>(m->q_stage[0]);
  }
  void* outs[4] = {(out_mask & KSDF_BHM_LOGODDS) ? logodds : nullptr, (out_mask & KSDF_BHM_SIGN) ? sign : nullptr,
                   (out_mask & KSDF_BHM_GRAD) ? grad : nullptr, (out_mask & KSDF_BHM_PROB) ? prob : nullptr};
  const size_t bytes[4] = {4 * (size_t)Q, (size_t)Q, 12 * (size_t)Q, 4 * (size_t)Q};
  void* dv[4];
  bool host_out = false;
  for (int i = 0; i < 4; ++i) {
    dv[i] = outs[i];
    if (outs[i] && !dev_ptr(outs[i])) {
      BHM_CUDA(m, ensure(m->q_stage[1 + i], bytes[i]));
      dv[i] = m->q_stage[1 + i].p;
      host_out = true;
    }
  }
  BhmDev d = dev_view(m);
  switch (m->rw) {
#define Q_CASE(RWV)                                                                                    \
  case RWV:                                                                                            \
    launch(k_bhm_query<RWV>, nblk(Q), kT, 0, st, d, dq, Q, out_mask & 15u, (float*)dv[0], (int8_t*)dv[1], \
           (float*)dv[2], (float*)dv[3]);                                                              \
    break;
    Q_CASE(0)
    Q_CASE(1)
    Q_CASE(2)
#undef Q_CASE
  }
  BHM_CUDA(m, cudaGetLastError());
  for (int i = 0; i < 4; ++i)
    if (outs[i] && dv[i] != outs[i])
      BHM_CUDA(m, cudaMemcpyAsync(outs[i], dv[i], bytes[i], cudaMemcpyDeviceToHost, st));
  if (host_out) BHM_CUDA(m, cudaStreamSynchronize(st));
  return KSDF_OK;
}

ksdf_status ksdf_bhm_size(ksdf_bhm* m, int64_t* n_blocks, int64_t* n_samples_last) {
  if (!m) return KSDF_ERR_ARG;
  BhmState s;
  BHM_CUDA(m, cudaMemcpyAsync(&s, m->state.p, sizeof(s), cudaMemcpyDeviceToHost, m->stream));
  BHM_CUDA(m, cudaStreamSynchronize(m->stream));
  if (n_blocks) *n_blocks = s.n_blocks;
  if (n_samples_last) *n_samples_last = (int64_t)s.n_samples;
  return KSDF_OK;
}

ksdf_status ksdf_bhm_get(ksdf_bhm* m, uint64_t* keys, uint8_t* active, float* mu, float* prec) {
  if (!m) return KSDF_ERR_ARG;
  int64_t nb = 0;
  ksdf_status s = ksdf_bhm_size(m, &nb, nullptr);
  if (s != KSDF_OK) return s;
  cudaStream_t st = m->stream;
  if (keys) BHM_CUDA(m, cudaMemcpyAsync(keys, m->bkey.p, 8 * nb, cudaMemcpyDeviceToHost, st));
  if (active) BHM_CUDA(m, cudaMemcpyAsync(active, m->active.p, nb, cudaMemcpyDeviceToHost, st));
  if (mu || prec) {
    std::vector<float4> w((size_t)nb * m->nw);
    BHM_CUDA(m, cudaMemcpyAsync(w.data(), m->W.p, 16 * w.size(), cudaMemcpyDeviceToHost, st));
    BHM_CUDA(m, cudaStreamSynchronize(st));
    for (size_t i = 0; i < w.size(); ++i) {
      if (mu) mu[i] = w[i].x;
      if (prec) prec[i] = w[i].y;
    }
  }
  BHM_CUDA(m, cudaStreamSynchronize(st));
  return KSDF_OK;
}

ksdf_status ksdf_bhm_tau(ksdf_bhm* m, double* tau) {
  if (!m || !tau) return KSDF_ERR_ARG;
  BHM_CUDA(m, cudaMemcpyAsync(tau, reinterpret_cast<char*>(m->state.p) + offsetof(BhmState, tau), 8,
                              cudaMemcpyDeviceToHost, m->stream));
  BHM_CUDA(m, cudaStreamSynchronize(m->stream));
  return KSDF_OK;
}

ksdf_status ksdf_bhm_sync_status(ksdf_bhm* m) {
  if (!m) return KSDF_ERR_ARG;
  BHM_CUDA(m, cudaStreamSynchronize(m->stream));
  uint32_t w = 0;
  BHM_CUDA(m, cudaMemcpy(&w, reinterpret_cast<char*>(m->state.p) + offsetof(BhmState, status), 4,
                         cudaMemcpyDeviceToHost));
  if (w) {
    const uint32_t z = 0;
    BHM_CUDA(m, cudaMemcpy(reinterpret_cast<char*>(m->state.p) + offsetof(BhmState, status), &z, 4,
                           cudaMemcpyHostToDevice));
  }
  if (w & ST_CAPACITY) return berr(m, KSDF_ERR_CAPACITY, "the block or marked-block capacity was exceeded");
  if (w & ST_NONFINITE) return berr(m, KSDF_ERR_NONFINITE, "NaN/Inf or out-of-range point(s)");
  return KSDF_OK;
}

const char* ksdf_bhm_last_error(const ksdf_bhm* m) { return m ? m->err.c_str() : "null map"; }

}  // extern "C"
