// ksdf_bhm.cu -- the Bayesian Hilbert map front-end of Kernel-SDF (Sec. IV-A, App. A, App. B) on one GPU: a device
// hash table of hinge blocks, the samples of each ray, the diagonal-covariance variational EM, the online threshold,
// prediction (log-odds, sign, gradient, probit occupancy) and the surface points of the marked marching cells.
// C ABI in include/ksdf_bhm.h, which also states the definitions every kernel here follows.
//
// Data layout in HBM (one map):
//   Wmp[slot * NW + i] float2 {mu, P} per weight (NW = n_h^3 + 1, the bias last): mean and precision of the map
//                     before the running update; A0, A1, B[slot * NW + i] floats: the update's accumulators,
//                     A = sum c(xi) phi^2 of odd (A0) and even (A1) EM rounds and B = sum (t - 1/2) phi
//   hash table        block key -> slot (open addressing, linear probing), 4x the block capacity
//   per block         packed key, active flag, the frame stamps of the touched / marked lists, its marked-cell index
//   masks             one bit per marching cell of each marked block ((n_h m)^3 bits)
//   samples           one 32-byte record per sample of the running update (lattice cell, 32-bit fraction, label)
// An update sets up each ray once (one thread per ray, binary64: its sample count and fixed-point step), then walks
// every ray twice (a warp per ray, 32 samples per step, integers only): once to count its samples, once, after a
// scan of the counts, to write them.  Each EM round is then one launch in which a warp takes 32 consecutive samples
// and, for each, splits the sample's candidate hinges (the offsets a point of that octant of the cell can reach,
// tabulated once per map) across its lanes: the M-step is a warp reduction and the E-step's atomics of one warp
// instruction fall on neighbouring weights.
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
  unsigned long long n_features;
  double lsum;
  double tau;
  uint32_t status;
  uint32_t pad3;
};

struct BhmDev {
  double o[3], h, p[3], up[3];
  long long Up[3];          // rint(2^32 u_p): the sensor's lattice coordinate in 2^-32 fixed point
  double fstep, fgap;
  double tau_a, tau_b;      // tau <- tau_a tau + tau_b sum_k l(x_k)
  double inv_m;             // 1 / march_sub (exact: a power of two)
  float gh2, g2h;           // gamma h^2 and -2 gamma h (binary32)
  float prior_prec, xi0, beta;
  long long r2q;
  int nh, nw, msub, cdim, mask_words;
  int frame, max_blocks, max_marked;
  int bias, rw;
  uint64_t hcap;
  uint64_t* hkeys;
  int32_t* hvals;
  uint64_t* bkey;
  uint8_t* active;
  int32_t *stamp_touch, *stamp_mark, *mark_idx;
  int32_t *new_list, *touched, *marked;
  float2* Wmp;
  float *A0, *A1, *Bacc;
  // candidate hinge offsets (dz + 8) << 16 | (dy + 8) << 8 | (dx + 8), z-major, per octant of the fraction (the
  // offsets within reach of that half-cell sub-cube): 8 tables of ostride entries, kNoCand padded
  const int32_t* ocand;
  int ostride;           // entries per octant table, a multiple of 32
  uint32_t* masks;
  BhmState* st;
};

struct __align__(16) Sample {
  int g[3];        // floor of the lattice coordinate
  uint32_t fq[3];  // fraction u - floor(u) as floor(2^32 (u - floor(u)))
  int t;           // label: 1 hit, 0 free
  int pad;
};

// per-ray set-up of the walk (binary64 once per ray, one thread each): the free-sample count, the fixed-point
// step, and the hit's own sample record (t = -1: the hit was invalid and the ray has no samples)
struct __align__(16) RayInfo {
  long long D[3];
  long long jmax;
  Sample hit;
};

constexpr int kMaxRounds = 7;  // candidate rounds of 32 lanes: (2 r + 2)^3 <= 216 offsets for r <= 2
constexpr int kNoCand = -1;

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
    const float2 r = d.Wmp[idx];
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
    const float2 r = d.Wmp[b];
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
      const int64_t i = (int64_t)id * d.nw + k;
      d.Wmp[i] = make_float2(0.f, d.prior_prec);
      d.A0[i] = 0.f;
      d.A1[i] = 0.f;
      d.Bacc[i] = 0.f;
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
  st->n_features = 0ull;
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

__device__ __forceinline__ Sample make_sample(const double u[3], int t) {
  Sample sm;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double fl = floor(u[a]);
    sm.g[a] = (int)fl;
    sm.fq[a] = (uint32_t)__dmul_rn(__dsub_rn(u[a], fl), 4294967296.0);  // exact scaling, truncation = floor
  }
  sm.t = t;
  sm.pad = 0;
  return sm;
}

__global__ void k_bhm_rays(BhmDev d, const double* __restrict__ hits, int64_t R, RayInfo* __restrict__ ri) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  RayInfo o;
  o.D[0] = o.D[1] = o.D[2] = 0;
  o.jmax = 0;
  double ux[3];
  if (!hit_lattice(d, hits, r, ux)) {
    o.hit.t = -1;
    ri[r] = o;
    return;
  }
  const double dx = __dsub_rn(hits[3 * r], d.p[0]), dy = __dsub_rn(hits[3 * r + 1], d.p[1]),
               dz = __dsub_rn(hits[3 * r + 2], d.p[2]);
  const double L = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
  if (L > 0.0) {
    const double t = floor(__ddiv_rn(__dsub_rn(L, d.fgap), d.fstep));
    o.jmax = t > 0.0 ? (long long)t : 0;
  }
  // free samples in 2^-32 fixed point: U_j = U_p + j D, D = rint((U_x - U_p) sigma), exact in integers
  if (o.jmax > 0) {
    const double sig = __ddiv_rn(d.fstep, L);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long Ux = __double2ll_rn(__dmul_rn(ux[a], 4294967296.0));
      o.D[a] = __double2ll_rn(__dmul_rn((double)(Ux - d.Up[a]), sig));
    }
  }
  o.hit = make_sample(ux, 1);
  ri[r] = o;
}

// The samples of every ray, a warp per ray: lanes take 32 consecutive free samples U_j = U_p + j D (lattice
// coordinates in 2^-32 fixed point, exact integer steps) at a time, the lowest lane of each group of lanes in the
// same block looks the block up, and the samples in active blocks are kept in j order; then the hit.  COUNT:
// cnt[r] = the ray's sample count; otherwise the samples are written from off[r] on.
template <bool COUNT>
__global__ void __launch_bounds__(kT) k_bhm_walk(BhmDev d, const RayInfo* __restrict__ ri, int64_t R, int64_t* cnt,
                                                 const int64_t* __restrict__ off, Sample* __restrict__ smp) {
  constexpr unsigned FULL = 0xffffffffu;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= R) return;  // whole warps
  const long long jmax = ri[r].jmax;
  const int hit_t = ri[r].hit.t;
  if (hit_t < 0) {
    if (COUNT && lane == 0) cnt[r] = 0;
    return;
  }
  const long long D[3] = {ri[r].D[0], ri[r].D[1], ri[r].D[2]};
  int64_t k = COUNT ? 0 : off[r];
  const unsigned lt = (1u << lane) - 1u;
  for (long long jb = 1; jb <= jmax; jb += 32) {
    const long long j = jb + lane;
    const bool valid = j <= jmax;
    long long U[3] = {0, 0, 0};
    uint64_t key = ~0ull;
    int b[3] = {0, 0, 0};
    if (valid) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        U[a] = d.Up[a] + j * D[a];
        b[a] = fdiv((int)(U[a] >> 32), d.nh);
      }
      key = pack_key(b[0], b[1], b[2]);
    }
    const unsigned grp = __match_any_sync(FULL, key);
    const int leader = __ffs(grp) - 1;
    int act = 0;
    if (valid && lane == leader) {
      const int sl = find_block(d, b[0], b[1], b[2]);
      act = sl >= 0 && d.active[sl];
    }
    act = __shfl_sync(FULL, act, leader);
    const bool keep = valid && act;
    const unsigned bal = __ballot_sync(FULL, keep);
    if (!COUNT && keep) {
      Sample sm;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        sm.g[a] = (int)(U[a] >> 32);
        sm.fq[a] = (uint32_t)(U[a] & 0xffffffffLL);
      }
      sm.t = 0;
      sm.pad = 0;
      smp[k + __popc(bal & lt)] = sm;
    }
    k += __popc(bal);
  }
  if (lane == 0) {
    if (!COUNT) smp[k] = ri[r].hit;
    if (COUNT) cnt[r] = k + 1;
  }
}

// One EM round over the update's samples, a warp per 32 consecutive samples.  FIRST: xi = xi_init, accumulates B
// and A into A0 (and builds the touched-block list).  Otherwise: the M-step of each sample from the previous
// round's posterior (its A in src: 0 = A0, 1 = A1), then the E-step statistic c(xi) phi^2 into dst.
template <bool FIRST>
__global__ void __launch_bounds__(kT) k_bhm_em(BhmDev d, const Sample* __restrict__ smp,
                                               const unsigned long long* __restrict__ n_dev, int src, int dst) {
  constexpr unsigned FULL = 0xffffffffu;
  const int64_t N = (int64_t)*n_dev;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nh = d.nh, nw = d.nw, RW = d.rw;
  // the candidate offsets of each octant of the fraction (a sample's octant is the top bit of each fraction)
  __shared__ int s_cand[8 * kMaxRounds * 32];
  for (int i = threadIdx.x; i < 8 * d.ostride; i += blockDim.x) s_cand[i] = d.ocand[i];
  __syncthreads();
  const int nrounds = d.ostride / 32;
  const float* Asrc = src ? d.A1 : d.A0;
  float* Adst = dst ? d.A1 : d.A0;
  int wlo[3] = {INT_MIN, INT_MIN, INT_MIN};
  int myslot = -1;  // lanes 0..7: slot of window block lo + (lane & 1, lane >> 1 & 1, lane >> 2)
  unsigned long long nfeat = 0;
  for (int64_t base = gw * 32; base < N; base += nwarps * 32) {
    Sample my = {};
    if (base + lane < N) my = smp[base + lane];
    const int nv = (int)(N - base < 32 ? N - base : 32);
    for (int s = 0; s < nv; ++s) {
      int g[3], bse[3], lo[3], q[3];
      float f[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        g[a] = __shfl_sync(FULL, my.g[a], s);
        const uint32_t fq = __shfl_sync(FULL, my.fq[a], s);
        q[a] = (int)(fq >> 12);
        f[a] = (float)fq * 2.3283064365386963e-10f;  // 2^-32
        lo[a] = fdiv(g[a] - RW, nh);
        bse[a] = g[a] - nh * lo[a];
      }
      const float tb = (float)__shfl_sync(FULL, my.t, s) - 0.5f;
      const int* oc = s_cand + (((q[2] >> 19) << 2) | ((q[1] >> 19) << 1) | (q[0] >> 19)) * d.ostride;
      if (lo[0] != wlo[0] || lo[1] != wlo[1] || lo[2] != wlo[2]) {
        wlo[0] = lo[0];
        wlo[1] = lo[1];
        wlo[2] = lo[2];
        if (lane < 8) {
          myslot = find_block(d, lo[0] + (lane & 1), lo[1] + ((lane >> 1) & 1), lo[2] + (lane >> 2));
          if (FIRST && myslot >= 0 && d.stamp_touch[myslot] != d.frame) {
            if (atomicExch(&d.stamp_touch[myslot], d.frame) != d.frame)
              d.touched[atomicAdd(&d.st->n_touched, 1)] = myslot;
          }
        }
      }
      const int bsl = __shfl_sync(FULL, myslot, (bse[2] >= nh) * 4 + (bse[1] >= nh) * 2 + (bse[0] >= nh));
      const int bidx = (d.bias && bsl >= 0) ? bsl * nw + nw - 1 : -1;
      float phr[kMaxRounds];
      int idr[kMaxRounds];
      float vs = 0.f, ms = 0.f;
#pragma unroll
      for (int r = 0; r < kMaxRounds; ++r) {
        idr[r] = -1;
        phr[r] = 0.f;
        if (r >= nrounds) continue;  // uniform across the warp
        const int cd = oc[r * 32 + lane];
        const int ox = (cd & 255) - 8, oy = ((cd >> 8) & 255) - 8, oz = ((cd >> 16) & 255) - 8;
        // |fraction - offset|^2 in units of 2^-40, each term one 32 x 32 -> 64-bit product
        const int tx = q[0] - ox * (1 << kQ), ty = q[1] - oy * (1 << kQ), tz = q[2] - oz * (1 << kQ);
        const long long D = (long long)tx * tx + (long long)ty * ty + (long long)tz * tz;
        const int lx = bse[0] + ox, ly = bse[1] + oy, lz = bse[2] + oz;
        const int sl = __shfl_sync(FULL, myslot, (lz >= nh) * 4 + (ly >= nh) * 2 + (lx >= nh));
        const bool ok = cd != kNoCand && D <= d.r2q && sl >= 0;
        const float fx = f[0] - (float)ox, fy = f[1] - (float)oy, fz = f[2] - (float)oz;
        const float phi = __expf(-d.gh2 * (fx * fx + fy * fy + fz * fz));
        const int idx = sl * nw + ((lz - (lz >= nh ? nh : 0)) * nh + (ly - (ly >= nh ? nh : 0))) * nh +
                        (lx - (lx >= nh ? nh : 0));
        phr[r] = phi;
        idr[r] = ok ? idx : -1;
        if (!FIRST && ok) {
          const float2 w = d.Wmp[idx];
          const float inv = __fdividef(1.0f, w.y + Asrc[idx]);
          const float mu = fmaf(w.y, w.x, d.Bacc[idx]) * inv;
          vs = fmaf(phi * phi, inv, vs);
          ms = fmaf(mu, phi, ms);
        }
        if (FIRST) nfeat += (unsigned long long)__popc(__ballot_sync(FULL, ok));
      }
      float xi = d.xi0;
      if (!FIRST) {
        if (lane == 0 && bidx >= 0) {
          const float2 w = d.Wmp[bidx];
          const float P = w.y + Asrc[bidx];
          vs += 1.0f / P;
          ms += fmaf(w.y, w.x, d.Bacc[bidx]) / P;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          vs += __shfl_xor_sync(FULL, vs, o);
          ms += __shfl_xor_sync(FULL, ms, o);
        }
        xi = sqrtf(fmaf(ms, ms, vs));
      }
      const float c = jj_coef(xi);
#pragma unroll
      for (int r = 0; r < kMaxRounds; ++r) {
        if (idr[r] >= 0) {
          atomicAdd(&Adst[idr[r]], c * phr[r] * phr[r]);
          if (FIRST) atomicAdd(&d.Bacc[idr[r]], tb * phr[r]);
        }
      }
      if (lane == 0 && bidx >= 0) {
        atomicAdd(&Adst[bidx], c);
        if (FIRST) atomicAdd(&d.Bacc[bidx], tb);
      }
    }
  }
  if (FIRST && lane == 0 && nfeat) atomicAdd(&d.st->n_features, nfeat);
}

// zero one accumulator of every touched block (before EM rounds three and four, which reuse them)
__global__ void k_bhm_zero_acc(BhmDev d, int which) {
  const int n = d.st->n_touched;
  for (int b = blockIdx.x; b < n; b += gridDim.x) {
    const int64_t base = (int64_t)d.touched[b] * d.nw;
    float* A = which ? d.A1 : d.A0;
    for (int k = threadIdx.x; k < d.nw; k += blockDim.x) A[base + k] = 0.f;
  }
}

// the last E-step's posterior becomes the map: P = P_prev + A, mu = (P_prev mu_prev + B) / P; accumulators cleared
__global__ void k_bhm_commit(BhmDev d, int last) {
  const int n = d.st->n_touched;
  for (int b = blockIdx.x; b < n; b += gridDim.x) {
    const int64_t base = (int64_t)d.touched[b] * d.nw;
    for (int k = threadIdx.x; k < d.nw; k += blockDim.x) {
      const int64_t i = base + k;
      const float a = last ? d.A1[i] : d.A0[i];
      if (a != 0.f) {
        const float2 w = d.Wmp[i];
        const float P = w.y + a;
        d.Wmp[i] = make_float2(fmaf(w.y, w.x, d.Bacc[i]) / P, P);
      }
      d.A0[i] = 0.f;
      d.A1[i] = 0.f;
      d.Bacc[i] = 0.f;
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

// One CTA per marked block.  Shared memory: the means of every hinge the block's nodes can reach ((n_h + 2 RW + 2)^3,
// hinge local coordinate + RW), the biases and mark indices of the 27 blocks around, the per-axis factors of a node
// (node fractions are multiples of 1/m, so exp(-gamma h^2 (k/m - delta)^2) and the fixed-point distances are
// tabulated per k), the processed-edge bits of the owned nodes and the log-odds of the (C + 1)^3 nodes they use.
struct MarchSmem {
  int nbr_mark[27];
  float nbr_bias[27];
};

template <int RW>
__device__ __forceinline__ float node_logodds(const BhmDev& d, const MarchSmem& sm, const float* mus, const float* te,
                                              const long long* tq, int HN, const int gl[3], const int kk[3]) {
  constexpr int NO = 2 * RW + 2;
  const int m = d.msub, nh = d.nh;
  float acc = 0.f;
#pragma unroll 1
  for (int iz = 0; iz < NO; ++iz) {
    const long long dz = tq[kk[2] * NO + iz];
    if (dz > d.r2q) continue;
    const float ez = te[kk[2] * NO + iz];
    const int hz = gl[2] + iz;  // (g0 + delta) + RW with delta = iz - RW
#pragma unroll 1
    for (int iy = 0; iy < NO; ++iy) {
      const long long dzy = dz + tq[kk[1] * NO + iy];
      if (dzy > d.r2q) continue;
      const float ezy = ez * te[kk[1] * NO + iy];
      const float* row = mus + ((hz * HN) + gl[1] + iy) * HN + gl[0];
#pragma unroll
      for (int ix = 0; ix < NO; ++ix) {
        if (dzy + tq[kk[0] * NO + ix] > d.r2q) continue;
        acc = fmaf(row[ix], ezy * te[kk[0] * NO + ix], acc);
      }
    }
  }
  (void)m;
  // bias of the node's own block (its g0 lies in the block or on its upper faces)
  const int bsel = ((gl[2] >= nh) + 1) * 9 + ((gl[1] >= nh) + 1) * 3 + ((gl[0] >= nh) + 1);
  return acc + sm.nbr_bias[bsel];
}

template <int RW>
__global__ void __launch_bounds__(kT) k_bhm_march(BhmDev d, MarchOut mo) {
  constexpr int NO = 2 * RW + 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  MarchSmem& sm = *reinterpret_cast<MarchSmem*>(smraw);
  const int nh = d.nh, C = d.cdim, m = d.msub, HN = nh + 2 * RW + 2, C1 = C + 1;
  long long* tq = reinterpret_cast<long long*>(smraw + sizeof(MarchSmem) + (8 - sizeof(MarchSmem) % 8) % 8);
  float* te = reinterpret_cast<float*>(tq + m * NO);
  float* mus = te + m * NO;
  float* lv = mus + HN * HN * HN;
  uint8_t* doit = reinterpret_cast<uint8_t*>(lv + C1 * C1 * C1);
  const int nmk = min(d.st->n_marked, d.max_marked);
  const double tau = d.st->tau;
  const float tauf = (float)tau;
  (void)tauf;
  // per-axis node factors: fraction k / m, offsets delta = i - RW
  for (int i = threadIdx.x; i < m * NO; i += blockDim.x) {
    const int k = i / NO, delta = i % NO - RW;
    const long long q = ((long long)k << kQ) / m;  // exact: m is a power of two
    const long long t = q - ((long long)delta << kQ);
    tq[i] = t * t;
    const float df = (float)k / (float)m - (float)delta;
    te[i] = expf(-d.gh2 * df * df);
  }
  for (int mb = blockIdx.x; mb < nmk; mb += gridDim.x) {
    const int slot = d.marked[mb];
    int bx, by, bz;
    unpack_key(d.bkey[slot], bx, by, bz);
    __syncthreads();
    __shared__ int nslot[27];
    if (threadIdx.x < 27) {
      const int s = find_block(d, bx + threadIdx.x % 3 - 1, by + (threadIdx.x / 3) % 3 - 1, bz + threadIdx.x / 9 - 1);
      nslot[threadIdx.x] = s;
      sm.nbr_mark[threadIdx.x] = (s >= 0 && d.stamp_mark[s] == d.frame) ? d.mark_idx[s] : -1;
      sm.nbr_bias[threadIdx.x] = (s >= 0 && d.bias) ? d.Wmp[(int64_t)s * d.nw + d.nw - 1].x : 0.f;
    }
    __syncthreads();
    // means of the reachable hinges: local hinge coordinate g in [-RW, nh + RW + 1], stored at g + RW
    for (int i = threadIdx.x; i < HN * HN * HN; i += blockDim.x) {
      const int hx = i % HN, hy = (i / HN) % HN, hz = i / (HN * HN);
      const int g[3] = {hx - RW, hy - RW, hz - RW};
      int o[3], loc[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        o[a] = g[a] < 0 ? -1 : (g[a] >= nh ? 1 : 0);
        loc[a] = g[a] - nh * o[a];
      }
      const int s = nslot[(o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1)];
      mus[i] = s >= 0 ? d.Wmp[(int64_t)s * d.nw + (loc[2] * nh + loc[1]) * nh + loc[0]].x : 0.f;
    }
    // processed-edge bits of the owned nodes: edge (n, a) when one of its four adjacent cells is marked
    auto marked = [&](int cx, int cy, int cz) -> bool {
      const int k = sm.nbr_mark[(cz < 0 ? 0 : 1) * 9 + (cy < 0 ? 0 : 1) * 3 + (cx < 0 ? 0 : 1)];
      if (k < 0) return false;
      const int lx = cx < 0 ? C - 1 : cx, ly = cy < 0 ? C - 1 : cy, lz = cz < 0 ? C - 1 : cz;
      const int bitn = (lz * C + ly) * C + lx;
      return (d.masks[(int64_t)k * d.mask_words + (bitn >> 5)] >> (bitn & 31)) & 1u;
    };
    for (int n = threadIdx.x; n < C * C * C; n += blockDim.x) {
      const int l3[3] = {n % C, (n / C) % C, n / (C * C)};
      int bits = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
        bool mk = false;
#pragma unroll
        for (int ib = 0; ib < 2; ++ib)
#pragma unroll
          for (int ic = 0; ic < 2; ++ic) {
            int cc[3] = {l3[0], l3[1], l3[2]};
            cc[b] -= ib;
            cc[c] -= ic;
            mk = mk || marked(cc[0], cc[1], cc[2]);
          }
        bits |= mk ? (1 << a) : 0;
      }
      doit[n] = (uint8_t)bits;
    }
    __syncthreads();
    // log-odds of every node an edge uses: n itself, and n + e_a for its processed axes
    for (int n = threadIdx.x; n < C1 * C1 * C1; n += blockDim.x) {
      const int l3[3] = {n % C1, (n / C1) % C1, n / (C1 * C1)};
      bool need = l3[0] < C && l3[1] < C && l3[2] < C && doit[(l3[2] * C + l3[1]) * C + l3[0]];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (need || l3[a] == 0) continue;
        int p3[3] = {l3[0], l3[1], l3[2]};
        p3[a] -= 1;
        if (p3[0] < C && p3[1] < C && p3[2] < C && (doit[(p3[2] * C + p3[1]) * C + p3[0]] >> a & 1)) need = true;
      }
      if (!need) continue;
      int gl[3], kk[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        gl[a] = l3[a] / m;  // local g0 of the node (l3 >= 0)
        kk[a] = l3[a] - m * gl[a];
      }
      lv[n] = node_logodds<RW>(d, sm, mus, te, tq, HN, gl, kk);
    }
    __syncthreads();
    // edges: crossings of the level set, the point at the linear interpolation, its variance and normal
    for (int n = threadIdx.x; n < C * C * C; n += blockDim.x) {
      const int bits = doit[n];
      if (!bits) continue;
      const int l3[3] = {n % C, (n / C) % C, n / (C * C)};
      const int nu[3] = {bx * C + l3[0], by * C + l3[1], bz * C + l3[2]};
      const float la = lv[(l3[2] * C1 + l3[1]) * C1 + l3[0]];
#pragma unroll 1
      for (int a = 0; a < 3; ++a) {
        if (!(bits >> a & 1)) continue;
        int p3[3] = {l3[0], l3[1], l3[2]};
        p3[a] += 1;
        const float lb = lv[(p3[2] * C1 + p3[1]) * C1 + p3[0]];
        if (((double)la >= tau) == ((double)lb >= tau)) continue;
        const double t = (tau - (double)la) / ((double)lb - (double)la);
        double ui[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) ui[e] = __dmul_rn((double)nu[e], d.inv_m);
        ui[a] = __dmul_rn(__dadd_rn((double)nu[a], t), d.inv_m);
        // the point's features: the two other axes keep the node's tabulated factors, axis a its own
        const double fl = floor(ui[a]);
        const int ga = (int)fl;
        const double fr = __dsub_rn(ui[a], fl);
        const long long qa = (long long)__dmul_rn(fr, (double)(1 << kQ));
        const float fa = (float)fr;
        float ea[NO], da[NO];
        long long qd[NO];
#pragma unroll
        for (int i = 0; i < NO; ++i) {
          const long long tt = qa - ((long long)(i - RW) << kQ);
          qd[i] = tt * tt;
          da[i] = fa - (float)(i - RW);
          ea[i] = expf(-d.gh2 * da[i] * da[i]);
        }
        int gl[3], kk[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          gl[e] = l3[e] / m;
          kk[e] = l3[e] - m * gl[e];
        }
        gl[a] = ga - (a == 0 ? bx : (a == 1 ? by : bz)) * nh;
        float sl = 0.f, g3[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
        for (int iz = 0; iz < NO; ++iz) {
          const long long dz = a == 2 ? qd[iz] : tq[kk[2] * NO + iz];
          if (dz > d.r2q) continue;
          const float ez = a == 2 ? ea[iz] : te[kk[2] * NO + iz];
          const float fz = a == 2 ? da[iz] : (float)kk[2] / (float)m - (float)(iz - RW);
#pragma unroll 1
          for (int iy = 0; iy < NO; ++iy) {
            const long long dzy = dz + (a == 1 ? qd[iy] : tq[kk[1] * NO + iy]);
            if (dzy > d.r2q) continue;
            const float ezy = ez * (a == 1 ? ea[iy] : te[kk[1] * NO + iy]);
            const float fy = a == 1 ? da[iy] : (float)kk[1] / (float)m - (float)(iy - RW);
            const float* row = mus + (((gl[2] + iz) * HN) + gl[1] + iy) * HN + gl[0];
#pragma unroll
            for (int ix = 0; ix < NO; ++ix) {
              if (dzy + (a == 0 ? qd[ix] : tq[kk[0] * NO + ix]) > d.r2q) continue;
              const float fx = a == 0 ? da[ix] : (float)kk[0] / (float)m - (float)(ix - RW);
              const float mp = row[ix] * (ezy * (a == 0 ? ea[ix] : te[kk[0] * NO + ix]));
              sl += mp;
              g3[0] = fmaf(mp, fx, g3[0]);
              g3[1] = fmaf(mp, fy, g3[1]);
              g3[2] = fmaf(mp, fz, g3[2]);
            }
          }
        }
        sl += sm.nbr_bias[((gl[2] >= nh) + 1) * 9 + ((gl[1] >= nh) + 1) * 3 + ((gl[0] >= nh) + 1)];
        const float gx = d.g2h * g3[0], gy = d.g2h * g3[1], gz = d.g2h * g3[2];
        const float g2 = gx * gx + gy * gy + gz * gz;
        if (!(g2 > 0.f)) continue;
        const int64_t k = atomicAdd(&d.st->n_out, 1);
        if (k >= mo.cap) continue;
        const float dl = (float)(tau - (double)sl);
        const float ig = rsqrtf(g2);
        mo.key[k] = ((uint64_t)(nu[2] + kEdgeBias) << 42) | ((uint64_t)(nu[1] + kEdgeBias) << 22) |
                    ((uint64_t)(nu[0] + kEdgeBias) << 2) | (uint64_t)a;
        mo.val[k] = (uint32_t)k;
#pragma unroll
        for (int e = 0; e < 3; ++e) mo.x[3 * k + e] = __dadd_rn(d.o[e], __dmul_rn(ui[e], d.h));
        mo.var[k] = d.beta * dl * dl / g2;
        mo.nrm[3 * k] = -gx * ig;
        mo.nrm[3 * k + 1] = -gy * ig;
        mo.nrm[3 * k + 2] = -gz * ig;
      }
    }
  }
}

size_t march_smem(int nh, int rw, int m, int C) {
  const int NO = 2 * rw + 2, HN = nh + 2 * rw + 2, C1 = C + 1;
  size_t b = sizeof(MarchSmem);
  b += (8 - b % 8) % 8;
  b += (size_t)m * NO * 8 + (size_t)m * NO * 4 + (size_t)HN * HN * HN * 4 + (size_t)C1 * C1 * C1 * 4 + (size_t)C * C * C;
  return b;
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

// Prediction, a warp per 32 points: each lane sets up one point (binary64 lattice coordinate, fixed-point and
// binary32 fraction), then the warp takes the points one at a time, its lanes splitting the point's candidate
// offsets (the octant table of the EM); sums by warp reduction; each lane writes its own point's outputs.
template <bool GV>
__global__ void __launch_bounds__(kT) k_bhm_query(BhmDev d, const float* __restrict__ xq, int64_t Q, uint32_t mask,
                                                  float* lo_out, int8_t* sg, float* gr, float* pr) {
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ int s_cand[8 * kMaxRounds * 32];
  for (int i = threadIdx.x; i < 8 * d.ostride; i += blockDim.x) s_cand[i] = d.ocand[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nh = d.nh, nw = d.nw, RW = d.rw, nrounds = d.ostride / 32;
  const double tau = d.st->tau;
  int wlo[3] = {INT_MIN, INT_MIN, INT_MIN};
  int myslot = -1;
  for (int64_t base = gw * 32; base < Q; base += nwarps * 32) {
    const int64_t i = base + lane;
    int g[3] = {0, 0, 0}, q[3] = {0, 0, 0};
    float f[3] = {0.f, 0.f, 0.f};
    bool ok = i < Q;
    if (ok) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double u = lat((double)xq[3 * i + a], d.o[a], d.h);
        ok = ok && lat_ok(u);
        const double fl = ok ? floor(u) : 0.0;
        const double fr = ok ? __dsub_rn(u, fl) : 0.0;
        g[a] = (int)fl;
        q[a] = (int)__dmul_rn(fr, (double)(1 << kQ));
        f[a] = (float)fr;
      }
      if (!ok) set_status(d.st, ST_NONFINITE);
    }
    float my_l = 0.f, my_v = 0.f, my_g[3] = {0.f, 0.f, 0.f};
    const int nv = (int)(Q - base < 32 ? Q - base : 32);
    for (int s = 0; s < nv; ++s) {
      if (!__shfl_sync(FULL, (int)ok, s)) continue;  // uniform
      int gg[3], qq[3], bse[3], lo[3];
      float ff[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        gg[a] = __shfl_sync(FULL, g[a], s);
        qq[a] = __shfl_sync(FULL, q[a], s);
        ff[a] = __shfl_sync(FULL, f[a], s);
        lo[a] = fdiv(gg[a] - RW, nh);
        bse[a] = gg[a] - nh * lo[a];
      }
      if (lo[0] != wlo[0] || lo[1] != wlo[1] || lo[2] != wlo[2]) {
        wlo[0] = lo[0];
        wlo[1] = lo[1];
        wlo[2] = lo[2];
        if (lane < 8) myslot = find_block(d, lo[0] + (lane & 1), lo[1] + ((lane >> 1) & 1), lo[2] + (lane >> 2));
      }
      const int* oc = s_cand + (((qq[2] >> 19) << 2) | ((qq[1] >> 19) << 1) | (qq[0] >> 19)) * d.ostride;
      float sl = 0.f, sv = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
      for (int r = 0; r < kMaxRounds; ++r) {
        if (r >= nrounds) continue;  // uniform
        const int cd = oc[r * 32 + lane];
        const int ox = (cd & 255) - 8, oy = ((cd >> 8) & 255) - 8, oz = ((cd >> 16) & 255) - 8;
        const int tx = qq[0] - ox * (1 << kQ), ty = qq[1] - oy * (1 << kQ), tz = qq[2] - oz * (1 << kQ);
        const long long D = (long long)tx * tx + (long long)ty * ty + (long long)tz * tz;
        const int lx = bse[0] + ox, ly = bse[1] + oy, lz = bse[2] + oz;
        const int slt = __shfl_sync(FULL, myslot, (lz >= nh) * 4 + (ly >= nh) * 2 + (lx >= nh));
        if (cd == kNoCand || D > d.r2q || slt < 0) continue;
        const float fx = ff[0] - (float)ox, fy = ff[1] - (float)oy, fz = ff[2] - (float)oz;
        const float phi = expf(-d.gh2 * (fx * fx + fy * fy + fz * fz));
        const int idx = slt * nw + ((lz - (lz >= nh ? nh : 0)) * nh + (ly - (ly >= nh ? nh : 0))) * nh +
                        (lx - (lx >= nh ? nh : 0));
        const float2 w = d.Wmp[idx];
        const float mp = w.x * phi;
        sl += mp;
        if (GV) {
          sx = fmaf(mp, fx, sx);
          sy = fmaf(mp, fy, sy);
          sz = fmaf(mp, fz, sz);
          sv = fmaf(phi * phi, 1.0f / w.y, sv);
        }
      }
      const int bsl = __shfl_sync(FULL, myslot, (bse[2] >= nh) * 4 + (bse[1] >= nh) * 2 + (bse[0] >= nh));
      if (lane == 0 && d.bias && bsl >= 0) {
        const float2 w = d.Wmp[(int64_t)bsl * nw + nw - 1];
        sl += w.x;
        if (GV) sv += 1.0f / w.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sl += __shfl_xor_sync(FULL, sl, o);
        if (GV) {
          sv += __shfl_xor_sync(FULL, sv, o);
          sx += __shfl_xor_sync(FULL, sx, o);
          sy += __shfl_xor_sync(FULL, sy, o);
          sz += __shfl_xor_sync(FULL, sz, o);
        }
      }
      if (lane == s) {
        my_l = sl;
        my_v = sv;
        my_g[0] = d.g2h * sx;
        my_g[1] = d.g2h * sy;
        my_g[2] = d.g2h * sz;
      }
    }
    if (i < Q) {
      if (!ok) {
        my_l = my_v = __int_as_float(0x7fc00000);
        my_g[0] = my_g[1] = my_g[2] = my_l;
      }
      if (mask & KSDF_BHM_LOGODDS) lo_out[i] = my_l;
      if (mask & KSDF_BHM_SIGN) sg[i] = (!ok || (double)my_l < tau) ? (int8_t)1 : (int8_t)-1;
      if (mask & KSDF_BHM_GRAD) {
        gr[3 * i] = my_g[0];
        gr[3 * i + 1] = my_g[1];
        gr[3 * i + 2] = my_g[2];
      }
      if (mask & KSDF_BHM_PROB) pr[i] = 1.0f / (1.0f + expf(-my_l / sqrtf(1.0f + 0.39269908169872414f * my_v)));
    }
  }
}

// whether the last update's marks process edge `key`: one of its four adjacent cells is marked (a thread per key)
__global__ void k_bhm_edges_marked(BhmDev d, const uint64_t* __restrict__ keys, int64_t n, uint8_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = keys[i];
  const int a = (int)(k & 3ull);
  const int nu[3] = {(int)((k >> 2) & 0xFFFFFull) - (int)kEdgeBias, (int)((k >> 22) & 0xFFFFFull) - (int)kEdgeBias,
                     (int)((k >> 42) & 0xFFFFFull) - (int)kEdgeBias};
  uint8_t hit = 0;
  if (a < 3) {
    const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
    for (int ib = 0; ib < 2 && !hit; ++ib)
      for (int ic = 0; ic < 2 && !hit; ++ic) {
        int cc[3] = {nu[0], nu[1], nu[2]};
        cc[b] -= ib;
        cc[c] -= ic;
        const int bx = fdiv(cc[0], d.cdim), by = fdiv(cc[1], d.cdim), bz = fdiv(cc[2], d.cdim);
        const int s = find_block(d, bx, by, bz);
        if (s < 0 || d.stamp_mark[s] != d.frame) continue;
        const int mk = d.mark_idx[s];
        if (mk < 0) continue;
        const int bitn = ((cc[2] - bz * d.cdim) * d.cdim + (cc[1] - by * d.cdim)) * d.cdim + (cc[0] - bx * d.cdim);
        hit = (uint8_t)((d.masks[(int64_t)mk * d.mask_words + (bitn >> 5)] >> (bitn & 31)) & 1u);
      }
  }
  out[i] = hit;
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
  DevBuf hkeys, hvals, bkey, active, stamps, lists, Wmp, A0, A1, B, ocand, masks, state;
  DevBuf stage_hits, mkey, mval, mx, mvar, mnrm, sort_tmp, out_stage[4], q_stage[5];
  DevBuf smp, scnt, soff, scan_tmp, rays;
  int64_t mcap = 0, scap = 0;
  int ostride = 0;
  double up[3] = {0, 0, 0}, p_last[3] = {0, 0, 0};
  long long Up[3] = {0, 0, 0};
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
    d.Up[a] = m->Up[a];
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
  d.Wmp = ptr<float2>(m->Wmp);
  d.A0 = ptr<float>(m->A0);
  d.A1 = ptr<float>(m->A1);
  d.Bacc = ptr<float>(m->B);
  d.ocand = ptr<int32_t>(m->ocand);
  d.ostride = m->ostride;
  d.rw = m->rw;
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
            (p.bias_feature == 0 || p.bias_feature == 1) && max_blocks >= 1 && max_marked >= 0;
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
  if (cdim > 32) return KSDF_ERR_ARG;  // the march keeps (cdim + 1)^3 node values in shared memory
  const int64_t nw = (int64_t)p.block_hinges * p.block_hinges * p.block_hinges + 1;
  if (max_blocks * nw >= (1LL << 31)) return KSDF_ERR_ARG;  // weight indices are 32-bit
  const double rr2 = (double)r2q / 1099511627776.0 + 1e-9;
  // per octant of the fraction ([0, 1/2] or [1/2, 1] per axis): the offsets within reach of that sub-cube
  std::vector<int32_t> ocand[8];
  size_t omax = 0;
  for (int o = 0; o < 8; ++o) {
    for (int dz = -rw; dz <= rw + 1; ++dz)
      for (int dy = -rw; dy <= rw + 1; ++dy)
        for (int dx = -rw; dx <= rw + 1; ++dx) {
          const int dd[3] = {dx, dy, dz};
          double g2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            const double lo = 0.5 * ((o >> a) & 1), hi = lo + 0.5;
            const double gap = dd[a] < lo ? lo - dd[a] : (dd[a] > hi ? dd[a] - hi : 0.0);
            g2 += gap * gap;
          }
          if (g2 <= rr2) ocand[o].push_back(((dz + 8) << 16) | ((dy + 8) << 8) | (dx + 8));
        }
    omax = std::max(omax, ocand[o].size());
  }
  const int ostride = (int)((omax + 31) / 32 * 32);
  std::vector<int32_t> otab((size_t)8 * ostride, -1);
  for (int o = 0; o < 8; ++o) std::copy(ocand[o].begin(), ocand[o].end(), otab.begin() + (size_t)o * ostride);

  ksdf_bhm* m = new ksdf_bhm();
  m->p = p;
  m->stream = (cudaStream_t)stream;
  m->rw = rw;
  m->r2q = r2q;
  m->ostride = ostride;
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
  al(m->Wmp, 8 * (size_t)max_blocks * m->nw);
  al(m->A0, 4 * (size_t)max_blocks * m->nw);
  al(m->A1, 4 * (size_t)max_blocks * m->nw);
  al(m->B, 4 * (size_t)max_blocks * m->nw);
  al(m->ocand, 4 * (size_t)8 * ostride);
  al(m->masks, 4 * (size_t)m->max_marked * m->mask_words);
  al(m->state, sizeof(BhmState));
  if (e == cudaSuccess) e = cudaMemsetAsync(m->hkeys.p, 0xff, 8 * cap, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->hvals.p, 0xff, 4 * cap, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->state.p, 0, sizeof(BhmState), m->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->ocand.p, otab.data(), 4 * otab.size(), cudaMemcpyHostToDevice, m->stream);
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
  DevBuf* bufs[] = {&m->hkeys, &m->hvals, &m->bkey, &m->active, &m->stamps, &m->lists, &m->Wmp, &m->A0,
                    &m->A1, &m->B, &m->ocand, &m->masks, &m->state, &m->stage_hits, &m->mkey, &m->mval,
                    &m->mx, &m->mvar, &m->mnrm, &m->sort_tmp, &m->smp, &m->scnt, &m->soff, &m->scan_tmp,
                    &m->rays};
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
    m->Up[a] = std::llrint(u * 4294967296.0);  // round half to even
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
    // the samples: count per ray, scan, write (the count decides the buffer size: one synchronisation)
    BHM_CUDA(m, ensure(m->scnt, 8 * (size_t)R));
    BHM_CUDA(m, ensure(m->soff, 8 * (size_t)R));
    int64_t* cnt = ptr<int64_t>(m->scnt);
    int64_t* off = ptr<int64_t>(m->soff);
    BhmState* sdev = ptr<BhmState>(m->state);
    BHM_CUDA(m, ensure(m->rays, sizeof(RayInfo) * (size_t)R));
    RayInfo* ri = ptr<RayInfo>(m->rays);
    launch(k_bhm_rays, g, kT, 0, st, d, dh, R, ri);
    const unsigned gw = (unsigned)((R * 32 + kT - 1) / kT);  // a warp per ray
    launch(k_bhm_walk<true>, gw, kT, 0, st, d, (const RayInfo*)ri, R, cnt, (const int64_t*)nullptr, (Sample*)nullptr);
    BHM_CUDA(m, scan_i64(cnt, off, R, reinterpret_cast<int64_t*>(&sdev->n_samples), m->scan_tmp, st));
    unsigned long long ns = 0;
    BHM_CUDA(m, cudaMemcpyAsync(&ns, &sdev->n_samples, 8, cudaMemcpyDeviceToHost, st));
    BHM_CUDA(m, cudaStreamSynchronize(st));
    if ((int64_t)ns > m->scap) {
      const int64_t want = (int64_t)ns + ((int64_t)ns >> 3) + 1024;
      BHM_CUDA(m, ensure(m->smp, sizeof(Sample) * (size_t)want));
      m->scap = want;
    }
    Sample* smp = ptr<Sample>(m->smp);
    launch(k_bhm_walk<false>, gw, kT, 0, st, d, (const RayInfo*)ri, R, (int64_t*)nullptr, (const int64_t*)off, smp);
    const unsigned ge = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)ns + 255) / 256, 152 * 16));
    const int iters = m->p.em_iters;
    for (int it = 1; it <= iters; ++it) {
      const int dst = (it - 1) & 1, src = it >= 2 ? (it - 2) & 1 : 0;
      if (it >= 3) launch(k_bhm_zero_acc, kGridStride, kT, 0, st, d, dst);
      if (it == 1) launch(k_bhm_em<true>, ge, kT, 0, st, d, (const Sample*)smp, &sdev->n_samples, src, dst);
      else launch(k_bhm_em<false>, ge, kT, 0, st, d, (const Sample*)smp, &sdev->n_samples, src, dst);
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
    const size_t smb = march_smem(m->nh, m->rw, m->p.march_sub, m->cdim);
    switch (m->rw) {
      case 0:
        BHM_CUDA(m, cudaFuncSetAttribute(k_bhm_march<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb));
        launch(k_bhm_march<0>, kGridStride, kT, smb, st, d, mo);
        break;
      case 1:
        BHM_CUDA(m, cudaFuncSetAttribute(k_bhm_march<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb));
        launch(k_bhm_march<1>, kGridStride, kT, smb, st, d, mo);
        break;
      default:
        BHM_CUDA(m, cudaFuncSetAttribute(k_bhm_march<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb));
        launch(k_bhm_march<2>, kGridStride, kT, smb, st, d, mo);
        break;
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
  const unsigned gq = (unsigned)std::max<int64_t>(1, std::min<int64_t>((Q * 32 + kT - 1) / kT / 32 + 1, 152 * 16));
  if (out_mask & (KSDF_BHM_GRAD | KSDF_BHM_PROB))
    launch(k_bhm_query<true>, gq, kT, 0, st, d, dq, Q, out_mask & 15u, (float*)dv[0], (int8_t*)dv[1], (float*)dv[2],
           (float*)dv[3]);
  else
    launch(k_bhm_query<false>, gq, kT, 0, st, d, dq, Q, out_mask & 15u, (float*)dv[0], (int8_t*)dv[1],
           (float*)dv[2], (float*)dv[3]);
  BHM_CUDA(m, cudaGetLastError());
  for (int i = 0; i < 4; ++i)
    if (outs[i] && dv[i] != outs[i])
      BHM_CUDA(m, cudaMemcpyAsync(outs[i], dv[i], bytes[i], cudaMemcpyDeviceToHost, st));
  if (host_out) BHM_CUDA(m, cudaStreamSynchronize(st));
  return KSDF_OK;
}

ksdf_status ksdf_bhm_edges_marked(ksdf_bhm* m, const uint64_t* keys, int64_t n, uint8_t* out) {
  if (!m) return KSDF_ERR_ARG;
  if (n < 0 || (n > 0 && (!keys || !out))) return berr(m, KSDF_ERR_ARG, "ksdf_bhm_edges_marked: bad n or NULL array");
  if (n == 0) return KSDF_OK;
  cudaStream_t st = m->stream;
  if (m->frame < 0) {  // nothing marked yet
    if (dev_ptr(out)) BHM_CUDA(m, cudaMemsetAsync(out, 0, (size_t)n, st));
    else memset(out, 0, (size_t)n);
    return KSDF_OK;
  }
  const uint64_t* dk = keys;
  if (!dev_ptr(keys)) {
    BHM_CUDA(m, ensure(m->q_stage[0], 8 * (size_t)n));
    BHM_CUDA(m, cudaMemcpyAsync(m->q_stage[0].p, keys, 8 * (size_t)n, cudaMemcpyHostToDevice, st));
    dk = ptr<uint64_t>(m->q_stage[0]);
  }
  uint8_t* dout = out;
  const bool host_out = !dev_ptr(out);
  if (host_out) {
    BHM_CUDA(m, ensure(m->q_stage[1], (size_t)n));
    dout = ptr<uint8_t>(m->q_stage[1]);
  }
  launch(k_bhm_edges_marked, nblk(n), kT, 0, st, dev_view(m), dk, n, dout);
  BHM_CUDA(m, cudaGetLastError());
  if (host_out) {
    BHM_CUDA(m, cudaMemcpyAsync(out, dout, (size_t)n, cudaMemcpyDeviceToHost, st));
    BHM_CUDA(m, cudaStreamSynchronize(st));
  }
  return KSDF_OK;
}

ksdf_status ksdf_bhm_size(ksdf_bhm* m, int64_t* n_blocks, int64_t* n_samples_last, int64_t* n_features_last) {
  if (!m) return KSDF_ERR_ARG;
  BhmState s;
  BHM_CUDA(m, cudaMemcpyAsync(&s, m->state.p, sizeof(s), cudaMemcpyDeviceToHost, m->stream));
  BHM_CUDA(m, cudaStreamSynchronize(m->stream));
  if (n_blocks) *n_blocks = s.n_blocks;
  if (n_samples_last) *n_samples_last = (int64_t)s.n_samples;
  if (n_features_last) *n_features_last = (int64_t)s.n_features;
  return KSDF_OK;
}

ksdf_status ksdf_bhm_get(ksdf_bhm* m, uint64_t* keys, uint8_t* active, float* mu, float* prec) {
  if (!m) return KSDF_ERR_ARG;
  int64_t nb = 0;
  ksdf_status s = ksdf_bhm_size(m, &nb, nullptr, nullptr);
  if (s != KSDF_OK) return s;
  cudaStream_t st = m->stream;
  if (keys) BHM_CUDA(m, cudaMemcpyAsync(keys, m->bkey.p, 8 * nb, cudaMemcpyDeviceToHost, st));
  if (active) BHM_CUDA(m, cudaMemcpyAsync(active, m->active.p, nb, cudaMemcpyDeviceToHost, st));
  if (mu || prec) {
    std::vector<float2> w((size_t)nb * m->nw);
    BHM_CUDA(m, cudaMemcpyAsync(w.data(), m->Wmp.p, 8 * w.size(), cudaMemcpyDeviceToHost, st));
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
