// ksdf_query.cu -- the batched local-GP signed-distance query of Kernel-SDF (arXiv 2603.29227, Sec. IV-B).
//
// Pipeline (all stream ordered, no host synchronisation; device-side counts drive persistent kernels):
//   Q1  bin every query (binary64, same rounding as the fit) and insert its cell key in a hash table;
//   Q2  number the distinct query bins, count and group the queries by bin, cut bins into tiles;
//   Q3  candidate lists: per bin, the K valid GP cells nearest on the integer lattice (ring search over
//       Chebyshev shells, exact (distance, key) order; brute force beyond 16 shells);
//   Q4  phase A (per tile of one bin): the candidates' samples are staged to shared memory with TMA bulk
//       copies; one thread per query evaluates every candidate GP
//          f'_g = sum_i alpha_i exp(-lambda (r_i^2 - d_g^2)),   u_g = sqrt(-log f'_g / lambda + d_g^2)
//       (App. D scaling; d_g^2 = min_i r_i^2 is tracked online, the sum is rescaled when the minimum
//       drops, and accumulated with Kahan compensation) and keeps u = min_g u_g (min-fusion, Sec. IV-B.1);
//   Q5  group the queries by winning cell;
//   Q6  phase B (per tile of one winner): gradient grad u = -grad f'/|grad f'|, softmin variance
//       (Sec. IV-B.3) and the GP variance V[f] = 1 - e^{-2 lambda d^2} |L^{-1} k'|^2 (Sec. IV-B.1).
// The plain path runs Q4 and Q6 in binary64 with two-pass minima.
#include "ksdf_internal.cuh"

#include <algorithm>

namespace ksdf {

namespace {

constexpr int kTA = 128;   // phase A threads (one query each)
constexpr int kTB64 = 32;  // phase B threads, FP64 path
constexpr int kRingCells = 4;  // cell shells of the candidate search before it moves to bricks
constexpr float kLog2e = 1.4426950408889634f;

// ---------------------------------------------------------------------------------------------
// small PTX helpers: mbarrier + 1D bulk copy global -> shared (TMA)

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait of one thread (no barrier)
__device__ inline bool mbar_wait_one(uint64_t* bar, uint32_t parity) {
  for (unsigned it = 0; it < (kWaitLimit >> 4); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// bounded wait; returns false (for every thread of the CTA) if any thread gave up
__device__ inline bool mbar_wait_all(uint64_t* bar, uint32_t parity) {
  return !__syncthreads_or(!mbar_wait_one(bar, parity));
}

__device__ inline float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------------------------
// Q1/Q2: binning and grouping

template <class T>
__global__ void k_q_bin(const T* xq, int64_t Q, Params p, uint64_t* qkey, uint64_t* bhk, uint64_t bcap, uint32_t* st) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  int c[3] = {0, 0, 0};
  bool ok = true;
  for (int j = 0; j < p.dim; ++j) ok &= bin_coord((double)xq[q * p.dim + j], p.o[j], p.h, p.rh, c[j]);
  if (!ok) {
    atomicOr(st, ST_NONFINITE);
    qkey[q] = kEmptyKey;
    return;
  }
  uint64_t k = pack_key(c[0], c[1], c[2]);
  qkey[q] = k;
  uint64_t s = mix64(k) & (bcap - 1);
  for (uint64_t probe = 0; probe < bcap; ++probe) {
    uint64_t cur = bhk[s];
    if (cur == k) return;
    if (cur == kEmptyKey) {
      unsigned long long prev =
          atomicCAS((unsigned long long*)&bhk[s], (unsigned long long)kEmptyKey, (unsigned long long)k);
      if (prev == kEmptyKey || prev == k) return;
    }
    s = (s + 1) & (bcap - 1);
  }
  atomicOr(st, ST_CAPACITY);
}

// query counters of the refit scheduling (App. G): every cell fused for a query (a candidate of its bin) counts
// one request; counters are capped
__global__ void k_count_requests(const int64_t* bin_cnt, const int32_t* cand, const int32_t* ncand,
                                 const int64_t* n_bins, int K, int32_t* qc0) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= *n_bins) return;
  const int n = ncand[b];
  const int add = (int)(bin_cnt[b] < kQueryCounterCap ? bin_cnt[b] : (int64_t)kQueryCounterCap);
  for (int k = 0; k < n; ++k) {
    const int g = cand[b * K + k];
    if (atomicAdd(&qc0[g], add) + add > kQueryCounterCap) atomicMin(&qc0[g], kQueryCounterCap);
  }
}

__global__ void k_slot_flags(const uint64_t* bhk, uint64_t bcap, int64_t* flag) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < (int64_t)bcap) flag[s] = bhk[s] != kEmptyKey ? 1 : 0;
}

// the occupied slots numbered in slot order: bin b's key, and its query count cleared
__global__ void k_bin_table(const uint64_t* bhk, uint64_t bcap, const int64_t* slot_id, uint64_t* bin_key,
                            int64_t* bin_cnt) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < (int64_t)bcap && bhk[s] != kEmptyKey) {
    bin_key[slot_id[s]] = bhk[s];
    bin_cnt[slot_id[s]] = 0;
  }
}

__global__ void k_q_rank(const uint64_t* qkey, int64_t Q, const uint64_t* bhk, const int64_t* slot_id, uint64_t bcap,
                         int32_t* qbin, int32_t* qrank, int64_t* bin_cnt) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  uint64_t k = qkey[q];
  if (k == kEmptyKey) {
    qbin[q] = -1;
    return;
  }
  uint64_t s = mix64(k) & (bcap - 1);
  for (uint64_t probe = 0; probe < bcap; ++probe) {
    if (bhk[s] == k) break;
    s = (s + 1) & (bcap - 1);
  }
  int b = (int)slot_id[s];
  qbin[q] = b;
  qrank[q] = (int32_t)atomicAdd((unsigned long long*)&bin_cnt[b], 1ull);
}

__global__ void k_ntiles(const int64_t* cnt, int64_t n, int T, int64_t* ntiles, const int64_t* n_dev) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n_dev && *n_dev < n) n = *n_dev;
  if (i < n) ntiles[i] = (cnt[i] + T - 1) / T;
}

__global__ void k_scatter_grouped(const int32_t* grp, const int32_t* rank, int64_t Q, const int64_t* off,
                                  int32_t* sorted) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  int g = grp[q];
  if (g >= 0) sorted[off[g] + rank[q]] = (int32_t)q;
}

// tiles: for group i with cnt items starting at off[i]: tiles at tile_off[i] ...
__global__ void k_make_tiles(const int64_t* cnt, const int64_t* off, const int64_t* tile_off, int64_t ngroups, int T,
                             int4* tiles, const int64_t* n_dev) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n_dev && *n_dev < ngroups) ngroups = *n_dev;
  if (i >= ngroups) return;
  int64_t c = cnt[i];
  for (int64_t t = 0; t * T < c; ++t)
    tiles[tile_off[i] + t] = make_int4((int)i, (int)(off[i] + t * T), (int)(c - t * T < T ? c - t * T : T), 0);
}

// Phase A's tiles in a coarse spatial order of their bins, so that the bins processed at the same time share
// candidate cells (their samples then come from L2): a counting sort of the occupied bins by a 16-bit key of
// their 4 x 4 x 4-bin block ((cz/4) mod 16, (cy/4) mod 64, (cx/4) mod 64, lexicographic; wrap-around only
// coarsens the order), bins of one block in any order.
constexpr int kCoarseBuckets = 1 << 16;
__device__ inline uint32_t bin_coarse_key(uint64_t k) {
  const uint32_t x = (uint32_t)(k & 0x1FFFFF) >> 2, y = (uint32_t)((k >> 21) & 0x1FFFFF) >> 2;
  const uint32_t z = (uint32_t)((k >> 42) & 0x1FFFFF) >> 2;
  return ((z & 15u) << 12) | ((y & 63u) << 6) | (x & 63u);
}
__global__ void k_bin_coarse(const uint64_t* bin_key, const int64_t* n_dev, int32_t* coarse, int32_t* rank,
                             int64_t* hist) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= *n_dev) return;
  const uint32_t c = bin_coarse_key(bin_key[b]);
  coarse[b] = (int32_t)c;
  rank[b] = (int32_t)atomicAdd((unsigned long long*)&hist[c], 1ull);
}
__global__ void k_bin_order(const int32_t* coarse, const int32_t* rank, const int64_t* hoff, const int64_t* n_dev,
                            const int64_t* bin_nt, int32_t* order, int64_t* nt_ord) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= *n_dev) return;
  const int64_t pos = hoff[coarse[b]] + rank[b];
  order[pos] = (int32_t)b;
  nt_ord[pos] = bin_nt[b];
}
__global__ void k_make_tiles_ordered(const int32_t* order, const int64_t* cnt, const int64_t* off,
                                     const int64_t* tile_off, const int64_t* n_dev, int T, int4* tiles) {
  const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= *n_dev) return;
  const int b = order[pos];
  const int64_t c = cnt[b];
  for (int64_t t = 0; t * T < c; ++t)
    tiles[tile_off[pos] + t] = make_int4(b, (int)(off[b] + t * T), (int)(c - t * T < T ? c - t * T : T), 0);
}

// ---------------------------------------------------------------------------------------------
// Q3: candidate lists (warp per bin)

struct CandCtx {
  const uint64_t* hk;
  const int32_t* hv;
  uint64_t hcap;
  const int32_t* status;
  const uint64_t* cell_key;
  int64_t G;
  int bb_lo[3], bb_hi[3];  // bounding box of all cells
  const int64_t* bk_off;   // bricks: CSR offsets (nbricks + 1) into bk_cells, 0 bricks when absent
  const int32_t* bk_cells;
  int bk_lo[3], bk_n[3];
  int64_t nbricks;
  int K, dim;
};

// insert (D, key, g) into a sorted top-K list (lane 0 only)
__device__ inline void topk_insert(long long* D, uint64_t* Kk, int* Gg, int& n, int K, long long d, uint64_t key,
                                   int g) {
  int pos = n;
  while (pos > 0 && (d < D[pos - 1] || (d == D[pos - 1] && key < Kk[pos - 1]))) --pos;
  if (pos >= K) return;
  int last = n < K ? n : K - 1;
  for (int t = last; t > pos; --t) {
    D[t] = D[t - 1];
    Kk[t] = Kk[t - 1];
    Gg[t] = Gg[t - 1];
  }
  D[pos] = d;
  Kk[pos] = key;
  Gg[pos] = g;
  if (n < K) ++n;
}

constexpr int kCandWarps = 8;

// points of the Chebyshev shell of radius R around the origin (the cube's surface only): 24 R^2 + 2 in 3D
// (faces z = +-R; y = +-R with |z| < R; x = +-R with |y|, |z| < R), 8 R in 2D, 1 for R = 0
__device__ __forceinline__ int shell_size(int R, int dim) {
  if (R == 0) return 1;
  return dim == 3 ? 24 * R * R + 2 : 8 * R;
}
__device__ __forceinline__ void shell_point(int t, int R, int dim, int& dx, int& dy, int& dz) {
  dz = 0;
  if (R == 0) {
    dx = dy = 0;
    return;
  }
  const int side = 2 * R + 1, in = side - 2;
  if (dim == 2) {
    if (t < 2 * side) {  // rows y = -R, +R
      dy = t < side ? -R : R;
      dx = (t < side ? t : t - side) - R;
    } else {  // columns x = -R, +R with |y| < R
      const int u = t - 2 * side;
      dx = u < in ? -R : R;
      dy = (u < in ? u : u - in) - R + 1;
    }
    return;
  }
  const int f0 = 2 * side * side, f1 = f0 + 2 * side * in;
  if (t < f0) {  // z = -R, +R: (x, y) over the full square
    const int u = t < side * side ? t : t - side * side;
    dz = t < side * side ? -R : R;
    dy = u / side - R;
    dx = u - (u / side) * side - R;
  } else if (t < f1) {  // y = -R, +R: x over [-R, R], z over (-R, R)
    const int u0 = t - f0, half = side * in;
    const int u = u0 < half ? u0 : u0 - half;
    dy = u0 < half ? -R : R;
    dz = u / side - R + 1;
    dx = u - (u / side) * side - R;
  } else {  // x = -R, +R: y and z over (-R, R)
    const int u0 = t - f1, half = in * in;
    const int u = u0 < half ? u0 : u0 - half;
    dx = u0 < half ? -R : R;
    dz = u / in - R + 1;
    dy = u - (u / in) * in - R + 1;
  }
}

// each lane offers (d, key, g) when `found`; lane 0 merges the offers into the warp's sorted top-K list
struct WarpTopK {
  long long* D;
  uint64_t* Kk;
  int* Gg;
  int* n;
  long long* eD;
  uint64_t* eK;
  int* eG;
  int K;
  // whether (d, key) would enter the current list
  __device__ __forceinline__ bool admits(long long d, uint64_t key) const {
    const int c = *n;
    return c < K || d < D[K - 1] || (d == D[K - 1] && key < Kk[K - 1]);
  }
  __device__ __forceinline__ void offer(bool found, long long d, uint64_t key, int g, int lane) const {
    unsigned mask = __ballot_sync(0xffffffffu, found);
    if (found) {
      eD[lane] = d;
      eK[lane] = key;
      eG[lane] = g;
    }
    __syncwarp();
    if (lane == 0) {
      int c = *n;
      while (mask) {
        const int l = __ffs(mask) - 1;
        mask &= mask - 1;
        topk_insert(D, Kk, Gg, c, K, eD[l], eK[l], eG[l]);
      }
      *n = c;
    }
    __syncwarp();
  }
  // every cell not offered yet has D >= lb2: the list is final
  __device__ __forceinline__ bool final_below(long long lb2) const { return *n >= K && D[K - 1] < lb2; }
};

// The K valid cells nearest to a bin on the integer lattice, ordered by (squared distance D, key).  Three
// exact searches, cheapest first for the bin at hand, all giving the same list:
//   cell rings: Chebyshev shells R = 0, 1, ... of cells around the bin, looked up in the cell hash table,
//     until the K-th distance is below (R+1)^2 (bins near the surface: a few shells);
//   bricks: beyond kRingCells shells, Chebyshev shells of 8^3-cell bricks; the cells of a brick are
//     offered unless the rings already visited them or the brick's box is farther than the K-th
//     candidate; after brick shell Rb every unvisited cell is at least 8 Rb + 1 + (offset in the brick)
//     away along some axis;
//   all cells: one pass over every cell, when the shells would visit more lattice points than there are
//     cells (or bricks).
__global__ void __launch_bounds__(32 * kCandWarps)
    k_candidates(const uint64_t* bin_key, const int64_t* n_bins_dev, int64_t n_bins_host, CandCtx cc, int32_t* cand,
                 int32_t* ncand) {
  __shared__ long long sD[kCandWarps][kMaxK];
  __shared__ uint64_t sK[kCandWarps][kMaxK];
  __shared__ int sG[kCandWarps][kMaxK];
  __shared__ long long eD[kCandWarps][32];
  __shared__ uint64_t eK[kCandWarps][32];
  __shared__ int eG[kCandWarps][32];
  __shared__ int sN[kCandWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nb = n_bins_dev ? *n_bins_dev : n_bins_host;
  const int K = cc.K;
  const WarpTopK top{sD[w], sK[w], sG[w], &sN[w], eD[w], eK[w], eG[w], K};
  for (int64_t b = (int64_t)blockIdx.x * kCandWarps + w; b < nb; b += (int64_t)gridDim.x * kCandWarps) {
    int bx, by, bz;
    unpack_key(bin_key[b], bx, by, bz);
    const int bc[3] = {bx, by, bz};
    if (lane == 0) sN[w] = 0;
    __syncwarp();
    int rstop = 0;  // Chebyshev radius beyond which no cell exists
    for (int j = 0; j < 3; ++j) rstop = max(rstop, max(abs(bc[j] - cc.bb_lo[j]), abs(bc[j] - cc.bb_hi[j])));
    bool done = false, far = false;
    int Rdone = -1;    // cell shells 0..Rdone visited
    int64_t seen = 0;  // lattice points visited so far
    for (int R = 0; R <= rstop; ++R) {
      const int total = shell_size(R, cc.dim);
      if (R > kRingCells || seen + total > cc.G) {
        far = true;
        break;
      }
      seen += total;
      for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        bool found = false;
        long long d = 0;
        uint64_t key = 0;
        int g = -1;
        if (t < total) {
          int dx, dy, dz;
          shell_point(t, R, cc.dim, dx, dy, dz);
          const int64_t nx = (int64_t)bx + dx, ny = (int64_t)by + dy, nz = (int64_t)bz + dz;
          if (nx >= -kBias && nx < kBias && ny >= -kBias && ny < kBias && nz >= -kBias && nz < kBias) {
            key = pack_key(nx, ny, nz);
            g = hash_find(cc.hk, cc.hv, cc.hcap, key);
            if (g >= 0 && cc.status[g] == KSDF_CELL_OK) {
              found = true;
              d = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
            }
          }
        }
        top.offer(found, d, key, g, lane);
      }
      Rdone = R;
      if (top.final_below((long long)(R + 1) * (R + 1))) {
        done = true;
        break;
      }
    }
    bool brute = far && !done;
    if (brute && cc.nbricks > 0) {
      brute = false;
      int B[3], o[3], rbstop = 0;
      for (int j = 0; j < 3; ++j) {
        const int u = bc[j] - cc.bk_lo[j];
        B[j] = u >> kBrickShift;  // floor (arithmetic shift)
        o[j] = u - (B[j] << kBrickShift);
        rbstop = max(rbstop, max(abs(B[j]), abs(B[j] - (cc.bk_n[j] - 1))));
      }
      int64_t seenb = 0;
      for (int Rb = 0; Rb <= rbstop; ++Rb) {
        const int total = shell_size(Rb, cc.dim);
        if (seenb + total > cc.nbricks) {
          brute = true;
          break;
        }
        seenb += total;
        for (int t0 = 0; t0 < total; t0 += 32) {
          const int t = t0 + lane;
          int64_t boff = 0;
          int bcnt = 0;
          if (t < total) {
            int d3[3];
            shell_point(t, Rb, cc.dim, d3[0], d3[1], d3[2]);
            const int q0 = B[0] + d3[0], q1 = B[1] + d3[1], q2 = B[2] + d3[2];
            if (q0 >= 0 && q0 < cc.bk_n[0] && q1 >= 0 && q1 < cc.bk_n[1] && q2 >= 0 && q2 < cc.bk_n[2]) {
              const int64_t bi = ((int64_t)q2 * cc.bk_n[1] + q1) * cc.bk_n[0] + q0;
              boff = cc.bk_off[bi];
              bcnt = (int)(cc.bk_off[bi + 1] - boff);
              if (bcnt > 0) {
                // squared lattice distance from the bin to the brick's box
                const int q[3] = {q0, q1, q2};
                long long dmin = 0;
                for (int j = 0; j < 3; ++j) {
                  const int lo = cc.bk_lo[j] + (q[j] << kBrickShift), hi = lo + (1 << kBrickShift) - 1;
                  const long long gap = max(0, max(lo - bc[j], bc[j] - hi));
                  dmin += gap * gap;
                }
                if (sN[w] >= K && dmin > sD[w][K - 1]) bcnt = 0;
              }
            }
          }
          unsigned bm = __ballot_sync(0xffffffffu, bcnt > 0);
          while (bm) {
            const int l = __ffs(bm) - 1;
            bm &= bm - 1;
            const int64_t o0 = __shfl_sync(0xffffffffu, boff, l);
            const int cl = __shfl_sync(0xffffffffu, bcnt, l);
            for (int i0 = 0; i0 < cl; i0 += 32) {
              const int i = i0 + lane;
              bool found = false;
              long long d = 0;
              uint64_t key = 0;
              int g = -1;
              if (i < cl) {
                g = cc.bk_cells[o0 + i];
                key = cc.cell_key[g];
                int cx, cy, cz;
                unpack_key(key, cx, cy, cz);
                const int dx = cx - bx, dy = cy - by, dz = cz - bz;
                if (max(abs(dx), max(abs(dy), abs(dz))) > Rdone) {
                  d = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
                  found = top.admits(d, key);
                }
              }
              top.offer(found, d, key, g, lane);
            }
          }
        }
        int L = INT_MAX;
        for (int j = 0; j < cc.dim; ++j)
          L = min(L, min(o[j] + (Rb << kBrickShift) + 1, ((Rb + 1) << kBrickShift) - o[j]));
        if (top.final_below((long long)L * L)) break;
      }
    }
    if (brute) {
      if (lane == 0) sN[w] = 0;
      __syncwarp();
      for (int64_t g0 = 0; g0 < cc.G; g0 += 32) {
        const int64_t g = g0 + lane;
        bool found = false;
        long long d = 0;
        uint64_t key = 0;
        if (g < cc.G && cc.status[g] == KSDF_CELL_OK) {
          key = cc.cell_key[g];
          int cx, cy, cz;
          unpack_key(key, cx, cy, cz);
          d = (long long)(cx - bx) * (cx - bx) + (long long)(cy - by) * (cy - by) + (long long)(cz - bz) * (cz - bz);
          found = top.admits(d, key);
        }
        top.offer(found, d, key, (int)g, lane);
      }
    }
    const int n = sN[w];
    if (lane < K) cand[b * K + lane] = lane < n ? sG[w][lane] : -1;
    if (lane == 0) ncand[b] = n;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------------
// Q4: phase A, mixed precision

// Upper bound (with a factor 2 of margin) on |u - u_exact| for one candidate GP evaluated in FP32 by k_phaseA,
// u_exact being the binary64 value on the binary64 data.  Inputs: f = the compensated sum f', sa = the sum of
// |alpha_i k'_i| on the same scale, m = d^2 (FP32), u, nres = the number of rescalings of the running sum,
// qa = the largest |coordinate| of the query in the candidate's frame, dxs = the rounding bound of a stored
// FP32 sample coordinate.  Each term alpha_i k'_i carries a relative error eps from its exponent
// lambda (r_i^2 - d^2): the FP32 squares (a few 2^-24 r^2), the positions of the sample (dxs) and of the query
// (2^-23 qa) moving r_i^2 and d^2 by 2 r |delta| -- taken at r^2 = d^2 + 40 / lambda, beyond which the terms
// are below e^-40 of the largest -- plus ex2.approx and the FP32 alpha; the sums and rescalings add 2^-21
// and 2^-22 per rescale of sa.  Then d(ln f') = df'/f', d(u^2) = d(ln f')/lambda + the rounding of m and of
// the final fma, and du = d(u^2) / (u + sqrt(d(u^2))).  f' within its own error of zero gives +inf.
__device__ __forceinline__ float u_error_bound(float f, float sa, float m, float u, int nres, float qa, float lam,
                                               float dxs) {
  const float R = m + 40.f / lam;
  const float dpos = 1.7320508f * (dxs + qa * 0x1p-23f);
  const float dr2 = 2.f * sqrtf(R) * dpos + 3.f * 0x1p-24f * R;
  const float eps = lam * 2.f * dr2 + 1e-6f + (float)nres * 0x1p-22f;
  const float df = sa * (eps + 0x1p-21f);
  if (!(f > 2.f * df)) return INFINITY;
  const float du2 = df / (f * lam) + 0x1p-22f * (fabsf(__logf(f)) / lam + m) + dr2;
  return 2.f * du2 / (u + sqrtf(du2));
}

struct PhaseAArgs {
  const int4* tiles;           // (bin, start, count)
  const int64_t* n_tiles;      // device count
  int* counter;
  const int32_t* sorted_q;
  const uint64_t* bin_key;
  const int32_t* cand;
  const int32_t* ncand;
  const int64_t* ts_off;
  const int32_t* cell_n;
  const uint64_t* cell_key;
  const float4* mf4;
  const D4* md4;
  int32_t* qwin;
  float* qu;
  double* qu64;
  uint32_t* qflag;
  uint32_t* st;
  int chunks;  // phase A's shared-memory budget in chunks of 8 samples
};

// The same bound for the Matern 3/2 kernel, where u = -log f' / lambda + d is linear in log f' and d (m is d):
// each term's exponent lambda (r_i - d) carries the errors of r_i = sqrt.approx(r_i^2) (2^-22 relative) and of
// the positions (dxs, 2^-23 qa); the factor (1 + lambda r_i) carries a smaller relative error.
__device__ __forceinline__ float u_error_bound_matern(float f, float sa, float d, int nres, float qa, float lam,
                                                      float dxs) {
  const float R = d + 40.f / lam;
  const float dr = 0x1p-22f * R + 1.7320508f * (dxs + qa * 0x1p-23f);
  const float eps = lam * 2.f * dr + 1e-6f + (float)nres * 0x1p-22f;
  const float df = sa * (eps + 0x1p-21f);
  if (!(f > 2.f * df)) return INFINITY;
  return 2.f * (df / (f * lam) + 0x1p-22f * (fabsf(__logf(f)) / lam + d) + dr);
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Phase A shared memory, per tile: candidates' samples as chunks of 8 in SoA form -- one chunk is 40 floats,
// x[8] y[8] z[8] alpha[8] |alpha|[8] -- each candidate padded to whole chunks with far zero-weight samples, at
// most the budget's chunks at a time (a tile whose candidates hold more is done in rounds of whole candidates);
// then the per-(candidate, query) results u, du and flag bits.
constexpr int kChunkF = 40;
// the budget: the context's tile shape (ksdf_autotune_query), at least one whole largest candidate
__host__ __device__ inline int phase_a_chunks(int tuned, int n_max) { return max(tuned, (n_max + 7) / 8); }
__host__ __device__ inline size_t phase_a_smem(int K, int chunks) {
  return sizeof(float) * (size_t)kChunkF * chunks + (size_t)K * kTA * (2 * sizeof(float) + 1);
}

// One CTA per tile of up to kTA queries of one bin.  The candidates' samples are read into shared memory (SoA
// chunks); the warps then pull tasks (candidate k, block of 16 queries), two at a time (one per half-warp), and
// for a task each lane evaluates one query on candidate k over its samples, eight per step with packed FP32x2
// arithmetic:
//   r_i^2 = |q - x_i|^2, the running minimum m = d^2 (App. D), rescaled sums
//   f' = sum_i alpha_i 2^{c1 (m - r_i^2)} (Kahan-compensated across steps) and sum_i |alpha_i| 2^{c1 (m - r_i^2)},
//   u = sqrt(-log f' / lambda + m) (kernel table) with its error bound (u_error_bound).
// With the Matern 3/2 kernel the running minimum is over r_i = sqrt(r_i^2) (d itself), the terms are
// alpha_i (1 + lambda r_i) 2^{c1 (d - r_i)} and u = -log f' / lambda + d.
// Finally a thread per query takes the minimum over the candidates in list order (min-fusion, Sec. IV-B.1), the
// first on equal u, and sets the near-tie flag from the error bounds.
template <bool MATERN>
__global__ void __launch_bounds__(kTA) k_phaseA(PhaseAArgs a, const float* xq, Params p) {
  extern __shared__ __align__(16) float sA[];
  __shared__ int s_tile, s_nc, s_task, s_k1, s_c[kMaxK], s_n[kMaxK], s_ch[kMaxK];
  __shared__ float s_off[kMaxK][3];
  __shared__ float s_ql[kTA][3];
  __shared__ float s_bh[3], s_bl[3];
  const int tid = threadIdx.x, lane = tid & 31;
  const int K = p.K;
  const float c1 = (float)p.lambda * kLog2e;
  const float inv_lam = (float)(1.0 / p.lambda);
  const float lam = (float)p.lambda;
  const float dxs = (float)((p.h + p.mu) * 0x1p-24);  // rounding of a stored cell-local FP32 coordinate
  const int budget = a.chunks;
  float* s_u = sA + (size_t)kChunkF * budget;
  float* s_du = s_u + K * kTA;
  uint8_t* s_fl = reinterpret_cast<uint8_t*>(s_du + K * kTA);
  const int64_t ntiles = *a.n_tiles;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const int4 tile = a.tiles[t];
    const int b = tile.x;
    int bc[3];
    unpack_key(a.bin_key[b], bc[0], bc[1], bc[2]);
    if (tid < 32) {  // the candidate list and the candidates' frame offsets, a lane per candidate
      const int nc = a.ncand[b];
      if (lane < nc) {
        const int g = a.cand[(int64_t)b * K + lane];
        s_c[lane] = g;
        s_n[lane] = a.cell_n[g];
        int cc[3];
        unpack_key(a.cell_key[g], cc[0], cc[1], cc[2]);
        for (int j = 0; j < 3; ++j) s_off[lane][j] = (float)((double)(bc[j] - cc[j]) * p.h);
      }
      if (lane == 0) s_nc = nc;
      if (lane < 3) base_split(p.o[lane], bc[lane], p.h, s_bh[lane], s_bl[lane]);  // the bin corner, binary64 once
    }
    __syncthreads();
    // the tile's queries in the bin's frame (FP32 two-term subtraction of the bin corner)
    {
      const bool live = tid < tile.z;
      const int q = live ? a.sorted_q[tile.y + tid] : 0;
      for (int j = 0; j < 3; ++j)
        s_ql[tid][j] = (live && j < p.dim) ? local32(xq[(int64_t)q * p.dim + j], s_bh[j], s_bl[j]) : 0.f;
    }
    __syncthreads();
    const int nc = s_nc;
    const int nqb = (tile.z + 15) >> 4;  // blocks of 16 queries: a warp takes two tasks, one per half
    for (int k0 = 0; k0 < nc;) {
      // a round: candidates k0 .. k1-1 whose chunks fit the budget (at least one)
      if (tid == 0) {
        int k1 = k0, tot = 0;
        while (k1 < nc && (k1 == k0 || tot + ((s_n[k1] + 7) >> 3) <= budget)) {
          s_ch[k1] = tot;
          tot += (s_n[k1] + 7) >> 3;
          ++k1;
        }
        s_k1 = k1;
        s_task = 0;
      }
      __syncthreads();
      const int k1 = s_k1;
      // samples into SoA chunks: thread e takes sample slot e of the round's flattened (candidate, slot) space
      {
        const int tot = 8 * (s_ch[k1 - 1] + ((s_n[k1 - 1] + 7) >> 3));
        int k = k0;
        for (int e = tid; e < tot; e += kTA) {
          while (k + 1 < k1 && e >= 8 * s_ch[k + 1]) ++k;
          const int i = e - 8 * s_ch[k];
          float4 v = make_float4(1e15f, 1e15f, 1e15f, 0.f);  // padding: far away, zero weight
          if (i < s_n[k]) v = __ldg(a.mf4 + a.ts_off[s_c[k]] + i);
          float* ch = sA + (size_t)kChunkF * (s_ch[k] + (i >> 3)) + (i & 7);
          ch[0] = v.x;
          ch[8] = v.y;
          ch[16] = v.z;
          ch[24] = v.w;
          ch[32] = fabsf(v.w);
        }
      }
      __syncthreads();
      const int ntask = (k1 - k0) * nqb;
      for (;;) {
        int task = 0;
        if (lane == 0) task = atomicAdd(&s_task, 2);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= ntask) break;
        // the second half of the warp takes the next task (when there is none it repeats the first with no
        // query: its results are not stored)
        const bool hv = task + (lane >> 4) < ntask;
        const int tk = hv ? task + (lane >> 4) : task;
        const int k = k0 + tk / nqb;
        const int qi = hv ? (tk % nqb) * 16 + (lane & 15) : tile.z;
        const int qs = qi < tile.z ? qi : 0;
        const float qx = s_ql[qs][0] + s_off[k][0], qy = s_ql[qs][1] + s_off[k][1], qz = s_ql[qs][2] + s_off[k][2];
        const unsigned long long QX = f2pack(qx, qx), QY = f2pack(qy, qy), QZ = f2pack(qz, qz);
        const unsigned long long NC1 = f2pack(-c1, -c1);
        const unsigned long long LAM2 = f2pack(lam, lam), ONE2 = f2pack(1.f, 1.f);
        const float* ch = sA + (size_t)kChunkF * s_ch[k];
        const int nch = (s_n[k] + 7) >> 3;
        float m = INFINITY, s = 0.f, comp = 0.f;
        unsigned long long SA = f2pack(0.f, 0.f);
        int nres = 0;
        for (int c = 0; c < nch; ++c, ch += kChunkF) {
          const float4* c4 = reinterpret_cast<const float4*>(ch);
          unsigned long long r2[4];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float4 x4 = c4[h], y4 = c4[2 + h], z4 = c4[4 + h];
            const unsigned long long dx0 = f2sub(QX, f2pack(x4.x, x4.y)), dx1 = f2sub(QX, f2pack(x4.z, x4.w));
            const unsigned long long dy0 = f2sub(QY, f2pack(y4.x, y4.y)), dy1 = f2sub(QY, f2pack(y4.z, y4.w));
            const unsigned long long dz0 = f2sub(QZ, f2pack(z4.x, z4.y)), dz1 = f2sub(QZ, f2pack(z4.z, z4.w));
            r2[2 * h] = f2fma(dx0, dx0, f2fma(dy0, dy0, f2mul(dz0, dz0)));
            r2[2 * h + 1] = f2fma(dx1, dx1, f2fma(dy1, dy1, f2mul(dz1, dz1)));
          }
          float rv[8];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float2 u = f2unpack(r2[h]);
            rv[2 * h] = u.x;
            rv[2 * h + 1] = u.y;
          }
          if (MATERN) {  // distances, and the exponents below act on them
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              rv[2 * h] = sqrt_approx(rv[2 * h]);
              rv[2 * h + 1] = sqrt_approx(rv[2 * h + 1]);
              r2[h] = f2pack(rv[2 * h], rv[2 * h + 1]);
            }
          }
          const float cm = fminf(fminf(fminf(rv[0], rv[1]), fminf(rv[2], rv[3])),
                                 fminf(fminf(rv[4], rv[5]), fminf(rv[6], rv[7])));
          const float mn = fminf(m, cm);
          nres += mn < m ? 1 : 0;
          const float sc = ex2(c1 * (mn - m));
          s *= sc;
          comp *= sc;
          SA = f2mul(SA, f2pack(sc, sc));
          m = mn;
          const unsigned long long CMN = f2pack(c1 * mn, c1 * mn);
          unsigned long long T[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float2 ev = f2unpack(f2fma(NC1, r2[h], CMN));
            unsigned long long kk = f2pack(ex2(ev.x), ex2(ev.y));
            if (MATERN) kk = f2mul(kk, f2fma(LAM2, r2[h], ONE2));  // (1 + lambda r) 2^{c1 (d - r)}
            const float4 al4 = c4[6 + (h >> 1)], ab4 = c4[8 + (h >> 1)];
            const unsigned long long AL = (h & 1) ? f2pack(al4.z, al4.w) : f2pack(al4.x, al4.y);
            const unsigned long long AB = (h & 1) ? f2pack(ab4.z, ab4.w) : f2pack(ab4.x, ab4.y);
            T[h] = f2mul(AL, kk);
            SA = f2fma(AB, kk, SA);
          }
          // the step's eight terms summed as a tree, then added to the running sum with compensation
          const float2 cs2 = f2unpack(f2add(f2add(T[0], T[1]), f2add(T[2], T[3])));
          const float cs = cs2.x + cs2.y;
          const float y = cs - comp;
          const float tt = s + y;
          comp = (tt - s) - y;
          s = tt;
        }
        const float f = s - comp;
        const float2 sa2 = f2unpack(SA);
        const float sa = sa2.x + sa2.y;
        float u;
        uint32_t fl = 0;
        if (f > 0.f) {
          if (MATERN) {
            u = fmaf(-logf(f), inv_lam, m);
          } else {
            u = fmaf(-logf(f), inv_lam, m);
            u = u < 0.f ? u : sqrtf(u);
          }
          if (u < 0.f) {
            u = 0.f;
            fl |= KSDF_FLAG_CLAMPED;
          }
        } else {
          u = MATERN ? m : sqrtf(m);
          fl |= KSDF_FLAG_FALLBACK;
        }
        const float qa = fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz)));
        const float du = MATERN ? u_error_bound_matern(f, sa, m, nres, qa, lam, dxs)
                                : u_error_bound(f, sa, m, u, nres, qa, lam, dxs);
        if (qi < tile.z) {
          s_u[k * kTA + qi] = u;
          s_du[k * kTA + qi] = du;
          s_fl[k * kTA + qi] = (uint8_t)fl;
        }
      }
      __syncthreads();
      k0 = k1;
    }
    // min-fusion over the candidates in list order, thread per query
    if (tid < tile.z) {
      float bu = INFINITY, su = INFINITY, bdu = 0.f, olo = INFINITY;
      int bk = -1;
      uint32_t bflag = 0;
      for (int k = 0; k < nc; ++k) {
        const float u = s_u[k * kTA + tid], du = s_du[k * kTA + tid];
        if (u < bu) {
          su = bu;
          olo = fminf(olo, bu - bdu);
          bu = u;
          bdu = du;
          bk = k;
          bflag = s_fl[k * kTA + tid];
        } else {
          su = fminf(su, u);
          olo = fminf(olo, u - du);
        }
      }
      uint32_t fl = bflag;
      // near tie: another candidate within 1e-5 m, or one whose u may lie below the winner's given the error
      // bounds of the two FP32 evaluations
      if (nc >= 2 && (su - bu <= 1e-5f || olo <= bu + bdu)) fl |= KSDF_FLAG_NEAR_TIE;
      if (nc == 0) fl |= KSDF_FLAG_NO_GP;
      const int q = a.sorted_q[tile.y + tid];
      a.qwin[q] = bk >= 0 ? s_c[bk] : -1;
      a.qu[q] = bu;
      a.qflag[q] = fl;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Q4 (plain path): phase A in binary64, two passes per candidate

template <bool MATERN>
__global__ void __launch_bounds__(kTA) k_phaseA64(PhaseAArgs a, const double* xq, Params p) {
  extern __shared__ __align__(128) D4 s_d[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_tile, s_nc, s_c[kMaxK], s_n[kMaxK], s_base[kMaxK];
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_proxy_async();
  }
  __syncthreads();
  uint32_t phase = 0;
  const int64_t ntiles = *a.n_tiles;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const int4 tile = a.tiles[t];
    const int b = tile.x;
    if (tid == 0) {
      const int nc = a.ncand[b];
      s_nc = nc;
      uint32_t bytes = 0;
      int base = 0;
      for (int k = 0; k < nc; ++k) {
        const int g = a.cand[(int64_t)b * p.K + k];
        s_c[k] = g;
        s_n[k] = a.cell_n[g];
        s_base[k] = base;
        base += s_n[k];
        bytes += (uint32_t)s_n[k] * 32u;
      }
      fence_proxy_async();
      mbar_expect_tx(&bar, bytes);
      for (int k = 0; k < nc; ++k)
        bulk_g2s(s_d + s_base[k], a.md4 + a.ts_off[s_c[k]], (uint32_t)s_n[k] * 32u, &bar);
    }
    const bool live = tid < tile.z;
    const int q = live ? a.sorted_q[tile.y + tid] : 0;
    double xg[3] = {0, 0, 0};
    if (live)
      for (int j = 0; j < p.dim; ++j) xg[j] = xq[(int64_t)q * p.dim + j];
    if (!mbar_wait_all(&bar, phase)) {
      if (tid == 0) atomicOr(a.st, ST_TIMEOUT);
      return;
    }
    phase ^= 1;
    const int nc = s_nc;
    if (live) {
      double bu = INFINITY, su = INFINITY;
      int bk = -1;
      uint32_t bflag = 0;
      for (int k = 0; k < nc; ++k) {
        int cc[3];
        unpack_key(a.cell_key[s_c[k]], cc[0], cc[1], cc[2]);
        double ql[3];
        for (int j = 0; j < 3; ++j) ql[j] = j < p.dim ? __dsub_rn(xg[j], cell_base(p.o[j], cc[j], p.h)) : 0.0;
        const D4* xs = s_d + s_base[k];
        const int n = s_n[k];
        double m = INFINITY;
        for (int i = 0; i < n; ++i) {
          const D4 v = xs[i];
          const double dx = ql[0] - v.x, dy = ql[1] - v.y, dz = ql[2] - v.z;
          m = fmin(m, dx * dx + dy * dy + dz * dz);
        }
        double f = 0.0;
        const double dm = sqrt(m);
        for (int i = 0; i < n; ++i) {
          const D4 v = xs[i];
          const double dx = ql[0] - v.x, dy = ql[1] - v.y, dz = ql[2] - v.z;
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (MATERN) {
            const double r = sqrt(r2);
            f += v.w * (1.0 + p.lambda * r) * exp(-p.lambda * (r - dm));
          } else {
            f += v.w * exp(-p.lambda * (r2 - m));
          }
        }
        double u;
        uint32_t fl = 0;
        if (f > 0.0) {
          u = MATERN ? -log(f) / p.lambda + dm : -log(f) / p.lambda + m;
          if (u < 0.0) {
            u = 0.0;
            fl |= KSDF_FLAG_CLAMPED;
          } else if (!MATERN) {
            u = sqrt(u);
          }
        } else {
          u = dm;
          fl |= KSDF_FLAG_FALLBACK;
        }
        if (u < bu) {
          su = bu;
          bu = u;
          bk = k;
          bflag = fl;
        } else if (u < su) {
          su = u;
        }
      }
      uint32_t fl = bflag;
      if (nc >= 2 && su - bu <= 1e-5) fl |= KSDF_FLAG_NEAR_TIE;
      if (nc == 0) fl |= KSDF_FLAG_NO_GP;
      a.qwin[q] = bk >= 0 ? s_c[bk] : -1;
      a.qu64[q] = bu;
      a.qflag[q] = fl;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Q5: grouping by winner; queries without a winner get their final outputs here

template <class T>
__global__ void k_w_rank(const int32_t* qwin, const uint32_t* qflag, const int32_t* qbin, int64_t Q, int32_t* wrank,
                         int64_t* wcnt, uint32_t mask, int dim, T* sdf, T* grad, T* var_sdf, T* var_f,
                         T* var_grad, int32_t* winner, uint32_t* flags) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const int w = qbin[q] < 0 ? -1 : qwin[q];
  if (w >= 0) {
    wrank[q] = (int32_t)atomicAdd((unsigned long long*)&wcnt[w], 1ull);
    return;
  }
  const bool invalid = qbin[q] < 0;
  const T nan = (T)NAN;
  if (mask & KSDF_OUT_SDF) sdf[q] = invalid ? nan : (T)INFINITY;
  if (mask & KSDF_OUT_GRAD)
    for (int j = 0; j < dim; ++j) grad[q * dim + j] = invalid ? nan : (T)0;
  if (mask & KSDF_OUT_VAR_SDF) var_sdf[q] = invalid ? nan : (T)0;
  if (mask & KSDF_OUT_VAR_F) var_f[q] = invalid ? nan : (T)1;
  if (mask & KSDF_OUT_VAR_GRAD)
    for (int j = 0; j < dim; ++j) var_grad[q * dim + j] = invalid ? nan : (T)0;
  if (mask & KSDF_OUT_WINNER) winner[q] = -1;
  if (mask & KSDF_OUT_FLAGS) flags[q] = invalid ? KSDF_FLAG_INVALID : (qflag[q] | KSDF_FLAG_NO_GP);
}

__global__ void k_w_scatter(const int32_t* qwin, const int32_t* qbin, const int32_t* wrank, int64_t Q,
                            const int64_t* woff, int32_t* sorted) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  if (qbin[q] < 0) return;
  int w = qwin[q];
  if (w >= 0) sorted[woff[w] + wrank[q]] = (int32_t)q;
}

// ---------------------------------------------------------------------------------------------
// Q6: phase B, mixed precision.  A tile is up to 32 queries sharing the winner cell (lane = query); the
// 4 warps of the CTA split the cell's samples for the minimum, k', the gradient and the softmin sums,
// and split the 8-row blocks of L^{-1} for V[f] = 1 - e^{-2 lambda d^2} |L^{-1} k'|^2.

constexpr int kBQ = 32;
constexpr int kBW = 4;

// The per-sample kernel terms of phase B from e = r_i^2 - d^2 (excess_sq) and z = r_i: the scaled kernel value
// k' (the A operand of V[f]), the factor wg of its gradient (grad k' = -c wg (x - x_i)) and y = z - d for the
// softmin weights.  RBF: k' = wg = 2^{-c1 e}, y = z - d.  Matern 3/2: y = e / (z + d) (z - d without the
// cancellation of two metre-scale numbers), wg = 2^{-c1 y}, k' = (1 + lambda z) wg.
template <bool MATERN>
__device__ __forceinline__ void kernel_terms(float e, float z, float zmin, float c1, float lam, float& kp, float& wg,
                                             float& y) {
  if (MATERN) {
    const float den = z + zmin;
    y = den > 0.f ? fmaxf(e, 0.f) * __frcp_rn(den) : 0.f;
    wg = ex2(-c1 * y);
    kp = fmaf(lam, z, 1.f) * wg;
  } else {
    kp = ex2(-c1 * e);
    wg = kp;
    y = fmaxf(z - zmin, 0.f);
  }
}

struct PhaseBArgs {
  const int4* tiles;
  const int64_t* n_tiles;
  int* counter;
  const int32_t* sorted_w;
  const int64_t* ts_off;
  const int32_t* cell_n;
  const uint64_t* cell_key;
  const int64_t* chol_off;
  const int64_t* linv_off;
  const float4* mf4;
  const D4* md4;
  const float* mvar;
  const float4* mnrm;
  const float* linv32;
  const double* chol64;
  const float* qu;
  const double* qu64;
  const uint32_t* qflag;
  const int8_t* sign;
  int has_normals;
  uint32_t mask;
  uint32_t* st;
};

__device__ __forceinline__ float vf_rows(const float* Lb, int n, int w, const float* s_k, int lane) {
  // sum over this warp's 8-row blocks R = w, w + 4, ... of |L^{-1}[8R..8R+7][:] k'|^2
  float vsum = 0.f;
  const int nb = (n + 7) / 8;
  // serpentine assignment: blocks w, 2 kBW - 1 - w, 2 kBW + w, ... (the work of block R grows with R)
  for (int k = 0;; ++k) {
    const int R = (k >> 1) * 2 * kBW + ((k & 1) ? 2 * kBW - 1 - w : w);
    if (R >= nb) {
      if (k & 1) continue;
      break;
    }
    const float4* blk = reinterpret_cast<const float4*>(Lb + linv_block_off(R));
    const int imax = min(8 * R + 8, n);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int i = 0; i < imax; ++i) {
      const float4 l0 = blk[2 * i], l1 = blk[2 * i + 1];
      const float kk = s_k[i * kBQ + lane];
      acc[0] = fmaf(l0.x, kk, acc[0]);
      acc[1] = fmaf(l0.y, kk, acc[1]);
      acc[2] = fmaf(l0.z, kk, acc[2]);
      acc[3] = fmaf(l0.w, kk, acc[3]);
      acc[4] = fmaf(l1.x, kk, acc[4]);
      acc[5] = fmaf(l1.y, kk, acc[5]);
      acc[6] = fmaf(l1.z, kk, acc[6]);
      acc[7] = fmaf(l1.w, kk, acc[7]);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) vsum = fmaf(acc[r], acc[r], vsum);
  }
  return vsum;
}

constexpr int kBItem = 256;     // queries per phase-B work item (processed 32 at a time)
constexpr int kLinvStageN = 128;  // L^{-1} of cells up to this N is staged in shared memory

// One work item = up to 256 queries sharing the winner cell; the cell's samples and (for N <= 128) its
// L^{-1} are staged once by TMA bulk copies and reused by every chunk of 32 queries.
template <bool MATERN>
__global__ void __launch_bounds__(kBQ* kBW) k_phaseB(PhaseBArgs a, const float* xq, Params p, float* sdf, float* grad,
                                                     float* var_sdf, float* var_f, int32_t* winner, uint32_t* flags,
                                                     int smax_n) {
  // dynamic shared memory: [smax_n] samples (float4) | [linv_blocked_size(128)] L^{-1} | [smax_n] var |
  // [smax_n][32] k'
  extern __shared__ __align__(128) float4 s_x[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_tile;
  __shared__ float s_red[kBW][9][kBQ];
  __shared__ int s_nn[kBW][kBQ];
  __shared__ float s_bh[3], s_bl[3];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  float* s_linv = reinterpret_cast<float*>(s_x + smax_n);
  float* s_var = s_linv + linv_blocked_size(kLinvStageN);
  float* s_k = s_var + smax_n;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_proxy_async();
  }
  __syncthreads();
  const float c1 = (float)p.lambda * kLog2e;
  const float as = (float)p.alpha_s;
  const float c2 = as * kLog2e;
  uint32_t phase = 0;
  const int64_t ntiles = *a.n_tiles;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const int4 tile = a.tiles[t];
    const int g = tile.x;
    const int n = a.cell_n[g];
    const int64_t m0 = a.ts_off[g];
    const bool staged = n <= kLinvStageN;
    if (tid == 0) {
      fence_proxy_async();
      const uint32_t lbytes = staged ? (uint32_t)linv_blocked_size(n) * 4u : 0u;
      mbar_expect_tx(&bar, (uint32_t)n * 16u + lbytes);
      bulk_g2s(s_x, a.mf4 + m0, (uint32_t)n * 16u, &bar);
      if (staged) bulk_g2s(s_linv, a.linv32 + a.linv_off[g], lbytes, &bar);
      int cc[3];
      unpack_key(a.cell_key[g], cc[0], cc[1], cc[2]);
      for (int j = 0; j < 3; ++j) base_split(p.o[j], cc[j], p.h, s_bh[j], s_bl[j]);
    }
    for (int i = tid; i < n; i += blockDim.x) s_var[i] = a.mvar[m0 + i];  // not 16-byte aligned: plain loads
    if (!mbar_wait_all(&bar, phase)) {
      if (tid == 0) atomicOr(a.st, ST_TIMEOUT);
      return;
    }
    phase ^= 1;
    const float* Lb = staged ? s_linv : a.linv32 + a.linv_off[g];
    const int per = (n + kBW - 1) / kBW;
    const int i0 = w * per, i1 = min(n, i0 + per);
    for (int q0 = 0; q0 < tile.z; q0 += kBQ) {
      const bool live = q0 + lane < tile.z;
      const int q = live ? a.sorted_w[tile.y + q0 + lane] : 0;
      float ql[3] = {0.f, 0.f, 0.f};
      if (live)
        for (int j = 0; j < p.dim; ++j) ql[j] = local32(xq[(int64_t)q * p.dim + j], s_bh[j], s_bl[j]);
      // pass 1: nearest sample (first minimum in id order), this warp's share of the samples
      {
        float m = INFINITY;
        int nn = 0x7fffffff;
        for (int i = i0; i < i1; ++i) {
          const float4 v = s_x[i];
          const float dx = ql[0] - v.x, dy = ql[1] - v.y, dz = ql[2] - v.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (r2 < m) {
            m = r2;
            nn = i;
          }
        }
        s_red[w][0][lane] = m;
        s_nn[w][lane] = nn;
      }
      __syncthreads();
      float m = s_red[0][0][lane];
      int nn = s_nn[0][lane];
      for (int v = 1; v < kBW; ++v)
        if (s_red[v][0][lane] < m) {
          m = s_red[v][0][lane];
          nn = s_nn[v][lane];
        }
      const float zmin = sqrtf(m);
      __syncthreads();
      // pass 2: k'_i (kept for V[f]), grad f', softmin sums; exponents relative to the nearest sample
      {
        float G0 = 0.f, G1 = 0.f, G2 = 0.f, W = 0.f, HY = 0.f, T0 = 0.f, T1 = 0.f, T2 = 0.f;
        const float4 xn = s_x[nn];
        const float wx = 2.f * (ql[0] - xn.x), wy = 2.f * (ql[1] - xn.y), wz = 2.f * (ql[2] - xn.z);
        for (int i = i0; i < i1; ++i) {
          const float4 v = s_x[i];
          const float dx = ql[0] - v.x, dy = ql[1] - v.y, dz = ql[2] - v.z;
          const float e = excess_sq(v.x, v.y, v.z, xn.x, xn.y, xn.z, wx, wy, wz);
          const float r2 = m + e;
          const float z = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
          float kp, wg, y;
          kernel_terms<MATERN>(e, z, zmin, c1, (float)p.lambda, kp, wg, y);
          s_k[i * kBQ + lane] = kp;
          const float ak = v.w * wg;
          G0 = fmaf(ak, dx, G0);
          G1 = fmaf(ak, dy, G1);
          G2 = fmaf(ak, dz, G2);
          const float wt = ex2(-c2 * y);
          W += wt;
          HY = fmaf(wt, y, HY);
          const float tw = wt * wt * s_var[i];
          T0 += tw;
          T1 = fmaf(tw, y, T1);
          T2 = fmaf(tw * y, y, T2);
        }
        s_red[w][1][lane] = G0;
        s_red[w][2][lane] = G1;
        s_red[w][3][lane] = G2;
        s_red[w][4][lane] = W;
        s_red[w][5][lane] = HY;
        s_red[w][6][lane] = T0;
        s_red[w][7][lane] = T1;
        s_red[w][8][lane] = T2;
      }
      __syncthreads();
      const float vsum = (a.mask & KSDF_OUT_VAR_F) ? vf_rows(Lb, n, w, s_k, lane) : 0.f;
      __syncthreads();  // everyone has read s_red[.][1..8] and s_k
      s_red[w][0][lane] = vsum;
      __syncthreads();
      if (w == 0 && live) {
        float G0 = 0.f, G1 = 0.f, G2 = 0.f, W = 0.f, HY = 0.f, T0 = 0.f, T1 = 0.f, T2 = 0.f, VS = 0.f;
        for (int v = 0; v < kBW; ++v) {
          G0 += s_red[v][1][lane];
          G1 += s_red[v][2][lane];
          G2 += s_red[v][3][lane];
          W += s_red[v][4][lane];
          HY += s_red[v][5][lane];
          T0 += s_red[v][6][lane];
          T1 += s_red[v][7][lane];
          T2 += s_red[v][8][lane];
          VS += s_red[v][0][lane];
        }
        const float hy = HY / W;
        const float B = fmaf(as, hy, 1.f);
        const float vs = fmaxf((B * B * T0 - 2.f * B * as * T1 + as * as * T2) / (W * W), 0.f);
        const float vf = fmaxf(1.f - ex2(-2.f * c1 * (MATERN ? sqrtf(m) : m)) * VS, 0.f);
        float s = 1.f;
        if (a.sign) {
          s = a.sign[q] < 0 ? -1.f : 1.f;
        } else if (p.sign_mode == 1 && a.has_normals) {
          const float4 v = s_x[nn];
          const float4 nv = a.mnrm[m0 + nn];
          s = (nv.x * (ql[0] - v.x) + nv.y * (ql[1] - v.y) + nv.z * (ql[2] - v.z)) >= 0.f ? 1.f : -1.f;
        }
        uint32_t fl = a.qflag[q];
        const float gn = sqrtf(G0 * G0 + G1 * G1 + G2 * G2);
        if (a.mask & KSDF_OUT_SDF) sdf[q] = s * a.qu[q];
        if (a.mask & KSDF_OUT_GRAD) {
          const float gv[3] = {G0, G1, G2};
          const float ig = gn > 0.f ? s / gn : 0.f;
          for (int j = 0; j < p.dim; ++j) grad[(int64_t)q * p.dim + j] = gv[j] * ig;
        }
        if (!(gn > 0.f)) fl |= KSDF_FLAG_ZERO_GRAD;
        if (a.mask & KSDF_OUT_VAR_SDF) var_sdf[q] = vs;
        if (a.mask & KSDF_OUT_VAR_F) var_f[q] = vf;
        if (a.mask & KSDF_OUT_WINNER) winner[q] = g;
        if (a.mask & KSDF_OUT_FLAGS) flags[q] = fl;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Q6 with the variance contraction on the tensor cores (cells of N <= kTcMaxN samples).  A tile is up to
// 128 queries of one winner cell, one thread per query (= row m of the MMA and TMEM lane m).  The thread
// finds the nearest sample, then walks the samples in steps of 8 -- k'_i, grad f', the softmin sums, two
// samples per packed FP32x2 instruction -- and writes the step's k' values as the A operand (TF32 hi = rna(k'),
// lo = rna(k' - hi)).  The B operand of the step -- 8 columns of L^-1, i.e. rows j of L^-1 restricted to the
// step's K range -- arrives by a TMA bulk copy from the cell's FP32 tensor-core image, and the producer warp
// splits it in place (hi = rna(x), lo = rna(x - hi) beside it).  One thread issues
//   D[:, n0:Np] (+)= A_hi B_hi + A_hi B_lo + A_lo B_hi   (tcgen05.mma kind::tf32, M = 128, K = 8),
// with n0 = 16 floor(8 c / 16) skipping the zero upper blocks of L^-1; D = K' L^-T lives in TMEM.  A ring of
// three A stages and a ring of three B stages (the copy for step c + 2 is issued with the MMA of step c), each
// with its mbarriers.  Finally each thread reads its TMEM row, |V_row|^2, and
// V[f] = 1 - e^{-2 lambda d^2} |V_row|^2.  While the query warps finish a tile, the producer warp fetches the
// next one into the other of two tile buffers: its samples by TMA, their variances, the padding, and each
// query's index, cell-local position, flags and u.  A warp whose 32 rows hold no query of the tile zeroes its
// A rows once and sits the tile out.

constexpr int kTcM = 128;
constexpr int kTcThreads = kTcM + 32;  // a query thread per row, one producer warp
constexpr float kTcPad = 1e7f;        // cell-local coordinate of the padding samples (n .. Kp): far from every query
// cells up to the context's qt_tc_small (96 by default; a multiple of 16, at most 128) take 128 TMEM columns
// (four CTAs per SM), the larger ones up to kTcMaxN 256
constexpr int kTcStages = 3;   // A operand ring
constexpr int kTcBStages = 3;  // B operand ring: a step's B copy is issued two steps ahead
constexpr uint32_t kTcStageA = 8192;  // A hi + lo: 2 K-quads x 128 rows x 16 B, twice

__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor, K-major without swizzle: lbo = bytes between core matrices along K,
// sbo = bytes between 8-row groups
__device__ inline uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor: D FP32, A and B TF32, both K-major, N and M
__device__ inline uint32_t umma_idesc_tf32(int n, int m) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ inline void umma_tf32(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ inline void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ inline float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// sum of squares of 16 consecutive TMEM columns of this thread's lane
__device__ inline float tmem_sumsq16(uint32_t taddr) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) s = fmaf(__uint_as_float(r[k]), __uint_as_float(r[k]), s);
  return s;
}

struct TcArgs {
  const int4* tiles;
  const int64_t* n_tiles;
  int* counter;
  const int64_t* ltc_off;
  const float* ltc;  // FP32 images of L^-1 (K-major B operand)
};

// shared memory of one CTA: two tile buffers, each [kcap] samples (float4), [kcap] var, [kTcM] query records
// (cell-local position and u as a float4, index and flags as a uint2) | A ring (hi, lo) | B ring (hi, lo)
__host__ __device__ inline size_t tc_bstage_bytes(int npm) { return 64u * (size_t)npm; }
__host__ __device__ inline size_t tc_head_bytes(int kcap) {
  return ((size_t)40 * kcap + (size_t)2 * kTcM * 24 + 1023) & ~(size_t)1023;
}
__host__ __device__ inline size_t tc_smem_bytes(int kcap) {
  return tc_head_bytes(kcap) + kTcStages * (size_t)kTcStageA + kTcBStages * tc_bstage_bytes(tc_np(kcap));
}

__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ inline void mbar_arrive_n(uint64_t* bar, uint32_t n) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(n) : "memory");
}

// Warp roles: warps 0..3 hold the tile's 128 queries (one per thread, = row m of the MMA and TMEM lane m) and
// write the A operand step by step, signalling bar_full; warp 4 is the producer: it fetches tiles, streams the B
// chunks by TMA, splits them, and (lane 0) issues the MMAs once a step's A is written.  The query threads wait
// only to reuse an A stage (its MMA done) and for the tile's last MMA.
template <bool MATERN>
__global__ void __launch_bounds__(kTcThreads, 4) k_phaseB_tc(PhaseBArgs a, TcArgs t, const float* xq, Params p,
                                                             float* sdf, float* grad, float* var_sdf, float* var_f,
                                                             int32_t* winner, uint32_t* flags, int kcap,
                                                             uint32_t ncols) {
  extern __shared__ __align__(1024) unsigned char smb[];
  // bar_x: a sample buffer's copy; bar_full / bar_mma: A ring (operands written, MMA done); bar_tma / bar_bfree:
  // B ring (copy landed, MMA done)
  __shared__ __align__(8) uint64_t bar_x[2], bar_full[kTcStages], bar_mma[kTcStages], bar_tma[kTcBStages],
      bar_bfree[kTcBStages];
  __shared__ uint32_t s_tmem;
  __shared__ int4 s_tile[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = warp == kTcM / 32;
  const int npm = tc_np(kcap);
  float4* s_xb = reinterpret_cast<float4*>(smb);             // [2][kcap]
  float4* s_qpb = s_xb + 2 * kcap;                           // [2][kTcM]: cell-local query position, u
  uint2* s_qib = reinterpret_cast<uint2*>(s_qpb + 2 * kTcM);  // [2][kTcM]: query index, flags
  float* s_varb = reinterpret_cast<float*>(s_qib + 2 * kTcM);  // [2][kcap]
  unsigned char* stg = smb + tc_head_bytes(kcap);
  unsigned char* ringb = stg + kTcStages * kTcStageA;
  const uint32_t bstage_bytes = (uint32_t)tc_bstage_bytes(npm);
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) mbar_init(&bar_x[b], 1);
    for (int s = 0; s < kTcBStages; ++s) {
      mbar_init(&bar_tma[s], 1);
      mbar_init(&bar_bfree[s], 1);
    }
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&bar_mma[s], 1);
      mbar_init(&bar_full[s], kTcM);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const float c1 = (float)p.lambda * kLog2e;
  const float as = (float)p.alpha_s;
  const float c2 = as * kLog2e;
  const float lam = (float)p.lambda;
  const int64_t ntiles = *t.n_tiles;
  // The producer warp takes the next tile and stages it into tile buffer b in three parts, so that the latency of
  // its loads overlaps the current tile's steps: begin -- the tile index, the samples by TMA (lane 0), the
  // variances and the padding samples n .. Kp - 1 (far away, zero weight and variance, so that every step takes
  // 8 whole samples), the query indices into registers; middle -- the loads that depend on the query indices;
  // end -- the query records into shared memory.
  constexpr int kRK = kTcM / 32;
  int4 f_tl = make_int4(-1, 0, 0, 0);
  float f_x[kRK][3], f_u[kRK];
  int f_q[kRK];
  uint32_t f_fl[kRK];
  auto fetch_begin = [&](int b) {
    if (lane == 0) {
      const int ti = atomicAdd(t.counter, 1);
      f_tl = make_int4(-1, 0, 0, 0);
      if (ti < ntiles) {
        f_tl = t.tiles[ti];
        const int n = a.cell_n[f_tl.x];
        mbar_expect_tx(&bar_x[b], (uint32_t)n * 16u);
        bulk_g2s(s_xb + b * kcap, a.mf4 + a.ts_off[f_tl.x], (uint32_t)n * 16u, &bar_x[b]);
      }
      s_tile[b] = f_tl;
    }
    f_tl.x = __shfl_sync(0xFFFFFFFFu, f_tl.x, 0);
    f_tl.y = __shfl_sync(0xFFFFFFFFu, f_tl.y, 0);
    f_tl.z = __shfl_sync(0xFFFFFFFFu, f_tl.z, 0);
    if (f_tl.x >= 0) {
      const int n = a.cell_n[f_tl.x];
      const int64_t m0 = a.ts_off[f_tl.x];
#pragma unroll
      for (int k = 0; k < kRK; ++k) f_q[k] = lane + 32 * k < f_tl.z ? a.sorted_w[f_tl.y + lane + 32 * k] : 0;
      float* sv = s_varb + b * kcap;
      for (int i = lane; i < n; i += 32) sv[i] = a.mvar[m0 + i];  // not 16-byte aligned in HBM: plain loads
      for (int i = n + lane; i < tc_kp(n); i += 32) {
        s_xb[b * kcap + i] = make_float4(kTcPad, kTcPad, kTcPad, 0.f);
        sv[i] = 0.f;
      }
    }
  };
  auto fetch_mid = [&]() {
    if (f_tl.x < 0) return;
#pragma unroll
    for (int k = 0; k < kRK; ++k) {
      f_x[k][0] = f_x[k][1] = f_x[k][2] = 0.f;
      f_u[k] = 0.f;
      f_fl[k] = 0;
      if (lane + 32 * k < f_tl.z) {
        const int q = f_q[k];
#pragma unroll
        for (int j = 0; j < 3; ++j)
          if (j < p.dim) f_x[k][j] = xq[(int64_t)q * p.dim + j];
        f_u[k] = a.qu[q];
        f_fl[k] = a.qflag[q];
      }
    }
  };
  auto fetch_end = [&](int b) {
    if (f_tl.x < 0) return;
    float bh[3], bl[3];
    int cc[3];
    unpack_key(a.cell_key[f_tl.x], cc[0], cc[1], cc[2]);
#pragma unroll
    for (int j = 0; j < 3; ++j) base_split(p.o[j], cc[j], p.h, bh[j], bl[j]);
#pragma unroll
    for (int k = 0; k < kRK; ++k) {
      const int r = lane + 32 * k;
      if (r < f_tl.z) {
        float ql[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; ++j)
          if (j < p.dim) ql[j] = local32(f_x[k][j], bh[j], bl[j]);
        s_qpb[b * kTcM + r] = make_float4(ql[0], ql[1], ql[2], f_u[k]);
        s_qib[b * kTcM + r] = make_uint2((uint32_t)f_q[k], f_fl[k]);
      }
    }
  };
  if (producer) {
    fetch_begin(0);
    fetch_mid();
    fetch_end(0);
  }
  __syncthreads();
  uint32_t gstep = 0;  // global step counter: A stage gstep % 3, B stage gstep % 4
  bool fail = false;
  for (int it = 0;; ++it) {
    const int buf = it & 1;
    const int4 tile = s_tile[buf];
    if (tile.x < 0) break;
    const float4* s_x = s_xb + buf * kcap;
    const float* s_var = s_varb + buf * kcap;
    const int g = tile.x;
    const int n = a.cell_n[g];
    const int64_t m0 = a.ts_off[g];
    const int np16 = tc_np(n), nsteps = tc_kp(n) >> 3;
    if (producer) {
      const float* img = t.ltc + t.ltc_off[g];
      // (lane 0) B chunk of step c (FP32) into the B slot of global step gs: both K-quads, rows n0 .. np16-1, once
      // the slot's previous MMA (global step gs - kTcBStages) has finished reading it
      auto issue_b = [&](int c, uint32_t gs) {
        const int s = (int)(gs % kTcBStages);
        if (gs >= (uint32_t)kTcBStages && !mbar_wait_one(&bar_bfree[s], ((gs / kTcBStages) - 1) & 1)) fail = true;
        const int n0 = (c >> 1) << 4;
        const uint32_t bytes = (uint32_t)(np16 - n0) * 16u;
        unsigned char* bb = ringb + (size_t)s * bstage_bytes;
        mbar_expect_tx(&bar_tma[s], 2u * bytes);
        for (int qd = 0; qd < 2; ++qd)
          bulk_g2s(bb + (size_t)qd * npm * 16 + (size_t)n0 * 16, img + ((int64_t)(2 * c + qd) * np16 + n0) * 4,
                   bytes, &bar_tma[s]);
      };
      if (lane == 0)
        for (int c = 0; c < nsteps && c < kTcBStages - 1; ++c) issue_b(c, gstep + c);
      fetch_begin(buf ^ 1);  // the next tile, into the other buffer (its last readers finished before the
                             // previous barrier)
      for (int c = 0; c < nsteps && !fail; ++c) {
        const uint32_t gs = gstep + c;
        const int s = (int)(gs % kTcStages), sb = (int)(gs % kTcBStages);
        const int n0 = (c >> 1) << 4, rows = np16 - n0;
        // the step's B has landed: split it in place, TF32 hi = rna(x), lo = rna(x - hi) npm * 32 bytes further
        if (!mbar_wait_one(&bar_tma[sb], (gs / kTcBStages) & 1)) fail = true;
        {
          unsigned char* bb = ringb + (size_t)sb * bstage_bytes + (size_t)n0 * 16;
          for (int u = lane; u < 2 * rows; u += 32) {
            const int qd = u >= rows ? 1 : 0;
            float4* hp = reinterpret_cast<float4*>(bb + (size_t)qd * npm * 16 + (size_t)(u - qd * rows) * 16);
            const float4 v = *hp;
            const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
            *hp = h;
            *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(hp) + (size_t)npm * 32) =
                make_float4(tf32_rna(v.x - h.x), tf32_rna(v.y - h.y), tf32_rna(v.z - h.z), tf32_rna(v.w - h.w));
          }
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
          // A written by the query threads
          if (!mbar_wait_one(&bar_full[s], (gs / kTcStages) & 1)) fail = true;
          if (!fail) {
            tc_fence_after();
            unsigned char* sa = stg + (size_t)s * kTcStageA;
            const uint32_t idesc = umma_idesc_tf32(rows, kTcM);
            const uint32_t a_hi = smem_u32(sa), a_lo = a_hi + 4096;
            const uint32_t b_hi = smem_u32(ringb + (size_t)sb * bstage_bytes) + (uint32_t)n0 * 16;
            const uint32_t b_lo = b_hi + (uint32_t)npm * 32;
            const uint32_t d = tmem + (uint32_t)n0;
            const uint32_t lbo_b = (uint32_t)npm * 16;
            umma_tf32(d, umma_desc(a_hi, 2048, 128), umma_desc(b_hi, lbo_b, 128), idesc, c > 0 ? 1u : 0u);
            umma_tf32(d, umma_desc(a_hi, 2048, 128), umma_desc(b_lo, lbo_b, 128), idesc, 1u);
            umma_tf32(d, umma_desc(a_lo, 2048, 128), umma_desc(b_hi, lbo_b, 128), idesc, 1u);
            umma_commit(&bar_mma[s]);
            umma_commit(&bar_bfree[sb]);
            if (c + kTcBStages - 1 < nsteps) issue_b(c + kTcBStages - 1, gs + kTcBStages - 1);
          }
        }
        fail = __any_sync(0xFFFFFFFFu, fail);
        if (c == 0) fetch_mid();
      }
      if (!fail) fetch_end(buf ^ 1);
    } else {
      const bool live = tid < tile.z;
      const bool wlive = warp * 32 < tile.z;  // the warp holds at least one query (uniform over the warp)
      const int nlw = (tile.z + 31) >> 5;     // live warps: 0 .. nlw - 1
      const int r = live ? tid : 0;           // a dead row of a live warp computes row 0's query, unused
      const float4 qp = s_qpb[buf * kTcM + r];
      const uint2 qi = s_qib[buf * kTcM + r];
      const int q = (int)qi.x;
      const float ql[3] = {qp.x, qp.y, qp.z};
      const float qu = qp.w;
      uint32_t fl = qi.y;
      float m = INFINITY;
      int nn = 0;
      if (wlive) {
        if (!mbar_wait_one(&bar_x[buf], (it >> 1) & 1)) fail = true;
        // pass 1: nearest sample (first minimum in id order), two samples per packed instruction (sample n, when
        // n is odd, is a far padding sample)
        const unsigned long long QX = f2pack(ql[0], ql[0]), QY = f2pack(ql[1], ql[1]), QZ = f2pack(ql[2], ql[2]);
        for (int i = 0; i < n; i += 2) {
          const float4 v0 = s_x[i], v1 = s_x[i + 1];
          const unsigned long long dx = f2sub(QX, f2pack(v0.x, v1.x)), dy = f2sub(QY, f2pack(v0.y, v1.y));
          const unsigned long long dz = f2sub(QZ, f2pack(v0.z, v1.z));
          const float2 r2 = f2unpack(f2fma(dx, dx, f2fma(dy, dy, f2mul(dz, dz))));
          if (r2.x < m) {
            m = r2.x;
            nn = i;
          }
          if (r2.y < m) {
            m = r2.y;
            nn = i + 1;
          }
        }
      } else {
        // no query in these rows: zero A (hi and lo) in every stage once -- no MMA of the previous tile reads
        // them any more (every thread waited for its last MMA), and none of this tile's is issued before the
        // live warps arrive, after the barrier below -- then sit the tile out
        for (int s = 0; s < kTcStages; ++s) {
          unsigned char* sa = stg + (size_t)s * kTcStageA;
#pragma unroll
          for (int qd = 0; qd < 2; ++qd) {
            *reinterpret_cast<float4*>(sa + qd * 2048 + tid * 16) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(sa + 4096 + qd * 2048 + tid * 16) = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
        fence_proxy_async();
      }
      asm volatile("bar.sync 1, %0;" ::"r"(kTcM) : "memory");  // the dead warps' zero rows written
      if (wlive) {
        const float zmin = sqrtf(m);
        // exponents relative to the nearest sample (excess_sq); the per-query constants of the packed loop
        const float4 xn = s_x[nn];
        const float wx = 2.f * (ql[0] - xn.x), wy = 2.f * (ql[1] - xn.y), wz = 2.f * (ql[2] - xn.z);
        const unsigned long long QX = f2pack(ql[0], ql[0]), QY = f2pack(ql[1], ql[1]), QZ = f2pack(ql[2], ql[2]);
        const unsigned long long NX = f2pack(xn.x, xn.x), NY = f2pack(xn.y, xn.y), NZ = f2pack(xn.z, xn.z);
        const unsigned long long WX = f2pack(wx, wx), WY = f2pack(wy, wy), WZ = f2pack(wz, wz);
        const unsigned long long M2 = f2pack(m, m), ZM = f2pack(zmin, zmin);
        const unsigned long long NC1 = f2pack(-c1, -c1), NC2 = f2pack(-c2, -c2), LAM = f2pack(lam, lam);
        const unsigned long long ONE = f2pack(1.f, 1.f);
        unsigned long long G0 = 0ull, G1 = 0ull, G2 = 0ull, W = 0ull, HY = 0ull, T0 = 0ull, T1 = 0ull, T2 = 0ull;
        for (int c = 0; c < nsteps; ++c) {
          const uint32_t gs = gstep + c;
          const int s = (int)(gs % kTcStages);
          unsigned char* sa = stg + (size_t)s * kTcStageA;
          // the stage's previous MMA has finished reading A
          if (gs >= (uint32_t)kTcStages && !mbar_wait_one(&bar_mma[s], ((gs / kTcStages) - 1) & 1)) fail = true;
          float kv[8];
          // samples 8c .. 8c+7 in pairs: k'_i, grad f', the softmin sums
#pragma unroll
          for (int u = 0; u < 8; u += 2) {
            const int i = 8 * c + u;
            const float4 v0 = s_x[i], v1 = s_x[i + 1];
            const float2 vr = *reinterpret_cast<const float2*>(s_var + i);
            const unsigned long long X = f2pack(v0.x, v1.x), Y = f2pack(v0.y, v1.y), Z = f2pack(v0.z, v1.z);
            const unsigned long long dx = f2sub(QX, X), dy = f2sub(QY, Y), dz = f2sub(QZ, Z);
            // excess_sq, both samples
            const unsigned long long ax = f2sub(X, NX), ay = f2sub(Y, NY), az = f2sub(Z, NZ);
            const unsigned long long e = f2fma(ax, f2sub(ax, WX), f2fma(ay, f2sub(ay, WY), f2mul(az, f2sub(az, WZ))));
            const unsigned long long r2 = f2add(M2, e);
            const float2 r2s = f2unpack(r2);
            const unsigned long long z =
                f2mul(r2, f2pack(rsqrtf(fmaxf(r2s.x, 1e-30f)), rsqrtf(fmaxf(r2s.y, 1e-30f))));
            unsigned long long kp, wg, y;
            if (MATERN) {
              // y = max(e, 0) / (z + zmin), wg = 2^{-c1 y}, k' = (1 + lambda z) wg
              const float2 es = f2unpack(e), den = f2unpack(f2add(z, ZM));
              y = f2pack(den.x > 0.f ? fmaxf(es.x, 0.f) * __frcp_rn(den.x) : 0.f,
                         den.y > 0.f ? fmaxf(es.y, 0.f) * __frcp_rn(den.y) : 0.f);
              const float2 ey = f2unpack(f2mul(NC1, y));
              wg = f2pack(ex2(ey.x), ex2(ey.y));
              kp = f2mul(f2fma(LAM, z, ONE), wg);
            } else {
              const float2 ee = f2unpack(f2mul(NC1, e));
              kp = f2pack(ex2(ee.x), ex2(ee.y));
              wg = kp;
              const float2 ys = f2unpack(f2sub(z, ZM));
              y = f2pack(fmaxf(ys.x, 0.f), fmaxf(ys.y, 0.f));
            }
            const unsigned long long ak = f2mul(f2pack(v0.w, v1.w), wg);
            G0 = f2fma(ak, dx, G0);
            G1 = f2fma(ak, dy, G1);
            G2 = f2fma(ak, dz, G2);
            const float2 cy = f2unpack(f2mul(NC2, y));
            // softmin weights of the padding samples masked
            const unsigned long long wt = f2pack(i < n ? ex2(cy.x) : 0.f, i + 1 < n ? ex2(cy.y) : 0.f);
            const float2 k2 = f2unpack(kp);
            W = f2add(W, wt);
            HY = f2fma(wt, y, HY);
            const unsigned long long tw = f2mul(f2mul(wt, wt), f2pack(vr.x, vr.y));
            T0 = f2add(T0, tw);
            T1 = f2fma(tw, y, T1);
            T2 = f2fma(f2mul(tw, y), y, T2);
            kv[u] = live ? k2.x : 0.f;
            kv[u + 1] = live ? k2.y : 0.f;
          }
          // A operand (row tid): K-quad q at q * 2048 + tid * 16; lo part 4096 bytes further
#pragma unroll
          for (int qd = 0; qd < 2; ++qd) {
            float hv[4], lv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              hv[e] = tf32_rna(kv[4 * qd + e]);
              lv[e] = tf32_rna(kv[4 * qd + e] - hv[e]);
            }
            *reinterpret_cast<float4*>(sa + qd * 2048 + tid * 16) = make_float4(hv[0], hv[1], hv[2], hv[3]);
            *reinterpret_cast<float4*>(sa + 4096 + qd * 2048 + tid * 16) = make_float4(lv[0], lv[1], lv[2], lv[3]);
          }
          fence_proxy_async();
          mbar_arrive(&bar_full[s]);
          if (tid == 0 && nlw < kTcM / 32) mbar_arrive_n(&bar_full[s], 32u * (kTcM / 32 - nlw));  // the dead warps'
        }
        // the tile's last MMA (and so all of them) has finished
        {
          const uint32_t gl = gstep + nsteps - 1;
          if (!mbar_wait_one(&bar_mma[gl % kTcStages], (gl / kTcStages) & 1)) fail = true;
        }
        tc_fence_after();
        float VS = 0.f;
        {
          const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
          for (int c0 = 0; c0 < np16; c0 += 16) VS += tmem_sumsq16(ta + (uint32_t)c0);
        }
        const float2 g0 = f2unpack(G0), g1 = f2unpack(G1), g2 = f2unpack(G2), w2 = f2unpack(W), hy2 = f2unpack(HY);
        const float2 t0 = f2unpack(T0), t1 = f2unpack(T1), t2 = f2unpack(T2);
        const float gx = g0.x + g0.y, gy = g1.x + g1.y, gz = g2.x + g2.y, Ws = w2.x + w2.y;
        const float T0s = t0.x + t0.y, T1s = t1.x + t1.y, T2s = t2.x + t2.y;
        if (live && !fail) {
          const float hy = (hy2.x + hy2.y) / Ws;
          const float B = fmaf(as, hy, 1.f);
          const float vs = fmaxf((B * B * T0s - 2.f * B * as * T1s + as * as * T2s) / (Ws * Ws), 0.f);
          const float vf = fmaxf(1.f - ex2(-2.f * c1 * (MATERN ? zmin : m)) * VS, 0.f);
          float sg = 1.f;
          if (a.sign) {
            sg = a.sign[q] < 0 ? -1.f : 1.f;
          } else if (p.sign_mode == 1 && a.has_normals) {
            const float4 nv = a.mnrm[m0 + nn];
            sg = (nv.x * (ql[0] - xn.x) + nv.y * (ql[1] - xn.y) + nv.z * (ql[2] - xn.z)) >= 0.f ? 1.f : -1.f;
          }
          const float gn = sqrtf(gx * gx + gy * gy + gz * gz);
          if (a.mask & KSDF_OUT_SDF) sdf[q] = sg * qu;
          if (a.mask & KSDF_OUT_GRAD) {
            const float ig = gn > 0.f ? sg / gn : 0.f;
            grad[(int64_t)q * p.dim + 0] = gx * ig;
            grad[(int64_t)q * p.dim + 1] = gy * ig;
            if (p.dim == 3) grad[(int64_t)q * p.dim + 2] = gz * ig;
          }
          if (!(gn > 0.f)) fl |= KSDF_FLAG_ZERO_GRAD;
          if (a.mask & KSDF_OUT_VAR_SDF) var_sdf[q] = vs;
          if (a.mask & KSDF_OUT_VAR_F) var_f[q] = vf;
          if (a.mask & KSDF_OUT_WINNER) winner[q] = g;
          if (a.mask & KSDF_OUT_FLAGS) flags[q] = fl;
        }
      }
    }
    gstep += (uint32_t)nsteps;
    tc_fence_before();
    if (__syncthreads_or(fail)) {
      fail = true;
      break;
    }
  }
  if (fail && tid == 0) atomicOr(a.st, ST_TIMEOUT);
  // on a timeout, give the last committed MMAs a bounded chance to finish before the TMEM is released
  if (fail && gstep > 0 && tid == 0) {
    const uint32_t gl = gstep - 1;
    mbar_wait_one(&bar_mma[gl % kTcStages], (gl / kTcStages) & 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// Diagnostic of the bounded waits (ksdf_wait_diagnostic): one CTA shaped like the tensor-core phase B (TMEM
// allocated by warp 0, an mbarrier initialised by thread 0) waits on an mbarrier that nothing will complete --
// no bulk copy or MMA is issued, so nothing is in flight -- for at most `spins` polls, then leaves the way a
// production wait that gives up does: ST_TIMEOUT in the status word, the TMEM released, the kernel returned.
__global__ void __launch_bounds__(64) k_wait_diag(uint32_t spins, uint32_t* st) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(32u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  bool done = false;
  for (uint32_t it = 0; it < spins && !done; ++it) done = mbar_try_wait(&bar, 0);
  if (__syncthreads_or(!done) && tid == 0) atomicOr(st, ST_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u) : "memory");
}

// tile counts of the cells in three lists by cell size: (0, n1], (n1, n2] (tiles of T12 queries) and larger
// (tiles of T3 queries)
__global__ void k_ntiles3(const int64_t* cnt, const int32_t* cell_n, int64_t n, int n1, int n2, int T12, int T3,
                          int64_t* nt0, int64_t* nt1, int64_t* nt2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cn = cell_n[i];
  const int cl = cn <= n1 ? 0 : (cn <= n2 ? 1 : 2);
  const int T = cl == 2 ? T3 : T12;
  const int64_t t = (cnt[i] + T - 1) / T;
  nt0[i] = cl == 0 ? t : 0;
  nt1[i] = cl == 1 ? t : 0;
  nt2[i] = cl == 2 ? t : 0;
}

__global__ void k_make_tiles3(const int64_t* cnt, const int64_t* off, const int64_t* toff0, const int64_t* toff1,
                              const int64_t* toff2, const int32_t* cell_n, int n1, int n2, int64_t ngroups, int T12,
                              int T3, int4* tiles0, int4* tiles1, int4* tiles2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ngroups) return;
  const int64_t c = cnt[i];
  const int cn = cell_n[i];
  const int cl = cn <= n1 ? 0 : (cn <= n2 ? 1 : 2);
  const int T = cl == 2 ? T3 : T12;
  int4* dst = cl == 0 ? tiles0 + toff0[i] : (cl == 1 ? tiles1 + toff1[i] : tiles2 + toff2[i]);
  for (int64_t k = 0; k * T < c; ++k)
    dst[k] = make_int4((int)i, (int)(off[i] + k * T), (int)(c - k * T < T ? c - k * T : T), 0);
}

// Q6 (plain path): binary64 throughout; V[f] by forward substitution with the stored Cholesky factor,
// v = L^{-1} k' (in place over k'), V[f] = 1 - e^{-2 lambda d^2} |v|^2.
template <bool MATERN>
__global__ void __launch_bounds__(kTB64) k_phaseB64(PhaseBArgs a, const double* xq, Params p, double* sdf,
                                                    double* grad, double* var_sdf, double* var_f, int32_t* winner,
                                                    uint32_t* flags) {
  extern __shared__ __align__(128) D4 s_d[];  // [n_max] samples, [n_max] var (double), [n_max][kTB64] k'
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_tile;
  const int tid = threadIdx.x;
  double* s_var = reinterpret_cast<double*>(s_d + p.n_max);
  double* s_k = s_var + p.n_max;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_proxy_async();
  }
  __syncthreads();
  const double lam = p.lambda, as = p.alpha_s;
  uint32_t phase = 0;
  const int64_t ntiles = *a.n_tiles;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const int4 tile = a.tiles[t];
    const int g = tile.x;
    const int n = a.cell_n[g];
    const int64_t m0 = a.ts_off[g];
    if (tid == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bar, (uint32_t)n * 32u);
      bulk_g2s(s_d, a.md4 + m0, (uint32_t)n * 32u, &bar);
    }
    for (int i = tid; i < n; i += blockDim.x) s_var[i] = (double)a.mvar[m0 + i];
    int cc[3];
    unpack_key(a.cell_key[g], cc[0], cc[1], cc[2]);
    const bool live = tid < tile.z;
    const int q = live ? a.sorted_w[tile.y + tid] : 0;
    double ql[3] = {0, 0, 0};
    if (live)
      for (int j = 0; j < p.dim; ++j) ql[j] = __dsub_rn(xq[(int64_t)q * p.dim + j], cell_base(p.o[j], cc[j], p.h));
    if (!mbar_wait_all(&bar, phase)) {
      if (tid == 0) atomicOr(a.st, ST_TIMEOUT);
      return;
    }
    phase ^= 1;
    if (live) {
      double m = INFINITY;
      int nn = 0;
      for (int i = 0; i < n; ++i) {
        const D4 v = s_d[i];
        const double dx = ql[0] - v.x, dy = ql[1] - v.y, dz = ql[2] - v.z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < m) {
          m = r2;
          nn = i;
        }
      }
      const double zmin = sqrt(m);
      double G0 = 0, G1 = 0, G2 = 0, W = 0, HZ = 0;
      for (int i = 0; i < n; ++i) {
        const D4 v = s_d[i];
        const double dx = ql[0] - v.x, dy = ql[1] - v.y, dz = ql[2] - v.z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        // k' and the factor w of its gradient (grad k' = -c w (x - x_i)): RBF w = k'; Matern w = e^{-lambda (r - d)}
        double kp, wg;
        if (MATERN) {
          const double r = sqrt(r2);
          wg = exp(-lam * (r - zmin));
          kp = (1.0 + lam * r) * wg;
        } else {
          kp = exp(-lam * (r2 - m));
          wg = kp;
        }
        s_k[i * kTB64 + tid] = kp;
        const double ak = v.w * wg;
        G0 += ak * dx;
        G1 += ak * dy;
        G2 += ak * dz;
        const double z = sqrt(r2);
        const double wt = exp(-as * (z - zmin));
        W += wt;
        HZ += wt * z;
      }
      const double h = HZ / W;
      double vs = 0.0;
      for (int i = 0; i < n; ++i) {
        const D4 v = s_d[i];
        const double dx = ql[0] - v.x, dy = ql[1] - v.y, dz = ql[2] - v.z;
        const double z = sqrt(dx * dx + dy * dy + dz * dz);
        const double si = exp(-as * (z - zmin)) / W;
        const double tt = as * (h - z) + 1.0;
        vs += si * si * tt * tt * s_var[i];
      }
      double vf = 1.0;
      if (a.mask & KSDF_OUT_VAR_F) {
        const double* L = a.chol64 + a.chol_off[g];
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
          const double* Li = L + (int64_t)i * (i + 1) / 2;
          double sm = s_k[i * kTB64 + tid];
          for (int j = 0; j < i; ++j) sm = fma(-Li[j], s_k[j * kTB64 + tid], sm);
          const double v = sm / Li[i];
          s_k[i * kTB64 + tid] = v;
          acc = fma(v, v, acc);
        }
        vf = fmax(1.0 - exp(-2.0 * lam * (MATERN ? zmin : m)) * acc, 0.0);
      }
      double s = 1.0;
      if (a.sign) {
        s = a.sign[q] < 0 ? -1.0 : 1.0;
      } else if (p.sign_mode == 1 && a.has_normals) {
        const D4 v = s_d[nn];
        const float4 nv = a.mnrm[m0 + nn];
        const double dot = nv.x * (ql[0] - v.x) + nv.y * (ql[1] - v.y) + nv.z * (ql[2] - v.z);
        s = dot >= 0.0 ? 1.0 : -1.0;
      }
      uint32_t fl = a.qflag[q];
      const double gn = sqrt(G0 * G0 + G1 * G1 + G2 * G2);
      if (a.mask & KSDF_OUT_SDF) sdf[q] = s * a.qu64[q];
      if (a.mask & KSDF_OUT_GRAD) {
        const double gv[3] = {G0, G1, G2};
        for (int j = 0; j < p.dim; ++j) grad[(int64_t)q * p.dim + j] = gn > 0.0 ? s * gv[j] / gn : 0.0;
      }
      if (!(gn > 0.0)) fl |= KSDF_FLAG_ZERO_GRAD;
      if (a.mask & KSDF_OUT_VAR_SDF) var_sdf[q] = vs;
      if (a.mask & KSDF_OUT_VAR_F) var_f[q] = vf;
      if (a.mask & KSDF_OUT_WINNER) winner[q] = g;
      if (a.mask & KSDF_OUT_FLAGS) flags[q] = fl;
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Q7 (optional output): SDF-gradient variance, Sec. IV-B.3 and App. C
//
// Per tile of queries of one winner cell, one thread per query over the cell's samples (staged in shared
// memory with their variances), three passes:
//   1. z_min;
//   2. with y_i = z_i - z_min and e_i = e^{-a y_i} (the softmin's common factor e^{-a z_min} divided out):
//      W = sum e_i, HY = sum e_i y_i, SV = sum e_i v_i, SYV = sum e_i y_i v_i; then s_i = e_i / W,
//      B = a HY / W + 1 (so that l_i = s_i (a s^T z - a z_i + 1) = s_i (B - a y_i)), V s = SV / W and
//      g = sum_i l_i v_i = (B SV - a SYV) / W;
//   3. V[grad_k u] = sum_i sigma_i^2 |grad_{x_i} g_k|^2 with grad_{x_i} g_k = (a w_k + c_i v_k) v_i - c_i e_k,
//      w = l_i (v_i - V s) + s_i (v_i - g), c_i = l_i / z_i; since |v_i| = 1 the squared norm is
//      a^2 w_k^2 + c_i^2 (1 - v_k^2), and 1 - v_k^2 is formed as (r^2 - r_k^2) / r^2 (no cancellation).
// A query on a sample (r^2 = 0) gets +inf.  FP32 (mixed path; ex2.approx for the weights) or FP64.
constexpr int kVG = 128;

struct VarGradArgs {
  const int4* tiles;
  const int64_t* n_tiles;
  int* counter;
  const int32_t* sorted_w;
  const int64_t* ts_off;
  const int32_t* cell_n;
  const uint64_t* cell_key;
  const float4* mf4;
  const D4* md4;
  const float* mvar;
};

template <class T>
struct VgRec;
template <>
struct VgRec<float> {
  typedef float4 R;
};
template <>
struct VgRec<double> {
  typedef D4 R;
};

template <class T>
__device__ __forceinline__ T vg_exp(T x);  // e^x for x <= 0
template <>
__device__ __forceinline__ float vg_exp<float>(float x) { return ex2(x * kLog2e); }
template <>
__device__ __forceinline__ double vg_exp<double>(double x) { return exp(x); }

template <class T>
__global__ void __launch_bounds__(kVG) k_var_grad(VarGradArgs a, const T* xq, Params p, T* var_grad) {
  typedef typename VgRec<T>::R R;
  extern __shared__ __align__(32) unsigned char vg_sm[];
  R* sx = reinterpret_cast<R*>(vg_sm);  // cell-local (x, y, z) and sigma^2
  __shared__ int s_tile;
  __shared__ int s_cc[3];
  __shared__ float s_bh[3], s_bl[3];
  const T al = (T)p.alpha_s;
  const int dim = p.dim;
  const int64_t ntiles = *a.n_tiles;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.counter, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const int4 tile = a.tiles[t];
    const int g = tile.x, n = a.cell_n[g];
    const int64_t m0 = a.ts_off[g];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      R v;
      if constexpr (sizeof(T) == 4) v = a.mf4[m0 + i];
      else v = a.md4[m0 + i];
      v.w = (T)a.mvar[m0 + i];
      sx[i] = v;
    }
    if (threadIdx.x == 0) unpack_key(a.cell_key[g], s_cc[0], s_cc[1], s_cc[2]);
    __syncthreads();
    if (threadIdx.x < 3) base_split(p.o[threadIdx.x], s_cc[threadIdx.x], p.h, s_bh[threadIdx.x], s_bl[threadIdx.x]);
    __syncthreads();
    for (int qi = threadIdx.x; qi < tile.z; qi += blockDim.x) {
      const int q = a.sorted_w[tile.y + qi];
      T x[3] = {(T)0, (T)0, (T)0};
      for (int j = 0; j < dim; ++j) {
        if constexpr (sizeof(T) == 4) x[j] = local32(xq[(int64_t)q * dim + j], s_bh[j], s_bl[j]);
        else x[j] = __dsub_rn(xq[(int64_t)q * dim + j], cell_base(p.o[j], s_cc[j], p.h));
      }
      T* out = var_grad + (int64_t)q * dim;
      T r2min = (T)INFINITY;
      for (int i = 0; i < n; ++i) {
        const R v = sx[i];
        const T rx = x[0] - (T)v.x, ry = x[1] - (T)v.y, rz = x[2] - (T)v.z;
        r2min = fmin(r2min, rx * rx + ry * ry + rz * rz);
      }
      if (!(r2min > (T)0)) {
        for (int j = 0; j < dim; ++j) out[j] = (T)INFINITY;
        continue;
      }
      const T zmin = sqrt(r2min);
      T W = 0, HY = 0, SV[3] = {0, 0, 0}, SYV[3] = {0, 0, 0};
      for (int i = 0; i < n; ++i) {
        const R v = sx[i];
        const T r[3] = {x[0] - (T)v.x, x[1] - (T)v.y, x[2] - (T)v.z};
        const T r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const T z = sqrt(r2);
        const T y = z - zmin > (T)0 ? z - zmin : (T)0;
        const T e = vg_exp<T>(-al * y);
        const T ez = e / z;
        W += e;
        HY += e * y;
        for (int k = 0; k < 3; ++k) {
          SV[k] += ez * r[k];
          SYV[k] += ez * y * r[k];
        }
      }
      const T B = al * HY / W + (T)1;
      T Vs[3], gg[3];
      for (int k = 0; k < 3; ++k) {
        Vs[k] = SV[k] / W;
        gg[k] = (B * SV[k] - al * SYV[k]) / W;
      }
      T acc[3] = {0, 0, 0};
      for (int i = 0; i < n; ++i) {
        const R v = sx[i];
        const T r[3] = {x[0] - (T)v.x, x[1] - (T)v.y, x[2] - (T)v.z};
        const T r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const T z = sqrt(r2);
        const T y = z - zmin > (T)0 ? z - zmin : (T)0;
        const T si = vg_exp<T>(-al * y) / W;
        const T li = si * (B - al * y);
        const T ci = li / z;
        const T s2 = (T)v.w;
        for (int k = 0; k < dim; ++k) {
          const T vk = r[k] / z;
          const T wk = li * (vk - Vs[k]) + si * (vk - gg[k]);
          acc[k] += s2 * (al * al * wk * wk + ci * ci * ((r2 - r[k] * r[k]) / r2));
        }
      }
      for (int k = 0; k < dim; ++k) out[k] = acc[k];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// host orchestration

static CandCtx cand_ctx(ksdf_ctx* c) {
  CandCtx cc;
  Model& m = c->m;
  cc.hk = ptr<uint64_t>(m.hkeys);
  cc.hv = ptr<int32_t>(m.hvals);
  cc.hcap = m.hcap;
  cc.status = ptr<int32_t>(m.status);
  cc.cell_key = ptr<uint64_t>(m.key);
  cc.G = m.G;
  for (int j = 0; j < 3; ++j) {
    cc.bb_lo[j] = c->bb[j];
    cc.bb_hi[j] = c->bb[3 + j];
    cc.bk_lo[j] = m.bk_lo[j];
    cc.bk_n[j] = m.bk_n[j];
  }
  cc.bk_off = ptr<int64_t>(m.bk_off);
  cc.bk_cells = ptr<int32_t>(m.bk_cells);
  cc.nbricks = m.nbricks;
  cc.K = c->p.K;
  cc.dim = c->p.dim;
  return cc;
}

// ---- autotuning of the query tile shapes ----
namespace {
constexpr int kTuneChunks[3] = {64, 128, 256};
constexpr int kTuneTcSmall[3] = {64, 96, 128};
}  // namespace

int query_tune_count() { return 9; }

// Times every (phase A budget, phase B class split) pair on the caller's query batch -- each a full query of all
// outputs run twice, the second timed with CUDA events on the context stream -- and keeps the fastest.
ksdf_status autotune_query(ksdf_ctx* c, const float* xq, int64_t Q, const int8_t* sign, int* choice, double* ms) {
  const int dim = c->p.dim;
  KSDF_CUDA(c, ensure(c->ws[WS_A], sizeof(float) * (size_t)Q * (4 + dim) + sizeof(int32_t) * 2 * (size_t)Q + 64));
  float* o = ptr<float>(c->ws[WS_A]);
  float *sdf = o, *grad = o + Q, *vs = grad + (size_t)Q * dim, *vf = vs + Q;
  int32_t* win = reinterpret_cast<int32_t*>(vf + Q);
  uint32_t* fl = reinterpret_cast<uint32_t*>(win + Q);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KSDF_CUDA(c, cudaEventCreate(&e0));
  KSDF_CUDA(c, cudaEventCreate(&e1));
  const bool prof = c->prof;
  c->prof = false;
  int best = -1;
  double best_ms = 0.0;
  ksdf_status s = KSDF_OK;
  for (int t = 0; t < query_tune_count() && s == KSDF_OK; ++t) {
    c->qt_chunks = kTuneChunks[t / 3];
    c->qt_tc_small = kTuneTcSmall[t % 3];
    float tms = 0.f;
    for (int rep = 0; rep < 2 && s == KSDF_OK; ++rep) {
      if (rep == 1) cudaEventRecord(e0, c->stream);
      s = run_query(c, xq, false, Q, sign, KSDF_OUT_ALL, sdf, grad, vs, vf, nullptr, win, fl);
      if (rep == 1) cudaEventRecord(e1, c->stream);
    }
    if (s != KSDF_OK) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&tms, e0, e1);
    if (e != cudaSuccess) {
      s = cuda_err(c, e, "autotune_query timing");
      break;
    }
    if (ms) ms[t] = tms;
    if (best < 0 || tms < best_ms) {
      best = t;
      best_ms = tms;
    }
  }
  c->prof = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) best = 4;  // the defaults
  c->qt_chunks = kTuneChunks[best / 3];
  c->qt_tc_small = kTuneTcSmall[best % 3];
  if (choice) *choice = best;
  return s;
}

ksdf_status wait_diagnostic(ksdf_ctx* c, uint32_t spins) {
  launch(k_wait_diag, 1, 64, 0, c->stream, spins, ptr<uint32_t>(c->status_word));
  KSDF_CUDA(c, cudaGetLastError());
  return KSDF_OK;
}

ksdf_status candidates_for_keys(ksdf_ctx* c, const uint64_t* keys, int64_t n, int32_t* cand, int32_t* count) {
  if (n <= 0) return KSDF_OK;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, kCandWarps), 8LL * c->num_sms);
  launch(k_candidates, grid, 32 * kCandWarps, 0, c->stream, keys, nullptr, n, cand_ctx(c), cand, count);
  KSDF_CUDA(c, cudaGetLastError());
  return KSDF_OK;
}

static uint64_t bin_capacity(int64_t Q) {
  uint64_t bcap = 1024;
  while (bcap < 2 * (uint64_t)Q && bcap < (1ull << 25)) bcap <<= 1;
  return bcap;
}

ksdf_status query_reserve(ksdf_ctx* c, int64_t Q, int64_t G) {
  const uint64_t bcap = bin_capacity(Q);
  const int K = c->p.K;
  KSDF_CUDA(c, ensure(c->ws[WS_QKEY], sizeof(uint64_t) * Q));
  KSDF_CUDA(c, ensure(c->ws[WS_QBIN], sizeof(int32_t) * Q));
  KSDF_CUDA(c, ensure(c->ws[WS_QRANK], sizeof(int32_t) * Q));
  KSDF_CUDA(c, ensure(c->ws[WS_QSORT], sizeof(int32_t) * Q));
  KSDF_CUDA(c, ensure(c->ws[WS_QWIN], sizeof(int32_t) * Q));
  KSDF_CUDA(c, ensure(c->ws[WS_QU], sizeof(double) * Q));
  KSDF_CUDA(c, ensure(c->ws[WS_QFLAG], sizeof(uint32_t) * Q));
  KSDF_CUDA(c, ensure(c->ws[WS_QWSORT], sizeof(int32_t) * Q));
  KSDF_CUDA(c, ensure(c->ws[WS_BHKEY], sizeof(uint64_t) * bcap));
  // per-slot / per-bin arrays: slot ids, bin keys, counts, offsets, tile counts, tile offsets (+ totals)
  KSDF_CUDA(c, ensure(c->ws[WS_BHVAL], sizeof(int64_t) * (bcap + 1)));
  KSDF_CUDA(c, ensure(c->ws[WS_BIN], sizeof(int64_t) * (5 * bcap + 10)));
  KSDF_CUDA(c, ensure(c->ws[WS_CAND], sizeof(int32_t) * (bcap * (K + 1))));
  const int64_t max_tiles_a = Q / kTA + bcap + 1;
  const int64_t max_tiles_b = Q / kTB64 + G + 1;  // also covers the mixed path's three tile lists (+ 2 G + 2)
  KSDF_CUDA(c, ensure(c->ws[WS_TILE], sizeof(int4) * (max_tiles_a + max_tiles_b + 2 * G + 2)));
  KSDF_CUDA(c, ensure(c->ws[WS_CELLQ], sizeof(int64_t) * (8 * G + 8)));
  // coarse order of the bins: three int32 arrays over at most min(bcap, Q) bins, then the bucket counts
  const int64_t nb_max = std::min<int64_t>((int64_t)bcap, Q);
  KSDF_CUDA(c, ensure(c->ws[WS_BORD], sizeof(int32_t) * (3 * nb_max + 2) + sizeof(int64_t) * kCoarseBuckets));
  const int64_t nsc = std::max<int64_t>((int64_t)bcap, kCoarseBuckets) / 2048 + 2;
  KSDF_CUDA(c, ensure(c->ws[WS_SCAN], sizeof(int64_t) * nsc));
  return KSDF_OK;
}

ksdf_status run_query(ksdf_ctx* c, const void* xq, bool f64, int64_t Q, const int8_t* sign, uint32_t mask, void* sdf,
                      void* grad, void* var_sdf, void* var_f, void* var_grad, int32_t* winner, uint32_t* flags) {
  cudaStream_t st = c->stream;
  const Params& p = c->p;
  Model& m = c->m;
  uint32_t* stw = ptr<uint32_t>(c->status_word);
  const uint64_t bcap = bin_capacity(Q);
  const int64_t G = m.G;
  {
    ksdf_status rs = query_reserve(c, Q, G);
    if (rs) return rs;
  }
  const int64_t max_tiles_a = Q / kTA + bcap + 1;
  const int TBq = f64 ? kTB64 : kBItem;
  const int tc_small = c->qt_tc_small;
  uint64_t* qkey = ptr<uint64_t>(c->ws[WS_QKEY]);
  int32_t* qbin = ptr<int32_t>(c->ws[WS_QBIN]);
  int32_t* qrank = ptr<int32_t>(c->ws[WS_QRANK]);
  int32_t* qsort = ptr<int32_t>(c->ws[WS_QSORT]);
  int32_t* qwin = ptr<int32_t>(c->ws[WS_QWIN]);
  float* qu = ptr<float>(c->ws[WS_QU]);
  double* qu64 = ptr<double>(c->ws[WS_QU]);
  uint32_t* qflag = ptr<uint32_t>(c->ws[WS_QFLAG]);
  int32_t* qwsort = ptr<int32_t>(c->ws[WS_QWSORT]);
  uint64_t* bhk = ptr<uint64_t>(c->ws[WS_BHKEY]);
  int64_t* slot_id = ptr<int64_t>(c->ws[WS_BHVAL]);
  int64_t* binbuf = ptr<int64_t>(c->ws[WS_BIN]);
  uint64_t* bin_key = reinterpret_cast<uint64_t*>(binbuf);
  int64_t* bin_cnt = binbuf + bcap;
  int64_t* bin_off = binbuf + 2 * bcap;
  int64_t* bin_nt = binbuf + 3 * bcap;
  int64_t* bin_toff = binbuf + 4 * bcap;
  int64_t* totals = binbuf + 5 * bcap;  // [0] n_bins, [1] n_queries grouped, [2] tiles A, [3] tiles B, [4..5] ctr
  int32_t* cand = ptr<int32_t>(c->ws[WS_CAND]);
  int32_t* ncand = cand + bcap * p.K;
  int4* tiles_a = ptr<int4>(c->ws[WS_TILE]);
  int4* tiles_b = tiles_a + max_tiles_a;
  int64_t* cbuf = ptr<int64_t>(c->ws[WS_CELLQ]);
  int64_t* wcnt = cbuf;
  int64_t* woff = cbuf + G;
  int64_t* wnt = cbuf + 2 * G;
  int64_t* wtoff = cbuf + 3 * G;
  int* counters = reinterpret_cast<int*>(totals + 6);

  cudaEvent_t e_q = prof_begin(c), e0 = prof_begin(c);
  // Q1 (kEmptyKey is all ones)
  KSDF_CUDA(c, cudaMemsetAsync(bhk, 0xFF, sizeof(uint64_t) * bcap, st));
  KSDF_CUDA(c, cudaMemsetAsync(totals, 0, sizeof(int64_t) * 10, st));
  KSDF_CUDA(c, cudaMemsetAsync(wcnt, 0, sizeof(int64_t) * G, st));
  if (f64)
    launch(k_q_bin<double>, ceil_div(Q, 256), 256, 0, st, static_cast<const double*>(xq), Q, p, qkey, bhk, bcap, stw);
  else
    launch(k_q_bin<float>, ceil_div(Q, 256), 256, 0, st, static_cast<const float*>(xq), Q, p, qkey, bhk, bcap, stw);
  // Q2
  launch(k_slot_flags, ceil_div(bcap, 256), 256, 0, st, bhk, bcap, slot_id);
  KSDF_CUDA(c, scan_i64(slot_id, slot_id, bcap, &totals[0], c->ws[WS_SCAN], st));
  launch(k_bin_table, ceil_div(bcap, 256), 256, 0, st, bhk, bcap, slot_id, bin_key, bin_cnt);
  launch(k_q_rank, ceil_div(Q, 256), 256, 0, st, qkey, Q, bhk, slot_id, bcap, qbin, qrank, bin_cnt);
  // the per-bin passes cover the occupied bins only (their count is on the device, totals[0])
  const int64_t* nbins = &totals[0];
  KSDF_CUDA(c, scan_i64(bin_cnt, bin_off, bcap, &totals[1], c->ws[WS_SCAN], st, nbins));
  launch(k_ntiles, ceil_div(bcap, 256), 256, 0, st, bin_cnt, bcap, kTA, bin_nt, nbins);
  launch(k_scatter_grouped, ceil_div(Q, 256), 256, 0, st, qbin, qrank, Q, bin_off, qsort);
  // phase A's tiles in the bins' coarse spatial order (bin_toff holds the tile counts in that order, then their
  // offsets)
  {
    const int64_t nb_max = std::min<int64_t>((int64_t)bcap, Q);
    int32_t* coarse = ptr<int32_t>(c->ws[WS_BORD]);
    int32_t* brank = coarse + nb_max;
    int32_t* border = brank + nb_max;
    // the bucket counts after the three int32 arrays, at an int32 offset rounded up to even (8-byte aligned)
    int64_t* hist = reinterpret_cast<int64_t*>(coarse + ((3 * nb_max + 1) & ~(int64_t)1));
    const unsigned gb = ceil_div(nb_max, 256);
    KSDF_CUDA(c, cudaMemsetAsync(hist, 0, sizeof(int64_t) * kCoarseBuckets, st));
    launch(k_bin_coarse, gb, 256, 0, st, bin_key, nbins, coarse, brank, hist);
    KSDF_CUDA(c, scan_i64(hist, hist, kCoarseBuckets, nullptr, c->ws[WS_SCAN], st));
    launch(k_bin_order, gb, 256, 0, st, coarse, brank, hist, nbins, bin_nt, border, bin_toff);
    KSDF_CUDA(c, scan_i64(bin_toff, bin_toff, nb_max, &totals[2], c->ws[WS_SCAN], st, nbins));
    launch(k_make_tiles_ordered, gb, 256, 0, st, border, bin_cnt, bin_off, bin_toff, nbins, kTA, tiles_a);
  }
  prof_end(c, e0, "query.group");
  e0 = prof_begin(c);
  // Q3
  {
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(bcap, kCandWarps), 8LL * c->num_sms);
    launch(k_candidates, grid, 32 * kCandWarps, 0, st, bin_key, &totals[0], 0, cand_ctx(c), cand, ncand);
    launch(k_count_requests, ceil_div(bcap, 256), 256, 0, st, bin_cnt, cand, ncand, &totals[0], p.K,
           ptr<int32_t>(m.qc0));
  }
  prof_end(c, e0, "query.candidates");
  e0 = prof_begin(c);
  // Q4
  PhaseAArgs pa;
  pa.tiles = tiles_a;
  pa.n_tiles = &totals[2];
  pa.counter = &counters[0];
  pa.sorted_q = qsort;
  pa.bin_key = bin_key;
  pa.cand = cand;
  pa.ncand = ncand;
  pa.ts_off = ptr<int64_t>(m.ts_off);
  pa.cell_n = ptr<int32_t>(m.n);
  pa.cell_key = ptr<uint64_t>(m.key);
  pa.mf4 = ptr<float4>(m.mf4);
  pa.md4 = ptr<D4>(m.md4);
  pa.qwin = qwin;
  pa.qu = qu;
  pa.qu64 = qu64;
  pa.qflag = qflag;
  pa.st = stw;
  const int maxn = std::max(m.max_n, 1);
  if (f64) {
    const size_t smem = sizeof(D4) * (size_t)p.K * maxn;
    auto kern = p.kernel == KSDF_KERNEL_MATERN32 ? k_phaseA64<true> : k_phaseA64<false>;
    KSDF_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    KSDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTA, smem));
    launch(kern, std::max(1, occ) * c->num_sms, kTA, smem, st, pa, static_cast<const double*>(xq), p);
  } else {
    pa.chunks = phase_a_chunks(c->qt_chunks, p.n_max);
    const size_t smem = phase_a_smem(p.K, pa.chunks);
    auto kern = p.kernel == KSDF_KERNEL_MATERN32 ? k_phaseA<true> : k_phaseA<false>;
    KSDF_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    KSDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTA, smem));
    launch(kern, std::max(1, occ) * c->num_sms, kTA, smem, st, pa, static_cast<const float*>(xq), p);
  }
  KSDF_CUDA(c, cudaGetLastError());
  prof_end(c, e0, f64 ? "query64.phaseA" : "query.phaseA");
  e0 = prof_begin(c);
  // Q5
  int32_t* wrank = qrank;  // qrank no longer needed
  if (f64)
    launch(k_w_rank<double>, ceil_div(Q, 256), 256, 0, st, qwin, qflag, qbin, Q, wrank, wcnt, mask, p.dim,
                                                        static_cast<double*>(sdf), static_cast<double*>(grad),
                                                        static_cast<double*>(var_sdf), static_cast<double*>(var_f),
                                                        static_cast<double*>(var_grad), winner, flags);
  else
    launch(k_w_rank<float>, ceil_div(Q, 256), 256, 0, st, qwin, qflag, qbin, Q, wrank, wcnt, mask, p.dim,
                                                       static_cast<float*>(sdf), static_cast<float*>(grad),
                                                       static_cast<float*>(var_sdf), static_cast<float*>(var_f),
                                                       static_cast<float*>(var_grad), winner, flags);
  KSDF_CUDA(c, scan_i64(wcnt, woff, G, nullptr, c->ws[WS_SCAN], st));
  // mixed path: three tile lists by winner-cell size -- tensor-core tiles of kTcM queries for cells of at most
  // tc_small and kTcMaxN samples, SIMT tiles of kBItem for larger cells
  const int64_t tcap = Q / kTcM + G + 1;
  int4* tiles_b1 = tiles_b + tcap;
  int4* tiles_b2 = tiles_b1 + tcap;
  int64_t *nt1 = cbuf + 4 * G, *nt2 = cbuf + 5 * G, *toff1 = cbuf + 6 * G, *toff2 = cbuf + 7 * G;
  if (f64) {
    launch(k_ntiles, ceil_div(G, 256), 256, 0, st, wcnt, G, TBq, wnt, (const int64_t*)nullptr);
    KSDF_CUDA(c, scan_i64(wnt, wtoff, G, &totals[3], c->ws[WS_SCAN], st));
  } else {
    launch(k_ntiles3, ceil_div(G, 256), 256, 0, st, wcnt, ptr<int32_t>(m.n), G, tc_small, kTcMaxN, kTcM, kBItem, wnt,
           nt1, nt2);
    KSDF_CUDA(c, scan_i64(wnt, wtoff, G, &totals[3], c->ws[WS_SCAN], st));
    KSDF_CUDA(c, scan_i64(nt1, toff1, G, &totals[4], c->ws[WS_SCAN], st));
    KSDF_CUDA(c, scan_i64(nt2, toff2, G, &totals[5], c->ws[WS_SCAN], st));
  }
  launch(k_w_scatter, ceil_div(Q, 256), 256, 0, st, qwin, qbin, wrank, Q, woff, qwsort);
  if (f64)
    launch(k_make_tiles, ceil_div(G, 256), 256, 0, st, wcnt, woff, wtoff, G, TBq, tiles_b, (const int64_t*)nullptr);
  else
    launch(k_make_tiles3, ceil_div(G, 256), 256, 0, st, wcnt, woff, wtoff, toff1, toff2, ptr<int32_t>(m.n), tc_small,
           kTcMaxN, G, kTcM, kBItem, tiles_b, tiles_b1, tiles_b2);
  prof_end(c, e0, "query.regroup");
  e0 = prof_begin(c);
  // Q6
  PhaseBArgs pb;
  pb.tiles = tiles_b;
  pb.n_tiles = &totals[3];
  pb.counter = &counters[1];
  pb.sorted_w = qwsort;
  pb.ts_off = ptr<int64_t>(m.ts_off);
  pb.cell_n = ptr<int32_t>(m.n);
  pb.cell_key = ptr<uint64_t>(m.key);
  pb.linv_off = ptr<int64_t>(m.linv_off);
  pb.chol_off = ptr<int64_t>(m.chol_off);
  pb.mf4 = ptr<float4>(m.mf4);
  pb.md4 = ptr<D4>(m.md4);
  pb.mvar = ptr<float>(m.mvar);
  pb.mnrm = m.has_normals ? ptr<float4>(m.mnrm) : nullptr;
  pb.linv32 = ptr<float>(m.linv32);
  pb.chol64 = ptr<double>(m.chol64);
  pb.qu = qu;
  pb.qu64 = qu64;
  pb.qflag = qflag;
  pb.sign = sign;
  pb.has_normals = m.has_normals ? 1 : 0;
  pb.mask = mask;
  pb.st = stw;
  if (f64) {
    const size_t smem = sizeof(D4) * p.n_max + sizeof(double) * p.n_max * (1 + kTB64);
    auto kern = p.kernel == KSDF_KERNEL_MATERN32 ? k_phaseB64<true> : k_phaseB64<false>;
    KSDF_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    KSDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTB64, smem));
    launch(kern, std::max(1, occ) * c->num_sms, kTB64, smem, st, 
        pb, static_cast<const double*>(xq), p, static_cast<double*>(sdf), static_cast<double*>(grad),
        static_cast<double*>(var_sdf), static_cast<double*>(var_f), winner, flags);
  } else {
    // tensor-core tiles: cells of at most tc_small samples, then of at most kTcMaxN (one after the other, each
    // with the whole GPU: the TMEM of an SM is 512 columns); cells beyond kTcMaxN on the SIMT kernel meanwhile
    const int maxn = std::max(m.max_n, 1);
    if (maxn > kTcMaxN) {
      KSDF_CUDA(c, fork_streams(c));
      const int smax = maxn;
      const size_t smem = sizeof(float4) * smax + sizeof(float) * (linv_blocked_size(kLinvStageN) + (size_t)smax * (1 + kBQ));
      auto kb = p.kernel == KSDF_KERNEL_MATERN32 ? k_phaseB<true> : k_phaseB<false>;
      KSDF_CUDA(c, cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int occ = 0;
      KSDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb, kBQ * kBW, smem));
      PhaseBArgs p2 = pb;
      p2.tiles = tiles_b2;
      p2.n_tiles = &totals[5];
      p2.counter = &counters[3];
      launch(kb, std::max(1, occ) * c->num_sms, kBQ * kBW, smem, c->aux[0], p2, static_cast<const float*>(xq), p,
             static_cast<float*>(sdf), static_cast<float*>(grad), static_cast<float*>(var_sdf),
             static_cast<float*>(var_f), winner, flags, smax);
    }
    for (int part = 0; part < 2; ++part) {
      if (part == 1 && maxn <= tc_small) break;
      // whole steps of 8 samples are staged (padding samples up to Kp)
      const int kcap = tc_kp(std::min(part == 0 ? tc_small : kTcMaxN, maxn));
      uint32_t ncols = 32;
      while ((int)ncols < tc_np(kcap)) ncols <<= 1;
      const size_t smem = tc_smem_bytes(kcap);
      auto ktc = p.kernel == KSDF_KERNEL_MATERN32 ? k_phaseB_tc<true> : k_phaseB_tc<false>;
      KSDF_CUDA(c, cudaFuncSetAttribute(ktc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      KSDF_CUDA(c, cudaFuncSetAttribute(ktc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
      // CTAs per SM: bounded by the TMEM columns (512 per SM) and the shared memory (227 KB per SM usable,
      // plus the static part and the 1 KB the driver reserves per CTA)
      const int by_smem = (int)((size_t)(227 * 1024) / (smem + 2048));
      const int occ = std::max(1, std::min(by_smem, (int)(512 / ncols)));
      TcArgs ta;
      ta.tiles = part == 0 ? tiles_b : tiles_b1;
      ta.n_tiles = &totals[3 + part];
      ta.counter = &counters[1 + part];
      ta.ltc_off = ptr<int64_t>(m.ltc_off);
      ta.ltc = ptr<float>(m.ltc);
      launch(ktc, occ * c->num_sms, kTcThreads, smem, st, pb, ta, static_cast<const float*>(xq), p,
             static_cast<float*>(sdf), static_cast<float*>(grad), static_cast<float*>(var_sdf),
             static_cast<float*>(var_f), winner, flags, kcap, ncols);
    }
    if (maxn > kTcMaxN) KSDF_CUDA(c, join_streams(c));
  }
  KSDF_CUDA(c, cudaGetLastError());
  prof_end(c, e0, f64 ? "query64.phaseB" : "query.phaseB");
  if (mask & KSDF_OUT_VAR_GRAD) {
    e0 = prof_begin(c);
    VarGradArgs va;
    va.sorted_w = qwsort;
    va.ts_off = ptr<int64_t>(m.ts_off);
    va.cell_n = ptr<int32_t>(m.n);
    va.cell_key = ptr<uint64_t>(m.key);
    va.mf4 = ptr<float4>(m.mf4);
    va.md4 = ptr<D4>(m.md4);
    va.mvar = ptr<float>(m.mvar);
    const int nmax = std::max(m.max_n, 1);
    // the winner tiles of phase B: one list on the plain path, three on the mixed path (by cell size)
    const int nlists = f64 ? 1 : 3;
    const int4* lists[3] = {tiles_b, tiles_b1, tiles_b2};
    for (int l = 0; l < nlists; ++l) {
      VarGradArgs v = va;
      v.tiles = lists[l];
      v.n_tiles = &totals[3 + l];
      v.counter = &counters[4 + l];
      if (f64) {
        const size_t sm = sizeof(D4) * (size_t)nmax;
        KSDF_CUDA(c, cudaFuncSetAttribute(k_var_grad<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int occ = 0;
        KSDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_var_grad<double>, kVG, sm));
        launch(k_var_grad<double>, std::max(1, occ) * c->num_sms, kVG, sm, st, v, static_cast<const double*>(xq), p,
               static_cast<double*>(var_grad));
      } else {
        const size_t sm = sizeof(float4) * (size_t)nmax;
        KSDF_CUDA(c, cudaFuncSetAttribute(k_var_grad<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int occ = 0;
        KSDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_var_grad<float>, kVG, sm));
        launch(k_var_grad<float>, std::max(1, occ) * c->num_sms, kVG, sm, st, v, static_cast<const float*>(xq), p,
               static_cast<float*>(var_grad));
      }
    }
    KSDF_CUDA(c, cudaGetLastError());
    prof_end(c, e0, f64 ? "query64.var_grad" : "query.var_grad");
  }
  prof_end(c, e_q, f64 ? "query64" : "query");
  return KSDF_OK;
}

}  // namespace ksdf
