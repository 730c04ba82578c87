// ksdf_internal.cuh -- shared definitions of the libksdf.so translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ksdf.h"

namespace ksdf {

constexpr int64_t kBias = 1LL << 20;    // cell coordinates live in [-2^20, 2^20)
constexpr int kMaxPre = 8192;           // collection-box members before the cap, per cell
constexpr int kMaxK = 32;               // candidate list length limit
constexpr int kMaxNmax = 512;           // training-set cap limit
constexpr uint64_t kEmptyKey = ~0ull;   // empty hash slot
constexpr int kBrickShift = 3;          // bricks of 8 cells per axis
constexpr unsigned kWaitLimit = 1u << 26;  // bounded spin on an mbarrier (~seconds)

// device status word bits (ksdf_sync_status)
enum : uint32_t { ST_NONFINITE = 1u, ST_CAPACITY = 2u, ST_TIMEOUT = 4u, ST_NOT_PD = 8u };

// ------------------------------------------------------------------------------------------------
// cell keys: three biased 21-bit fields, z most significant, so ascending key = (cz, cy, cx) order

__host__ __device__ inline uint64_t pack_key(int64_t cx, int64_t cy, int64_t cz) {
  return ((uint64_t)(cz + kBias) << 42) | ((uint64_t)(cy + kBias) << 21) | (uint64_t)(cx + kBias);
}
__host__ __device__ inline void unpack_key(uint64_t k, int& cx, int& cy, int& cz) {
  cx = (int)((int64_t)(k & 0x1FFFFF) - kBias);
  cy = (int)((int64_t)((k >> 21) & 0x1FFFFF) - kBias);
  cz = (int)((int64_t)((k >> 42) & 0x1FFFFF) - kBias);
}

// bin of one coordinate: floor((x - o) / h) in IEEE binary64 with no contraction; false if out of range.
// rh = 1/h when h is a power of two, else 0: then (x - o) / h and (x - o) * rh are the same real number, so
// their correctly rounded results agree bit for bit and the multiplication stands in for the division.
__device__ inline bool bin_coord(double x, double o, double h, double rh, int& c) {
  const double d = __dsub_rn(x, o);
  double t = rh != 0.0 ? __dmul_rn(d, rh) : __ddiv_rn(d, h);
  double f = floor(t);
  if (!(f >= -(double)kBias && f < (double)kBias)) return false;
  c = (int)f;
  return true;
}

// lower corner o + c h of a cell along one axis, IEEE binary64, no contraction
__device__ inline double cell_base(double o, int c, double h) { return __dadd_rn(o, __dmul_rn((double)c, h)); }

// the cell base o + c h as an FP32 head + tail (computed once per tile in binary64), and a point's
// cell-local coordinate (x - head) - tail in FP32: within one FP32 rounding of fl32(x - (o + c h)),
// without per-point FP64 work (the FP64 pipe is 1/64 of the FP32 rate on this part)
__device__ inline void base_split(double o, int c, double h, float& hi, float& lo) {
  const double b = cell_base(o, c, h);
  hi = (float)b;
  lo = (float)(b - (double)hi);
}
__device__ __forceinline__ float local32(float x, float hi, float lo) { return __fsub_rn(__fsub_rn(x, hi), lo); }

// packed FP32x2 arithmetic (two lanes of one thread per instruction): a u64 holds (lo, hi) floats
__device__ __forceinline__ unsigned long long f2pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 f2unpack(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// The kernel exponent of the scaled posterior mean, lambda (r_i^2 - d^2) with r_i = |q - x_i| and d = |q - x_n|
// for the GP's nearest sample x_n (App. D scaling), in FP32 cell-local coordinates.  Subtracting the two
// squares r_i^2 - d^2 (each about d^2) would leave an absolute error of a few 2^-24 d^2, which lambda turns
// into a relative error of every k'_i of order lambda d^2 2^-23.  The identity
//   r_i^2 - d^2 = (x_i - x_n) . ((x_i - x_n) - 2 (q - x_n))
// forms it from the sample-to-sample difference a = x_i - x_n (one rounding of a small number) and the
// query's offset from x_n, so the error scales with |a| d instead of d^2.  w = 2 (q - x_n) is computed once
// per query.
__device__ __forceinline__ float excess_sq(float vx, float vy, float vz, float nx, float ny, float nz, float wx,
                                           float wy, float wz) {
  const float ax = vx - nx, ay = vy - ny, az = vz - nz;
  return fmaf(ax, ax - wx, fmaf(ay, ay - wy, az * (az - wz)));
}

// hash of a packed key (splitmix64 finaliser)
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// lookup in an open-addressing (linear probing) table of capacity cap (power of 2); -1 if absent
__device__ inline int hash_find(const uint64_t* keys, const int32_t* vals, uint64_t cap, uint64_t k) {
  uint64_t s = mix64(k) & (cap - 1);
  for (uint64_t probe = 0; probe < cap; ++probe) {
    uint64_t kk = keys[s];
    if (kk == k) return vals[s];
    if (kk == kEmptyKey) return -1;
    s = (s + 1) & (cap - 1);
  }
  return -1;
}

// four doubles, 32-byte aligned (one TMA-friendly member record of the FP64 path)
struct __align__(32) D4 {
  double x, y, z, w;
};
__host__ __device__ inline D4 D4make(double x, double y, double z, double w) {
  D4 r;
  r.x = x;
  r.y = y;
  r.z = z;
  r.w = w;
  return r;
}

struct Params {
  int dim;
  double o[3];
  double h;
  double rh;  // 1 / h when h is a power of two (exact), else 0
  double mu;
  int n_max;
  int K;
  double lambda;
  double alpha_s;  // softmin temperature
  int sign_mode;
  int kernel;      // KSDF_KERNEL_RBF or KSDF_KERNEL_MATERN32
};

// ------------------------------------------------------------------------------------------------
// device memory helper: grow-only buffer

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Model {
  int64_t S = 0, G = 0, M = 0;    // samples, cells, training-set members
  int64_t chol_total = 0;         // sum N (N+1) / 2 (packed FP64 L)
  int64_t linv_total = 0;         // sum 32 nb (nb+1), nb = ceil(N/8) (FP32 L^-1, 8-row interleaved)
  int64_t ltc_total = 0;          // sum ltc_size(N) (FP32 L^-1 as the tensor-core B operand)
  int max_n = 0;                  // largest training set
  bool has_normals = false;
  int n_not_pd = 0;
  // per cell
  DevBuf key, status, n, ts_off, chol_off, linv_off;  // uint64, int32, int32, int64 (G+1) x 3
  DevBuf hkeys, hvals;                          // GP cell hash table
  uint64_t hcap = 0;
  DevBuf cell_order;                            // cells sorted by descending N (fit work order)
  // per member (CSR by ts_off)
  DevBuf mf4;      // float4 (x, y, z, alpha) cell-local, FP32
  DevBuf md4;      // D4 (x, y, z, alpha) cell-local, FP64
  DevBuf mvar;     // float sigma^2
  DevBuf mnrm;     // float4 normal
  DevBuf mgid;     // int32 global sample id
  DevBuf mpad;     // int32 padded ids (G x n_max), assembly scratch
  DevBuf chol64;   // double: Cholesky factor L, packed lower rows (row i at i (i+1) / 2)
  DevBuf linv32;   // float: L^-1 in 8-row blocks: block R (rows 8R..8R+7) holds, for each column
                   // j <= 8R+7, the 8 values L^-1[8R+r][j] (0 above the diagonal); block R starts at
                   // 32 R (R+1); size per cell 32 nb (nb+1), nb = ceil(N/8)
  DevBuf x;        // sample positions (S x dim double), kept for the backward's scatter
  DevBuf var_all;  // float: every sample's sigma^2 (S), kept for updates
  DevBuf nrm_all;  // float: every sample's normal (S x dim), when the model has normals
  DevBuf ltc_off;  // int64 (G+1): offsets into ltc
  DevBuf ltc;      // float: for cells with N <= kTcMaxN, L^-1 as the K-major B operand of the variance
                   // contraction, rows (N dim) padded to Np = 16 ceil(N/16), columns (K dim) to Kp = 8 ceil(N/8),
                   // in K-quads: element (j, i) at (i / 4) Np 4 + j 4 + i % 4 (zero outside the lower triangle),
                   // FP32 (split into TF32 hi and lo parts in shared memory by the query)
  // bricks of 2^kBrickShift cells per axis over the cell bounding box, each listing its OK cells (the
  // coarse level of the candidate search for query bins far from the nearest cells); nbricks = 0 when the
  // box is too sparse for a dense brick grid
  DevBuf bk_off;    // int64 (nbricks + 1), brick index (bz nby + by) nbx + bx
  DevBuf bk_cells;  // int32 cell ids grouped by brick
  int bk_lo[3] = {0, 0, 0}, bk_n[3] = {0, 0, 0};
  int64_t nbricks = 0;
  // refit scheduling (Sec. IV-C, App. G), per cell (int32): the query counter c0 (requests as a fused candidate,
  // capped, halved when the cell is fitted), the training marks c2 (updates that changed the cell's training set
  // since its last fit), and whether the last fit or update fitted the cell
  DevBuf qc0, qc2, refit;
};

}  // namespace ksdf

namespace ksdf {
// one size class of the batched fit: cells of N up to np are factored by teams of `team` threads; the
// largest class keeps its matrices in a per-CTA global slot (gmat)
struct FitClassCfg {
  int np, team;
  bool gmat;
};
}  // namespace ksdf

struct ksdf_ctx {
  ksdf::Params p;
  ksdf_params abi;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string err;
  bool fitted = false;
  ksdf::Model m;
  ksdf::Model m_prev;  // the previous model during an update (its buffers are reused by the next one)
  std::vector<ksdf::FitClassCfg> fit_cls;  // the fit's size classes (empty: the default table); ksdf_autotune
  // workspaces
  ksdf::DevBuf status_word;       // uint32 device status
  ksdf::DevBuf ws[32];            // general workspaces (grow only), indexed by role
  int qt_chunks = 128;            // query tile shapes (ksdf_autotune_query): phase A's shared-memory budget in
  int qt_tc_small = 96;           // chunks of 8 samples, and the largest cell of phase B's 128-column TMEM class
  int64_t sched_max = 0;          // refit budget of ksdf_update (cells per update; 0 = every changed cell)
  float sched_eta = 1e-3f;        // weight of the query counter in the training priority
  ksdf::DevBuf stage[12];         // staging of host arrays
  int64_t reserved_q = 0, reserved_s = 0;
  int bb[6] = {0, 0, 0, 0, 0, 0};  // bounding box of the cells: min xyz, max xyz
  // stage profiling (ksdf_profile): event pairs recorded on the stream, folded into totals when read
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Pending {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<std::string> stage_names;
  std::vector<double> stage_ms;
  std::vector<long long> stage_calls;
  // auxiliary streams for concurrent launches inside one call (fork/join through events)
  static constexpr int kNumAux = 8;
  cudaStream_t aux[kNumAux] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kNumAux] = {}, ev_mid[kNumAux] = {};  // ev_mid: a stage boundary inside a fork
  // high-priority auxiliary streams: work queued there is dispatched ahead of the pending blocks of kernels on
  // the other streams as soon as SM resources free up
  cudaStream_t aux_hi[kNumAux] = {};
  cudaEvent_t ev_join_hi[kNumAux] = {};
};

namespace ksdf {

// error helpers (host)
ksdf_status set_err(ksdf_ctx* c, ksdf_status s, const char* fmt, ...);
ksdf_status cuda_err(ksdf_ctx* c, cudaError_t e, const char* what);
#define KSDF_CUDA(c, call)                                 \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return ksdf::cuda_err(c, e_, #call); \
  } while (0)

cudaError_t ensure(DevBuf& b, size_t bytes);
void release(DevBuf& b);
template <class T> inline T* ptr(DevBuf& b) { return static_cast<T*>(b.p); }

// ---- stage profiling (ksdf_abi.cu): no-ops unless enabled ----
cudaEvent_t prof_begin(ksdf_ctx* c);
void prof_end(ksdf_ctx* c, cudaEvent_t a, const char* name);

// ---- autotuning of the fit's size classes (ksdf_fit.cu) ----
int fit_table_count();
ksdf_status device_math(ksdf_ctx* c, int fn, const double* x, int64_t n, double* y);
const std::vector<FitClassCfg>& fit_table(int i);
ksdf_status autotune_fit(ksdf_ctx* c, int* chosen, double* ms);

// ---- fork/join of the context stream with the auxiliary streams (ksdf_abi.cu) ----
cudaError_t fork_streams(ksdf_ctx* c);
cudaError_t join_streams(ksdf_ctx* c);

// ---- sorting and scanning (ksdf_sort.cu) ----
// exclusive scan of n int64 values (in may equal out); total (optional) gets the sum on the device.  With
// n_dev (optional, a device count) only the first min(n, *n_dev) elements are scanned.
cudaError_t scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, DevBuf& tmp, cudaStream_t st,
                     const int64_t* n_dev = nullptr);
// stable LSD radix sort by the low `bits` bits of 64-bit keys, with 32-bit values.  Result in keys/vals.
cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int bits, DevBuf& tmp, cudaStream_t st);

// ---- fit (ksdf_fit.cu) ----
// the fit; with `prev` (the model being updated, whose samples are x[0 .. prev->S)), cells whose training set
// is unchanged copy prev's factors instead of being refitted, and *n_refit receives the number refitted
ksdf_status fit_model(ksdf_ctx* c, const double* x, const float* var, const float* nrm, int64_t S,
                      const Model* prev = nullptr, int64_t* n_refit = nullptr);
ksdf_status bin_points(ksdf_ctx* c, const double* x, int64_t n, uint64_t* keys);

// ---- query (ksdf_query.cu) ----
ksdf_status run_query(ksdf_ctx* c, const void* xq, bool f64, int64_t Q, const int8_t* sign, uint32_t mask, void* sdf,
                      void* grad, void* var_sdf, void* var_f, void* var_grad, int32_t* winner, uint32_t* flags);
ksdf_status candidates_for_keys(ksdf_ctx* c, const uint64_t* keys, int64_t n, int32_t* cand, int32_t* count);
ksdf_status query_reserve(ksdf_ctx* c, int64_t Q, int64_t G);
ksdf_status wait_diagnostic(ksdf_ctx* c, uint32_t spins);
int query_tune_count();
ksdf_status autotune_query(ksdf_ctx* c, const float* xq, int64_t Q, const int8_t* sign, int* choice, double* ms);

// ---- backward (ksdf_backward.cu) ----
ksdf_status run_backward(ksdf_ctx* c, const float* xq, int64_t Q, const int8_t* sign, const int32_t* winner,
                         const float* d_sdf, const float* d_grad, float* d_xq, float* d_x);

// workspace roles (indices into ksdf_ctx::ws)
enum WsRole {
  WS_SORT = 0,   // radix sort / scan temporaries
  WS_SCAN = 1,
  WS_A = 2,      // generic
  WS_B = 3,
  WS_C = 4,
  WS_D = 5,
  WS_E = 6,
  WS_F = 7,
  WS_QKEY = 8,   // per query
  WS_QBIN = 9,
  WS_QRANK = 10,
  WS_QSORT = 11,
  WS_QWIN = 12,
  WS_QU = 13,
  WS_QFLAG = 14,
  WS_QWSORT = 15,
  WS_BHKEY = 16,  // bin hash table
  WS_BHVAL = 17,
  WS_BIN = 18,    // per bin: keys, counts, offsets, candidates
  WS_TILE = 19,
  WS_CAND = 20,
  WS_CELLQ = 21,  // per cell query counts / offsets
  WS_FITSCR = 22, // FP64 fit scratch
  WS_BW = 23,     // backward accumulators
  WS_LINVSCR = 24, // FP32 L^-1 scratch of the largest cells
  WS_TOUCH = 25,  // update: per cell touched flag and previous id
  WS_UX = 26,     // update: the union of old and new samples (positions, variances, normals)
  WS_UV = 27,
  WS_UN = 28,
  WS_BRICK = 29,  // brick build: rank of each cell within its brick
  WS_SCHED = 30,  // refit scheduling: priority keys, cell ids, changed flags, previous ids
  WS_BORD = 31    // query bins in coarse spatial order: coarse keys, ranks, order; bucket counts
};
constexpr int kQueryCounterCap = 10000;  // cap of the per-cell query counter (App. G)

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

__host__ __device__ inline int64_t tri_sz(int64_t n) { return n * (n + 1) / 2; }

// cells up to this size run the variance contraction on the tensor cores (one MMA covers N <= 256)
constexpr int kTcMaxN = 256;
__host__ __device__ inline int tc_np(int n) { return (n + 15) & ~15; }
__host__ __device__ inline int tc_kp(int n) { return (n + 7) & ~7; }
__host__ __device__ inline int64_t ltc_size(int64_t n) {
  return (n > 0 && n <= kTcMaxN) ? (int64_t)tc_np((int)n) * tc_kp((int)n) : 0;
}
// size and block offset of the 8-row interleaved L^-1 layout
__host__ __device__ inline int64_t linv_blocked_size(int64_t n) {
  const int64_t nb = (n + 7) / 8;
  return 32 * nb * (nb + 1);
}
__host__ __device__ inline int64_t linv_block_off(int64_t R) { return 32 * R * (R + 1); }

// every kernel launch of the library goes through launch(): it counts launches (ksdf_profile_read)
extern std::atomic<long long> g_launches;
template <class... KArgs, class... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
}

}  // namespace ksdf
