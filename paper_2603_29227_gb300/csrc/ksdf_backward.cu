// ksdf_backward.cu -- adjoint of the Kernel-SDF query with respect to the query points and the sample
// positions (differentiation path; the paper states the SDF is differentiable, Sec. IV-B).
//
// With d held constant (u does not depend on the scaling of App. D), for a query q whose min-fusion
// winner is cell g with training set {x_i, alpha_i}:
//   u^2 = -log f'/lambda + d^2,  f' = sum_i alpha_i k'_i,  k'_i = exp(-lambda (|x - x_i|^2 - d^2))
//   dL/df'  = -s dsdf / (2 lambda u f')                                   (sdf = s u)
//   x_bar  += dL/df' grad_x f' = dL/df' (-2 lambda G),  G = sum_i alpha_i k'_i (x - x_i)
//   X_bar_i += dL/df' 2 lambda alpha_i k'_i (x - x_i),   alpha_bar_i += dL/df' k'_i
// For the gradient output s G/|G| with cotangent gb: v = s (I - g g^T) gb / |G|, and
//   x_bar += sum_i alpha_i k'_i (v - 2 lambda r_i (r_i . v)),  X_bar_i -= the i-th term,
//   alpha_bar_i += k'_i (r_i . v).
// Through alpha = A^{-1} 1 (A = K + Sigma = L L^T): b = A^{-1} alpha_bar (FP32 L^{-1} products with one
// FP64 refinement step against L), X_bar_i += sum_j 2 lambda K_ij (b_i alpha_j + b_j alpha_i)(x_i - x_j).
// Kernel 1 recomputes k' per (query, winner) tile and accumulates alpha_bar / X_bar per sample; kernel 2 runs
// once per touched cell.
#include "ksdf_internal.cuh"

#include <algorithm>

namespace ksdf {

namespace {

constexpr int kTW = 128;  // queries per backward tile
constexpr float kLog2e = 1.4426950408889634f;

__device__ inline float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void k_bw_count(const int32_t* winner, int64_t Q, int64_t G, int32_t* rank, int64_t* cnt, float* d_xq,
                           int dim, uint32_t* st) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  int w = winner[q];
  if (w >= G) {
    atomicOr(st, ST_CAPACITY);
    w = -1;
  }
  if (w < 0) {
    for (int j = 0; j < dim; ++j) d_xq[q * dim + j] = 0.f;
    rank[q] = -1;
    return;
  }
  rank[q] = (int32_t)atomicAdd((unsigned long long*)&cnt[w], 1ull);
}

__global__ void k_bw_scatter(const int32_t* winner, const int32_t* rank, int64_t Q, int64_t G, const int64_t* off,
                             int32_t* sorted) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  int w = winner[q];
  if (w >= 0 && w < G && rank[q] >= 0) sorted[off[w] + rank[q]] = (int32_t)q;
}

__global__ void k_bw_tiles(const int64_t* cnt, const int64_t* off, const int64_t* toff, int64_t G, int4* tiles) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  int64_t c = cnt[g];
  for (int64_t t = 0; t * kTW < c; ++t)
    tiles[toff[g] + t] = make_int4((int)g, (int)(off[g] + t * kTW), (int)(c - t * kTW < kTW ? c - t * kTW : kTW), 0);
}

__global__ void k_ntiles_w(const int64_t* cnt, int64_t n, int64_t* nt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) nt[i] = (cnt[i] + kTW - 1) / kTW;
}

struct BwArgs {
  const int4* tiles;
  const int64_t* n_tiles;
  int* counter;
  const int32_t* sorted;
  const int64_t* ts_off;
  const int32_t* cell_n;
  const uint64_t* cell_key;
  const float4* mf4;
  const int32_t* mgid;
  const float4* mnrm;
  int has_normals;
  const int8_t* sign;
  const float* d_sdf;
  const float* d_grad;
  float* d_xq;
  float* d_x;
  double* abar;  // per member
};

// Per (winner, tile of up to kTW queries), two passes.
//  Pass 1, a thread per query: the forward recomputation around the nearest sample x_n -- with p = x - x_n and
//  delta_i = x_n - x_i (so r_i = x - x_i = p + delta_i) and the exponent relative to x_n (excess_sq):
//    f' = sum_i alpha_i k'_i (compensated),  D = sum_i alpha_i k'_i delta_i,  M = sum_i alpha_i k'_i delta_i delta_i^T,
//  hence G = sum_i alpha_i k'_i r_i = f' p + D and, for any v, H v = sum_i alpha_i k'_i r_i (r_i . v) =
//  f' (p.v) p + (p.v) D + p (D.v) + M v.  (Sums of r_i r_i^T would hold d^2 p p^T-sized entries whose product
//  with v -- orthogonal to the gradient -- cancels; the offsets delta_i are small.)  Then the cotangent scalars
//  fb = dL/df', v (from d grad) and
//    x_bar = -2 lambda (fb G + H v) + f' v
//  (the sum over samples of alpha_i k'_i (v - 2 lambda r_i (r_i . v)) folded into f' and H v), written out; the
//  query's fb, v, x_n and 2 p go to shared memory.
//  Pass 2, a thread per sample (and per group of queries when the cell is small): over the tile's queries,
//    alpha_bar_i += k'_i c,   X_bar_i += alpha_i k'_i (2 lambda c r_i - v),   c = fb + r_i . v,
//  accumulated in registers, then added once per sample to the global accumulators.
// A query whose f' <= 0 (the distance fallback) has fb = 0 and its term on the nearest sample added directly.
// With the Matern 3/2 kernel (u = -log f'/lambda + d, k'_i = (1 + lambda r_i) w_i, w_i = e^{-lambda (r_i - d)},
// grad k'_i = -lambda^2 w_i r_i): fb = -s d_sdf / (lambda f'), G = sum_i alpha_i w_i r_i, the gradient output's
// Jacobian sum_i alpha_i w_i (I - (lambda / |r_i|) r_i r_i^T), so that
//   x_bar = -lambda^2 fb G + f_w v - lambda H' v  (f_w = sum alpha_i w_i, H' = sum (alpha_i w_i / |r_i|) r_i r_i^T),
//   alpha_bar_i += fb k'_i + w_i (r_i . v),  X_bar_i += alpha_i w_i ((lambda^2 fb + lambda (r_i . v) / |r_i|) r_i - v).
constexpr int kTQ = 128;  // backward tile: queries (pass 1) and threads

template <bool MATERN>
__global__ void __launch_bounds__(kTQ) k_bw_query(BwArgs a, const float* xq, Params p) {
  extern __shared__ __align__(16) float4 s_x[];  // [n_max] samples | per query: (x, fb) (w, -) (x_n, -) (v, -) |
                                                 // [kTQ][4] group partial sums
  __shared__ int s_tile;
  __shared__ float s_bh[3], s_bl[3];
  float4* QA = s_x + p.n_max;
  float4* QW = QA + kTQ;
  float4* QN = QW + kTQ;
  float4* QV = QN + kTQ;
  float4* RED = QV + kTQ;
  const int tid = threadIdx.x;
  const float lam = (float)p.lambda;
  const float c1 = lam * kLog2e;
  const float tl = 2.f * lam;
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
    for (int i = tid; i < n; i += kTQ) s_x[i] = __ldg(a.mf4 + m0 + i);
    if (tid == 0) {
      int cc[3];
      unpack_key(a.cell_key[g], cc[0], cc[1], cc[2]);
      for (int j = 0; j < 3; ++j) base_split(p.o[j], cc[j], p.h, s_bh[j], s_bl[j]);
    }
    __syncthreads();
    // ---- pass 1: a thread per query ----
    if (tid < tile.z) {
      const int q = a.sorted[tile.y + tid];
      float ql[3] = {0.f, 0.f, 0.f};
      for (int j = 0; j < p.dim; ++j) ql[j] = local32(xq[(int64_t)q * p.dim + j], s_bh[j], s_bl[j]);
      float m = INFINITY;
      int nn = 0;
      for (int i = 0; i < n; ++i) {
        const float4 v = s_x[i];
        const float dx = ql[0] - v.x, dy = ql[1] - v.y, dz = ql[2] - v.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (r2 < m) {
          m = r2;
          nn = i;
        }
      }
      const float4 xn = s_x[nn];
      const float px = ql[0] - xn.x, py = ql[1] - xn.y, pz = ql[2] - xn.z;
      const float wx = 2.f * px, wy = 2.f * py, wz = 2.f * pz;
      const float zmin = sqrtf(m);
      // f' (compensated); the gradient weights' sums fw, D (G = fw p + D); the Jacobian weights' sums fc, Dc, M
      // (RBF: the same weights; Matern: alpha_i w_i / |r_i|)
      float f = 0.f, comp = 0.f, fw = 0.f, D0 = 0.f, D1 = 0.f, D2 = 0.f;
      float fc = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
      float M00 = 0.f, M01 = 0.f, M02 = 0.f, M11 = 0.f, M12 = 0.f, M22 = 0.f;
      for (int i = 0; i < n; ++i) {
        const float4 v = s_x[i];
        const float ax = v.x - xn.x, ay = v.y - xn.y, az = v.z - xn.z;  // -delta_i
        const float e = fmaf(ax, ax - wx, fmaf(ay, ay - wy, az * (az - wz)));
        float ak, aw, ac;
        if (MATERN) {
          const float r2 = m + e, z = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
          const float den = z + zmin;
          const float y = den > 0.f ? fmaxf(e, 0.f) * __frcp_rn(den) : 0.f;
          aw = v.w * ex2(-c1 * y);
          ak = aw * fmaf(lam, z, 1.f);
          ac = z > 0.f ? aw * __frcp_rn(z) : 0.f;
        } else {
          ak = v.w * ex2(-c1 * e);
          aw = ak;
          ac = ak;
        }
        const float y = ak - comp;
        const float tt = f + y;
        comp = (tt - f) - y;
        f = tt;
        fw += aw;
        D0 -= aw * ax;
        D1 -= aw * ay;
        D2 -= aw * az;
        const float bx = ac * ax, by = ac * ay, bz = ac * az;
        if (MATERN) {
          fc += ac;
          C0 -= bx;
          C1 -= by;
          C2 -= bz;
        }
        M00 = fmaf(bx, ax, M00);
        M01 = fmaf(bx, ay, M01);
        M02 = fmaf(bx, az, M02);
        M11 = fmaf(by, ay, M11);
        M12 = fmaf(by, az, M12);
        M22 = fmaf(bz, az, M22);
      }
      f -= comp;
      if (!MATERN) {
        fw = f;  // the compensated sum
        fc = f;
        C0 = D0;
        C1 = D1;
        C2 = D2;
      }
      const float G0 = fmaf(fw, px, D0), G1 = fmaf(fw, py, D1), G2 = fmaf(fw, pz, D2);
      float s = 1.f;
      if (a.sign) {
        s = a.sign[q] < 0 ? -1.f : 1.f;
      } else if (p.sign_mode == 1 && a.has_normals) {
        const float4 nv = a.mnrm[m0 + nn];
        s = (nv.x * (ql[0] - xn.x) + nv.y * (ql[1] - xn.y) + nv.z * (ql[2] - xn.z)) >= 0.f ? 1.f : -1.f;
      }
      const float ub = s * a.d_sdf[q];
      float fb = 0.f;
      const bool fallback = !(f > 0.f);
      if (!fallback) {
        if (MATERN) {
          fb = fmaf(-logf(f), 1.f / lam, zmin) > 0.f ? -ub / (lam * f) : 0.f;
        } else {
          const float u2 = fmaf(-logf(f), 1.f / lam, m);
          fb = u2 > 0.f ? -ub / (2.f * lam * sqrtf(u2) * f) : 0.f;
        }
      }
      float v0 = 0.f, v1 = 0.f, v2 = 0.f;
      if (a.d_grad) {
        const float gn = sqrtf(G0 * G0 + G1 * G1 + G2 * G2);
        if (gn > 0.f) {
          const float g0 = G0 / gn, g1 = G1 / gn, g2 = G2 / gn;
          const float b0 = a.d_grad[(int64_t)q * p.dim + 0], b1 = a.d_grad[(int64_t)q * p.dim + 1];
          const float b2 = p.dim == 3 ? a.d_grad[(int64_t)q * p.dim + 2] : 0.f;
          const float dot = g0 * b0 + g1 * b1 + g2 * b2;
          const float sc = s / gn;
          v0 = sc * (b0 - g0 * dot);
          v1 = sc * (b1 - g1 * dot);
          v2 = sc * (b2 - g2 * dot);
        }
      }
      // x_bar = -cg fb G + fw v - beta H v with H v = fc (p.v) p + (p.v) C + p (C.v) + M v; RBF cg = beta = 2 lambda,
      // Matern cg = lambda^2, beta = lambda (the 1/|r_i| is inside the weights of fc, C, M)
      const float pv = fmaf(px, v0, fmaf(py, v1, pz * v2)), cv = fmaf(C0, v0, fmaf(C1, v1, C2 * v2));
      const float fpv = fc * pv;
      const float hv0 = fmaf(fpv, px, fmaf(pv, C0, fmaf(px, cv, fmaf(M00, v0, fmaf(M01, v1, M02 * v2)))));
      const float hv1 = fmaf(fpv, py, fmaf(pv, C1, fmaf(py, cv, fmaf(M01, v0, fmaf(M11, v1, M12 * v2)))));
      const float hv2 = fmaf(fpv, pz, fmaf(pv, C2, fmaf(pz, cv, fmaf(M02, v0, fmaf(M12, v1, M22 * v2)))));
      const float cg = MATERN ? lam * lam : tl, beta = MATERN ? lam : tl;
      float xb0 = fmaf(-cg * fb, G0, fmaf(-beta, hv0, fw * v0));
      float xb1 = fmaf(-cg * fb, G1, fmaf(-beta, hv1, fw * v1));
      float xb2 = fmaf(-cg * fb, G2, fmaf(-beta, hv2, fw * v2));
      if (fallback && m > 0.f) {
        // u = distance to the nearest sample: its own derivative, on the query and on that sample
        const float d = sqrtf(m);
        const float e0 = ub * (ql[0] - xn.x) / d, e1 = ub * (ql[1] - xn.y) / d, e2 = ub * (ql[2] - xn.z) / d;
        xb0 += e0;
        xb1 += e1;
        xb2 += e2;
        const int gid = a.mgid[m0 + nn];
        atomicAdd(&a.d_x[(int64_t)gid * p.dim + 0], -e0);
        atomicAdd(&a.d_x[(int64_t)gid * p.dim + 1], -e1);
        if (p.dim == 3) atomicAdd(&a.d_x[(int64_t)gid * p.dim + 2], -e2);
      }
      a.d_xq[(int64_t)q * p.dim + 0] = xb0;
      a.d_xq[(int64_t)q * p.dim + 1] = xb1;
      if (p.dim == 3) a.d_xq[(int64_t)q * p.dim + 2] = xb2;
      QA[tid] = make_float4(ql[0], ql[1], ql[2], fb);
      QW[tid] = make_float4(wx, wy, wz, 0.f);
      QN[tid] = make_float4(xn.x, xn.y, xn.z, m);
      QV[tid] = make_float4(v0, v1, v2, 0.f);
    }
    __syncthreads();
    // ---- pass 2: a thread per (sample, group of queries) ----
    const int nrep = n < kTQ ? kTQ / n : 1;  // query groups when the cell is small
    const int grp = tid / (n < kTQ ? n : kTQ);
    const int nq = tile.z;
    for (int i0 = 0; i0 < n; i0 += kTQ) {
      const int i = i0 + (n < kTQ ? tid - grp * n : tid);
      const bool act = grp < nrep && i < n;
      float ab = 0.f, X0 = 0.f, X1 = 0.f, X2 = 0.f;
      if (act) {
        const float4 xi = s_x[i];
        for (int qq = grp; qq < nq; qq += nrep) {
          const float4 A = QA[qq], W = QW[qq], Nn = QN[qq], V = QV[qq];
          const float r0 = A.x - xi.x, r1 = A.y - xi.y, r2 = A.z - xi.z;
          const float e = excess_sq(xi.x, xi.y, xi.z, Nn.x, Nn.y, Nn.z, W.x, W.y, W.z);
          const float rv = fmaf(r0, V.x, fmaf(r1, V.y, r2 * V.z));
          float t2, aw;
          if (MATERN) {
            const float rr = Nn.w + e, z = rr > 0.f ? rr * rsqrtf(rr) : 0.f, zm = sqrtf(Nn.w);
            const float den = z + zm;
            const float y = den > 0.f ? fmaxf(e, 0.f) * __frcp_rn(den) : 0.f;
            const float wg = ex2(-c1 * y);
            ab = fmaf(A.w * fmaf(lam, z, 1.f), wg, fmaf(wg, rv, ab));
            aw = xi.w * wg;
            t2 = fmaf(lam * lam, A.w, z > 0.f ? lam * rv * __frcp_rn(z) : 0.f);
          } else {
            const float kp = ex2(-c1 * e);
            const float c = rv + A.w;
            ab = fmaf(kp, c, ab);
            aw = xi.w * kp;
            t2 = tl * c;
          }
          X0 = fmaf(aw, fmaf(t2, r0, -V.x), X0);
          X1 = fmaf(aw, fmaf(t2, r1, -V.y), X1);
          X2 = fmaf(aw, fmaf(t2, r2, -V.z), X2);
        }
      }
      if (nrep > 1) {  // combine the query groups of each sample
        RED[tid] = make_float4(ab, X0, X1, X2);
        __syncthreads();
        if (grp == 0 && act)
          for (int r = 1; r < nrep; ++r) {
            const float4 o = RED[r * n + tid];
            ab += o.x;
            X0 += o.y;
            X1 += o.z;
            X2 += o.w;
          }
      }
      if (grp == 0 && act) {
        atomicAdd(&a.abar[m0 + i], (double)ab);
        const int gid = a.mgid[m0 + i];
        atomicAdd(&a.d_x[(int64_t)gid * p.dim + 0], X0);
        atomicAdd(&a.d_x[(int64_t)gid * p.dim + 1], X1);
        if (p.dim == 3) atomicAdd(&a.d_x[(int64_t)gid * p.dim + 2], X2);
      }
    }
    __syncthreads();
  }
}

// per touched cell: b = A^{-1} alpha_bar.  b0 = L^{-T} L^{-1} alpha_bar with the FP32 L^{-1}; one step of
// iterative refinement against the FP64 factor, r = alpha_bar - L (L^T b0) (the only FP64 work, N^2
// FMAs), b = b0 + L^{-T} L^{-1} r; then the alpha-path X_bar terms in FP32.
__device__ void linv_solve32(const float* Lb, int n, const float* rhs, float* y, float* out, bool add) {
  // y = L^{-1} rhs (rows over threads; 8 consecutive rows share a 32-byte sector per column)
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const float* row = Lb + linv_block_off(j >> 3) + (j & 7);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;  // four independent chains
    int i = 0;
    for (; i + 3 <= j; i += 4) {
      a0 = fmaf(row[(int64_t)i * 8], rhs[i], a0);
      a1 = fmaf(row[(int64_t)(i + 1) * 8], rhs[i + 1], a1);
      a2 = fmaf(row[(int64_t)(i + 2) * 8], rhs[i + 2], a2);
      a3 = fmaf(row[(int64_t)(i + 3) * 8], rhs[i + 3], a3);
    }
    for (; i <= j; ++i) a0 = fmaf(row[(int64_t)i * 8], rhs[i], a0);
    y[j] = (a0 + a1) + (a2 + a3);
  }
  __syncthreads();
  // out (+)= L^{-T} y (columns over threads; the 8 rows of a block at one column are contiguous)
  const int nb = (n + 7) >> 3;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float acc = 0.f;
    for (int R = i >> 3; R < nb; ++R) {
      const float4* v = reinterpret_cast<const float4*>(Lb + linv_block_off(R) + (int64_t)i * 8);
      const float4 l0 = __ldg(v), l1 = __ldg(v + 1);
      const float* yy = y + 8 * R;
      const int rmax = min(8, n - 8 * R);
      const float lr[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
      for (int r = 0; r < rmax; ++r) acc = fmaf(lr[r], yy[r], acc);
    }
    out[i] = add ? out[i] + acc : acc;
  }
  __syncthreads();
}

constexpr int kBwCellThreads = 64;  // two warps per cell: ~70-row cells keep most lanes busy, 32 cells per SM
constexpr int kBwCellSmallN = 128;  // the small-cell launch: shared memory for at most this many samples

template <bool MATERN>
__global__ void __launch_bounds__(kBwCellThreads) k_bw_cell(const int64_t* qcnt, int64_t G, const int64_t* ts_off,
                                                 const int32_t* cell_n, const int64_t* chol_off, const double* chol64,
                                                 const int64_t* linv_off, const float* linv32, const float4* mf4,
                                                 const int32_t* mgid, const double* abar, Params p, float* d_x,
                                                 int nlo, int nhi) {
  extern __shared__ double sh[];  // [n] alpha_bar, [n] t, [n] b0 (double), then floats: rhs, y, b
  for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
    if (qcnt[g] == 0) continue;
    const int n = cell_n[g];
    if (n < nlo || n > nhi) continue;  // another launch's size class
    const int64_t m0 = ts_off[g];
    const double* L = chol64 + chol_off[g];
    const float* Lb = linv32 + linv_off[g];
    double* sa = sh;
    double* st = sh + n;
    double* sbd = sh + 2 * n;
    float* srhs = reinterpret_cast<float*>(sh + 3 * n);
    float* sy = srhs + n;
    float* sb = sy + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      sa[i] = abar[m0 + i];
      srhs[i] = (float)sa[i];
    }
    __syncthreads();
    linv_solve32(Lb, n, srhs, sy, sb, false);  // b0
    for (int i = threadIdx.x; i < n; i += blockDim.x) sbd[i] = (double)sb[i];  // converted once, not per FMA
    __syncthreads();
    // t = L^T b0: rows in lockstep, threads over columns k (coalesced row reads)
    for (int k = threadIdx.x; k < n; k += blockDim.x) st[k] = 0.0;
    for (int k0 = 0; k0 < n; k0 += blockDim.x) {
      const int k = k0 + threadIdx.x;
      double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;  // four independent chains (DFMA latency ~64 cycles)
      // a warp walks rows from its first lane's column so that a row's loads coalesce; entries above the
      // diagonal (k > i, read in bounds from the following row) are masked to zero
      int i = k0 + (threadIdx.x & ~31);
      if (k < n) {
        for (; i + 3 < n; i += 4) {
          c0 = fma(k <= i ? L[tri_sz(i) + k] : 0.0, sbd[i], c0);
          c1 = fma(k <= i + 1 ? L[tri_sz(i + 1) + k] : 0.0, sbd[i + 1], c1);
          c2 = fma(k <= i + 2 ? L[tri_sz(i + 2) + k] : 0.0, sbd[i + 2], c2);
          c3 = fma(k <= i + 3 ? L[tri_sz(i + 3) + k] : 0.0, sbd[i + 3], c3);
        }
        for (; i < n; ++i) c0 = fma(k <= i ? L[tri_sz(i) + k] : 0.0, sbd[i], c0);
        st[k] = (c0 + c1) + (c2 + c3);
      }
    }
    __syncthreads();
    // r = alpha_bar - L t (rows over threads)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double* Li = L + (int64_t)i * (i + 1) / 2;
      double c0 = sa[i], c1 = 0.0, c2 = 0.0, c3 = 0.0;
      int k = 0;
      for (; k + 3 <= i; k += 4) {
        c0 = fma(-Li[k], st[k], c0);
        c1 = fma(-Li[k + 1], st[k + 1], c1);
        c2 = fma(-Li[k + 2], st[k + 2], c2);
        c3 = fma(-Li[k + 3], st[k + 3], c3);
      }
      for (; k <= i; ++k) c0 = fma(-Li[k], st[k], c0);
      srhs[i] = (float)((c0 + c1) + (c2 + c3));
    }
    __syncthreads();
    linv_solve32(Lb, n, srhs, sy, sb, true);  // b = b0 + L^{-T} L^{-1} r
    const float c1 = (float)p.lambda * kLog2e;
    const float tl = 2.f * (float)p.lambda, cm = (float)(p.lambda * p.lambda);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float4 xi = mf4[m0 + i];
      const float bi = sb[i], ai = xi.w;
      float X0 = 0.f, X1 = 0.f, X2 = 0.f;
      for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        const float4 xj = mf4[m0 + j];
        const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        // grad_{x_i} A_ij = -cg w_ij (x_i - x_j): RBF cg w = 2 lambda K_ij, Matern lambda^2 e^{-lambda r_ij}
        const float cw = MATERN ? cm * ex2(-c1 * sqrt_approx(r2)) : tl * ex2(-c1 * r2);
        const float cf = cw * fmaf(bi, xj.w, sb[j] * ai);
        X0 = fmaf(cf, dx, X0);
        X1 = fmaf(cf, dy, X1);
        X2 = fmaf(cf, dz, X2);
      }
      const int gid = mgid[m0 + i];
      atomicAdd(&d_x[(int64_t)gid * p.dim + 0], X0);
      atomicAdd(&d_x[(int64_t)gid * p.dim + 1], X1);
      if (p.dim == 3) atomicAdd(&d_x[(int64_t)gid * p.dim + 2], X2);
    }
    __syncthreads();
  }
}

}  // namespace

ksdf_status run_backward(ksdf_ctx* c, const float* xq, int64_t Q, const int8_t* sign, const int32_t* winner,
                         const float* d_sdf, const float* d_grad, float* d_xq, float* d_x) {
  cudaStream_t st = c->stream;
  const Params& p = c->p;
  Model& m = c->m;
  const int64_t G = m.G;
  uint32_t* stw = ptr<uint32_t>(c->status_word);
  KSDF_CUDA(c, ensure(c->ws[WS_QRANK], sizeof(int32_t) * Q));
  KSDF_CUDA(c, ensure(c->ws[WS_QWSORT], sizeof(int32_t) * Q));
  KSDF_CUDA(c, ensure(c->ws[WS_CELLQ], sizeof(int64_t) * (4 * G + 8)));
  const int64_t max_tiles = Q / kTW + G + 1;
  KSDF_CUDA(c, ensure(c->ws[WS_TILE], sizeof(int4) * max_tiles));
  KSDF_CUDA(c, ensure(c->ws[WS_BW], sizeof(double) * (m.M + 1)));
  int32_t* rank = ptr<int32_t>(c->ws[WS_QRANK]);
  int32_t* sorted = ptr<int32_t>(c->ws[WS_QWSORT]);
  int64_t* cb = ptr<int64_t>(c->ws[WS_CELLQ]);
  int64_t *cnt = cb, *off = cb + G, *nt = cb + 2 * G, *toff = cb + 3 * G, *tot = cb + 4 * G;
  int* counter = reinterpret_cast<int*>(tot + 2);
  int4* tiles = ptr<int4>(c->ws[WS_TILE]);
  double* abar = ptr<double>(c->ws[WS_BW]);
  cudaEvent_t e_b = prof_begin(c), e0 = prof_begin(c);
  KSDF_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int64_t) * G, st));
  KSDF_CUDA(c, cudaMemsetAsync(tot, 0, sizeof(int64_t) * 4, st));
  KSDF_CUDA(c, cudaMemsetAsync(abar, 0, sizeof(double) * (m.M + 1), st));
  launch(k_bw_count, ceil_div(Q, 256), 256, 0, st, winner, Q, G, rank, cnt, d_xq, p.dim, stw);
  KSDF_CUDA(c, scan_i64(cnt, off, G, nullptr, c->ws[WS_SCAN], st));
  launch(k_ntiles_w, ceil_div(G, 256), 256, 0, st, cnt, G, nt);
  KSDF_CUDA(c, scan_i64(nt, toff, G, &tot[0], c->ws[WS_SCAN], st));
  launch(k_bw_scatter, ceil_div(Q, 256), 256, 0, st, winner, rank, Q, G, off, sorted);
  launch(k_bw_tiles, ceil_div(G, 256), 256, 0, st, cnt, off, toff, G, tiles);
  prof_end(c, e0, "backward.group");
  BwArgs a;
  a.tiles = tiles;
  a.n_tiles = &tot[0];
  a.counter = counter;
  a.sorted = sorted;
  a.ts_off = ptr<int64_t>(m.ts_off);
  a.cell_n = ptr<int32_t>(m.n);
  a.cell_key = ptr<uint64_t>(m.key);
  a.mf4 = ptr<float4>(m.mf4);
  a.mgid = ptr<int32_t>(m.mgid);
  a.mnrm = m.has_normals ? ptr<float4>(m.mnrm) : nullptr;
  a.has_normals = m.has_normals ? 1 : 0;
  a.sign = sign;
  a.d_sdf = d_sdf;
  a.d_grad = d_grad;
  a.d_xq = d_xq;
  a.d_x = d_x;
  a.abar = abar;
  const size_t smem = sizeof(float4) * (p.n_max + 5 * kTQ);
  const bool matern = p.kernel == KSDF_KERNEL_MATERN32;
  auto kq = matern ? k_bw_query<true> : k_bw_query<false>;
  KSDF_CUDA(c, cudaFuncSetAttribute(kq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  KSDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kq, kTQ, smem));
  e0 = prof_begin(c);
  launch(kq, std::max(1, occ) * c->num_sms, kTQ, smem, st, a, xq, p);
  prof_end(c, e0, "backward.query");
  e0 = prof_begin(c);
  // two size classes, so that the many small cells run with shared memory for their own size (more CTAs per SM
  // to hide the factors' load latency); the larger cells beside them on an auxiliary stream
  auto kc = matern ? k_bw_cell<true> : k_bw_cell<false>;
  const int maxn = std::max(m.max_n, 1), nsplit = std::min(maxn, kBwCellSmallN);
  const bool two = maxn > nsplit;
  if (two) KSDF_CUDA(c, fork_streams(c));
  for (int part = 0; part < (two ? 2 : 1); ++part) {
    const int nlo = part == 0 ? 0 : nsplit + 1, nhi = part == 0 ? nsplit : maxn;
    const size_t smem2 = (sizeof(double) + sizeof(float)) * 3 * (size_t)nhi;
    KSDF_CUDA(c, cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    int occ2 = 0;
    KSDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, kc, kBwCellThreads, smem2));
    const unsigned grid2 = (unsigned)std::min<int64_t>(G, (int64_t)std::max(1, occ2) * c->num_sms);
    launch(kc, std::max(1u, grid2), kBwCellThreads, smem2, part == 0 ? st : c->aux[0], cnt, G,
           ptr<int64_t>(m.ts_off), ptr<int32_t>(m.n), ptr<int64_t>(m.chol_off), ptr<double>(m.chol64),
           ptr<int64_t>(m.linv_off), ptr<float>(m.linv32), ptr<float4>(m.mf4), ptr<int32_t>(m.mgid), abar, p, d_x,
           nlo, nhi);
  }
  if (two) KSDF_CUDA(c, join_streams(c));
  KSDF_CUDA(c, cudaGetLastError());
  prof_end(c, e0, "backward.cell");
  prof_end(c, e_b, "backward");
  return KSDF_OK;
}

}  // namespace ksdf
