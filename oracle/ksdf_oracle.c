/*
 * ksdf_oracle.c -- CPU FP64 oracle of the Kernel-SDF back-end (arXiv 2603.29227).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by the smoke check and by the benchmark's CPU-baseline
 * leg, never by the library.  It is written to be read against the paper, not to be fast: every step
 * is the textbook form of the definition it cites, in the paper's order and notation.
 *
 *   grid / cells / collection boxes      Sec. IV-B.1 (local GPs on overlapping collection boxes)
 *   kernel and inverse transform          Sec. IV-B.2 kernel table: RBF (lambda = 1/(2 l^2), App. I) and
 *                                         Matern 3/2 (lambda = sqrt(3)/l, the kernel scale of Sec. IV-B.1)
 *   posterior mean, gradient, variance    Sec. IV-B.1 posterior equation
 *   adaptive scaling                      App. D (gamma from the distance d to the nearest sample)
 *   min-fusion of the K nearest GPs       Sec. IV-B.1
 *   softmin UDF variance                  Sec. IV-B.3
 *   SDF-gradient variance                 Sec. IV-B.3 (gradient-variance approximation) and App. C
 *   SDF = sign * UDF                      Sec. IV-B.1 (d = s u), sign from the caller or a stand-in
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *   - cells are the grid cells of edge h that contain at least one sample; the collection box of a
 *     cell is the cell expanded by a margin mu on every side, half open [lo, hi);
 *   - a training set larger than n_max keeps the members of rank floor(j*cnt/n_max), j < n_max;
 *   - "the K nearest GPs" are the K valid cells nearest to the query's cell on the integer lattice
 *     (squared lattice distance), ties broken by the packed key, i.e. lexicographic (cz, cy, cx);
 *   - d in the scaling is the distance to the GP's nearest training sample (so max k' = 1);
 *   - f' <= 0 gives u = d (flagged); a negative argument of the square root is clamped to 0;
 *   - the softmin alpha defaults to lambda (the kernel ablation treats them as the same scale);
 *   - winner ties go to the first candidate in list order; the nearest sample tie to the lowest id;
 *   - in App. C the matrix printed for grad_{x_i} g has grad_{x_i} g_k as its k-th column (its first term
 *     is v_i w^T: column k is w_k v_i, the derivative of g_k along x_i); V[grad_k u] sums the squared norms
 *     of those columns; a query on a sample (z_i = 0, direction undefined) gets +inf.
 * Parity of every function here is pinned by tests/test_oracle_*.py (closed forms, brute force,
 * limits, invariants, finite differences).
 */
#include "ksdf_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KO_BIAS (1LL << 20) /* cell coordinates live in [-2^20, 2^20) */

struct ko_model {
  ko_params p;
  int dim;
  int64_t S;
  double* x;   /* S x dim */
  double* var; /* S */
  double* nrm; /* S x dim or NULL */
  int64_t G;
  uint64_t* key;    /* G, strictly ascending */
  int64_t* cc;      /* G x 3 integer cell coordinates */
  int32_t* status;  /* KO_CELL_* */
  int64_t* own_off; /* G+1: samples binned into the cell (ascending id) */
  int64_t* own_id;
  int64_t* ts_off; /* G+1: training sets (ascending id) */
  int64_t* ts_id;
  double** alpha; /* per cell, N_g */
  double** L;     /* per cell, N_g x N_g row-major lower-triangular Cholesky factor */
  int64_t n_valid;
  int64_t* valid; /* ids of cells with status OK, ascending */
};

/* ------------------------------------------------------------------------------------------------ */
/* threads                                                                                          */

int ko_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int ko_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------------------ */
/* grid                                                                                             */

static double alpha_softmin(const ko_params* p) { return p->softmin_alpha > 0 ? p->softmin_alpha : p->lambda; }

/* kernel table (Sec. IV-B.2) as a function of the squared distance r2 */
static double kernel_k(const ko_params* p, double r2) {
  if (p->kernel == KO_KERNEL_MATERN32) {
    const double r = sqrt(r2);
    return (1.0 + p->lambda * r) * exp(-p->lambda * r);
  }
  return exp(-p->lambda * r2);
}

/* The scaled kernel k' = gamma k (App. D) of a sample at squared distance r2 from a query whose nearest
 * sample is at squared distance d2, and the factor w of its gradient: grad_x k' = -c w (x - x_i) with c from
 * kernel_grad_c (RBF: w = k', c = 2 lambda; Matern 3/2: w = e^{-lambda (r - d)}, c = lambda^2). */
static double kernel_scaled(const ko_params* p, double r2, double d2, double* w) {
  if (p->kernel == KO_KERNEL_MATERN32) {
    const double r = sqrt(r2), e = exp(-p->lambda * (r - sqrt(d2)));
    if (w) *w = e;
    return (1.0 + p->lambda * r) * e;
  }
  const double k = exp(-p->lambda * (r2 - d2));
  if (w) *w = k;
  return k;
}
static double kernel_grad_c(const ko_params* p) {
  return p->kernel == KO_KERNEL_MATERN32 ? p->lambda * p->lambda : 2.0 * p->lambda;
}
/* grad_x k(|x - x_j|) of the unscaled kernel, as -c w (x - x_j): w = k (RBF) or e^{-lambda r} (Matern) */
static double kernel_grad_w(const ko_params* p, double r2) {
  if (p->kernel == KO_KERNEL_MATERN32) return exp(-p->lambda * sqrt(r2));
  return exp(-p->lambda * r2);
}
/* 1/gamma^2 = k(d)^2 / k'(d)^2 factor of the GP variance: e^{-2 lambda d^2} (RBF) or e^{-2 lambda d} (Matern) */
static double kernel_unscale2(const ko_params* p, double d2) {
  if (p->kernel == KO_KERNEL_MATERN32) return exp(-2.0 * p->lambda * sqrt(d2));
  return exp(-2.0 * p->lambda * d2);
}

/* c_j = floor((x_j - o_j) / h) for j < dim, 0 otherwise.  Returns 0 on success. */
static int bin_point(const ko_params* p, const double* x, int64_t c[3]) {
  for (int j = 0; j < 3; ++j) {
    if (j < p->dim) {
      double t = (x[j] - p->origin[j]) / p->cell;
      double f = floor(t);
      if (!(f >= -(double)KO_BIAS && f < (double)KO_BIAS)) return -1; /* also rejects NaN */
      c[j] = (int64_t)f;
    } else {
      c[j] = 0;
    }
  }
  return 0;
}

/* three 21-bit fields, z most significant: ascending key == lexicographic (cz, cy, cx) */
static uint64_t pack_key(const int64_t c[3]) {
  return ((uint64_t)(c[2] + KO_BIAS) << 42) | ((uint64_t)(c[1] + KO_BIAS) << 21) | (uint64_t)(c[0] + KO_BIAS);
}

static void unpack_key(uint64_t k, int64_t c[3]) {
  c[0] = (int64_t)(k & 0x1FFFFF) - KO_BIAS;
  c[1] = (int64_t)((k >> 21) & 0x1FFFFF) - KO_BIAS;
  c[2] = (int64_t)((k >> 42) & 0x1FFFFF) - KO_BIAS;
}

int ko_bin(const ko_params* p, const double* x, int64_t n, uint64_t* keys) {
  if (!p || (p->dim != 2 && p->dim != 3) || !(p->cell > 0)) return KO_ERR_ARG;
  for (int64_t i = 0; i < n; ++i) {
    int64_t c[3];
    if (bin_point(p, x + i * p->dim, c)) return KO_ERR_ARG;
    keys[i] = pack_key(c);
  }
  return KO_OK;
}

/* index of key k among the model's cells, or -1 (binary search over the ascending key array) */
static int64_t find_cell(const ko_model* m, uint64_t k) {
  int64_t lo = 0, hi = m->G - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (m->key[mid] == k) return mid;
    if (m->key[mid] < k) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

typedef struct { uint64_t key; int64_t id; } key_id;

static int cmp_key_id(const void* a, const void* b) {
  const key_id* x = (const key_id*)a;
  const key_id* y = (const key_id*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->id != y->id) return x->id < y->id ? -1 : 1;
  return 0;
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* ------------------------------------------------------------------------------------------------ */
/* fit                                                                                              */

static double sqdist(const double* a, const double* b, int dim) {
  double s = 0.0;
  for (int j = 0; j < dim; ++j) {
    double t = a[j] - b[j];
    s += t * t;
  }
  return s;
}

/* Cholesky A = L L^T of a symmetric N x N matrix (row-major), row by row.  Returns 0 if every pivot
 * is positive, -1 otherwise (the matrix is then not positive definite in FP64). */
static int cholesky(const double* A, double* L, int64_t N) {
  memset(L, 0, sizeof(double) * N * N);
  for (int64_t i = 0; i < N; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      double s = A[i * N + j];
      for (int64_t k = 0; k < j; ++k) s -= L[i * N + k] * L[j * N + k];
      if (i == j) {
        if (!(s > 0.0)) return -1;
        L[i * N + i] = sqrt(s);
      } else {
        L[i * N + j] = s / L[j * N + j];
      }
    }
  }
  return 0;
}

/* solve L y = b (forward substitution) */
static void forward_subst(const double* L, int64_t N, const double* b, double* y) {
  for (int64_t i = 0; i < N; ++i) {
    double s = b[i];
    for (int64_t k = 0; k < i; ++k) s -= L[i * N + k] * y[k];
    y[i] = s / L[i * N + i];
  }
}

/* solve L^T x = y (back substitution) */
static void back_subst(const double* L, int64_t N, const double* y, double* x) {
  for (int64_t i = N - 1; i >= 0; --i) {
    double s = y[i];
    for (int64_t k = i + 1; k < N; ++k) s -= L[k * N + i] * x[k];
    x[i] = s / L[i * N + i];
  }
}

void ko_free(ko_model* m) {
  if (!m) return;
  if (m->alpha) for (int64_t g = 0; g < m->G; ++g) free(m->alpha[g]);
  if (m->L) for (int64_t g = 0; g < m->G; ++g) free(m->L[g]);
  free(m->alpha); free(m->L);
  free(m->x); free(m->var); free(m->nrm);
  free(m->key); free(m->cc); free(m->status);
  free(m->own_off); free(m->own_id); free(m->ts_off); free(m->ts_id);
  free(m->valid);
  free(m);
}

int ko_fit(const ko_params* p, const double* x, const double* var, const double* normals, int64_t S,
           ko_model** out) {
  if (!p || !out || S < 0 || (p->dim != 2 && p->dim != 3) || !(p->cell > 0) || !(p->margin >= 0) ||
      p->n_max < 1 || p->k_cand < 1 || !(p->lambda > 0) ||
      (p->kernel != KO_KERNEL_RBF && p->kernel != KO_KERNEL_MATERN32))
    return KO_ERR_ARG;
  if (S > 0 && !x) return KO_ERR_ARG;
  const int dim = p->dim;
  ko_model* m = (ko_model*)calloc(1, sizeof(ko_model));
  if (!m) return KO_ERR_MEM;
  m->p = *p;
  m->dim = dim;
  m->S = S;
  m->x = (double*)malloc(sizeof(double) * (size_t)(S * dim + 1));
  m->var = (double*)malloc(sizeof(double) * (size_t)(S + 1));
  if (!m->x || !m->var) { ko_free(m); return KO_ERR_MEM; }
  if (S) memcpy(m->x, x, sizeof(double) * S * dim);
  for (int64_t i = 0; i < S; ++i) m->var[i] = var ? var[i] : 0.0;
  if (normals) {
    m->nrm = (double*)malloc(sizeof(double) * (size_t)(S * dim + 1));
    if (!m->nrm) { ko_free(m); return KO_ERR_MEM; }
    memcpy(m->nrm, normals, sizeof(double) * S * dim);
  }
  for (int64_t i = 0; i < S * dim; ++i) if (!isfinite(m->x[i])) { ko_free(m); return KO_ERR_ARG; }
  for (int64_t i = 0; i < S; ++i) if (!(m->var[i] >= 0) || !isfinite(m->var[i])) { ko_free(m); return KO_ERR_ARG; }

  /* 1. bin every sample, sort (key, id) */
  key_id* kid = (key_id*)malloc(sizeof(key_id) * (size_t)(S + 1));
  if (!kid) { ko_free(m); return KO_ERR_MEM; }
  for (int64_t i = 0; i < S; ++i) {
    int64_t c[3];
    if (bin_point(p, m->x + i * dim, c)) { free(kid); ko_free(m); return KO_ERR_ARG; }
    kid[i].key = pack_key(c);
    kid[i].id = i;
  }
  qsort(kid, (size_t)S, sizeof(key_id), cmp_key_id);

  /* 2. distinct keys are the cells, numbered in ascending key order */
  int64_t G = 0;
  for (int64_t i = 0; i < S; ++i) if (i == 0 || kid[i].key != kid[i - 1].key) ++G;
  m->G = G;
  m->key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(G + 1));
  m->cc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(3 * G + 1));
  m->status = (int32_t*)calloc((size_t)(G + 1), sizeof(int32_t));
  m->own_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(G + 1));
  m->own_id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S + 1));
  m->ts_off = (int64_t*)calloc((size_t)(G + 1), sizeof(int64_t));
  m->alpha = (double**)calloc((size_t)(G + 1), sizeof(double*));
  m->L = (double**)calloc((size_t)(G + 1), sizeof(double*));
  if (!m->key || !m->cc || !m->status || !m->own_off || !m->own_id || !m->ts_off || !m->alpha || !m->L) {
    free(kid); ko_free(m); return KO_ERR_MEM;
  }
  {
    int64_t g = -1;
    for (int64_t i = 0; i < S; ++i) {
      if (i == 0 || kid[i].key != kid[i - 1].key) {
        ++g;
        m->key[g] = kid[i].key;
        unpack_key(kid[i].key, m->cc + 3 * g);
        m->own_off[g] = i;
      }
      m->own_id[i] = kid[i].id;
    }
    m->own_off[G] = S;
  }
  free(kid);

  /* 3. training sets: samples inside the collection box [o + c h - mu, o + (c+1) h + mu) per axis.
   * A sample in that box has a bin within R = ceil(mu/h) + 1 of c on every axis (one extra cell covers
   * the rounding of the bin quotient), so scanning the own-lists of that neighbourhood is complete. */
  const int64_t R = (int64_t)ceil(p->margin / p->cell) + 1;
  int64_t** ts_tmp = (int64_t**)calloc((size_t)(G + 1), sizeof(int64_t*));
  int64_t* ts_cnt = (int64_t*)calloc((size_t)(G + 1), sizeof(int64_t));
  if (!ts_tmp || !ts_cnt) { free(ts_tmp); free(ts_cnt); ko_free(m); return KO_ERR_MEM; }
  int fail = 0;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t g = 0; g < G; ++g) {
    const int64_t* c = m->cc + 3 * g;
    double lo[3], hi[3];
    for (int j = 0; j < dim; ++j) {
      double base = p->origin[j] + (double)c[j] * p->cell;
      double top = p->origin[j] + (double)(c[j] + 1) * p->cell;
      lo[j] = base - p->margin;
      hi[j] = top + p->margin;
    }
    int64_t cap = 64, n = 0;
    int64_t* buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    if (!buf) { fail = 1; continue; }
    const int64_t zr = dim == 3 ? R : 0;
    for (int64_t dz = -zr; dz <= zr; ++dz)
      for (int64_t dy = -R; dy <= R; ++dy)
        for (int64_t dx = -R; dx <= R; ++dx) {
          int64_t nb[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
          if (nb[0] < -KO_BIAS || nb[0] >= KO_BIAS || nb[1] < -KO_BIAS || nb[1] >= KO_BIAS || nb[2] < -KO_BIAS ||
              nb[2] >= KO_BIAS)
            continue;
          int64_t h = find_cell(m, pack_key(nb));
          if (h < 0) continue;
          for (int64_t t = m->own_off[h]; t < m->own_off[h + 1]; ++t) {
            int64_t id = m->own_id[t];
            const double* xi = m->x + id * dim;
            int inside = 1;
            for (int j = 0; j < dim; ++j) inside &= (xi[j] >= lo[j]) && (xi[j] < hi[j]);
            if (!inside) continue;
            if (n == cap) {
              cap *= 2;
              int64_t* nbuf = (int64_t*)realloc(buf, sizeof(int64_t) * (size_t)cap);
              if (!nbuf) { fail = 1; break; }
              buf = nbuf;
            }
            buf[n++] = id;
          }
        }
    qsort(buf, (size_t)n, sizeof(int64_t), cmp_i64); /* ascending global index */
    if (n > p->n_max) {                              /* rank selection */
      for (int64_t j = 0; j < p->n_max; ++j) buf[j] = buf[(j * n) / p->n_max];
      n = p->n_max;
    }
    ts_tmp[g] = buf;
    ts_cnt[g] = n;
  }
  if (fail) {
    for (int64_t g = 0; g < G; ++g) free(ts_tmp[g]);
    free(ts_tmp); free(ts_cnt); ko_free(m); return KO_ERR_MEM;
  }
  for (int64_t g = 0; g < G; ++g) m->ts_off[g + 1] = m->ts_off[g] + ts_cnt[g];
  m->ts_id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m->ts_off[G] + 1));
  if (!m->ts_id) {
    for (int64_t g = 0; g < G; ++g) free(ts_tmp[g]);
    free(ts_tmp); free(ts_cnt); ko_free(m); return KO_ERR_MEM;
  }
  for (int64_t g = 0; g < G; ++g) {
    memcpy(m->ts_id + m->ts_off[g], ts_tmp[g], sizeof(int64_t) * ts_cnt[g]);
    free(ts_tmp[g]);
  }
  free(ts_tmp);
  free(ts_cnt);

  /* 4. fit every cell: A = K + diag(sigma^2), K_ij = k(|x_i - x_j|) (kernel table); A = L L^T;
   *    alpha = A^{-1} 1 (all labels are f(x_i) = exp(-lambda * 0) = 1, Sec. IV-B.1). */
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t g = 0; g < G; ++g) {
    const int64_t N = m->ts_off[g + 1] - m->ts_off[g];
    const int64_t* ids = m->ts_id + m->ts_off[g];
    if (N == 0) { m->status[g] = KO_CELL_EMPTY; continue; }
    double* A = (double*)malloc(sizeof(double) * (size_t)(N * N));
    double* L = (double*)malloc(sizeof(double) * (size_t)(N * N));
    double* y = (double*)malloc(sizeof(double) * (size_t)N);
    double* one = (double*)malloc(sizeof(double) * (size_t)N);
    double* al = (double*)malloc(sizeof(double) * (size_t)N);
    if (!A || !L || !y || !one || !al) { fail = 1; free(A); free(L); free(y); free(one); free(al); continue; }
    for (int64_t i = 0; i < N; ++i)
      for (int64_t j = 0; j < N; ++j) {
        double r2 = sqdist(m->x + ids[i] * dim, m->x + ids[j] * dim, dim);
        A[i * N + j] = kernel_k(p, r2) + (i == j ? m->var[ids[i]] : 0.0);
      }
    if (cholesky(A, L, N)) {
      m->status[g] = KO_CELL_NOT_PD;
      free(L); free(al);
    } else {
      for (int64_t i = 0; i < N; ++i) one[i] = 1.0;
      forward_subst(L, N, one, y);
      back_subst(L, N, y, al);
      m->L[g] = L;
      m->alpha[g] = al;
      m->status[g] = KO_CELL_OK;
    }
    free(A); free(y); free(one);
  }
  if (fail) { ko_free(m); return KO_ERR_MEM; }
  m->valid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(G + 1));
  if (!m->valid) { ko_free(m); return KO_ERR_MEM; }
  m->n_valid = 0;
  for (int64_t g = 0; g < G; ++g) if (m->status[g] == KO_CELL_OK) m->valid[m->n_valid++] = g;
  *out = m;
  return KO_OK;
}

int64_t ko_num_cells(const ko_model* m) { return m ? m->G : -1; }

int ko_cells(const ko_model* m, uint64_t* keys, int32_t* status, int64_t* ts_off) {
  if (!m) return KO_ERR_ARG;
  if (keys) memcpy(keys, m->key, sizeof(uint64_t) * m->G);
  if (status) memcpy(status, m->status, sizeof(int32_t) * m->G);
  if (ts_off) memcpy(ts_off, m->ts_off, sizeof(int64_t) * (m->G + 1));
  return KO_OK;
}

int ko_members(const ko_model* m, int64_t* ids) {
  if (!m || !ids) return KO_ERR_ARG;
  memcpy(ids, m->ts_id, sizeof(int64_t) * m->ts_off[m->G]);
  return KO_OK;
}

int ko_cell_alpha(const ko_model* m, int64_t g, double* alpha) {
  if (!m || g < 0 || g >= m->G || !alpha) return KO_ERR_ARG;
  if (m->status[g] != KO_CELL_OK) return KO_ERR_NOT_FITTED;
  memcpy(alpha, m->alpha[g], sizeof(double) * (m->ts_off[g + 1] - m->ts_off[g]));
  return KO_OK;
}

int ko_cell_chol(const ko_model* m, int64_t g, double* L) {
  if (!m || g < 0 || g >= m->G || !L) return KO_ERR_ARG;
  if (m->status[g] != KO_CELL_OK) return KO_ERR_NOT_FITTED;
  int64_t N = m->ts_off[g + 1] - m->ts_off[g];
  memcpy(L, m->L[g], sizeof(double) * N * N);
  return KO_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* candidates: the K valid cells nearest to bin b by squared lattice distance, then by key          */

static void candidates_of(const ko_model* m, uint64_t bkey, int32_t* out, int32_t* count) {
  const int K = m->p.k_cand;
  int64_t b[3];
  unpack_key(bkey, b);
  int64_t bestD[K > 0 ? K : 1];
  uint64_t bestK[K > 0 ? K : 1];
  int64_t bestG[K > 0 ? K : 1];
  int n = 0;
  for (int64_t v = 0; v < m->n_valid; ++v) {
    int64_t g = m->valid[v];
    const int64_t* c = m->cc + 3 * g;
    int64_t D = 0;
    for (int j = 0; j < 3; ++j) D += (b[j] - c[j]) * (b[j] - c[j]);
    uint64_t key = m->key[g];
    /* insertion into the sorted top-K list by (D, key) */
    int pos = n;
    while (pos > 0 && (D < bestD[pos - 1] || (D == bestD[pos - 1] && key < bestK[pos - 1]))) --pos;
    if (pos >= K) continue;
    int last = n < K ? n : K - 1;
    for (int t = last; t > pos; --t) { bestD[t] = bestD[t - 1]; bestK[t] = bestK[t - 1]; bestG[t] = bestG[t - 1]; }
    bestD[pos] = D; bestK[pos] = key; bestG[pos] = g;
    if (n < K) ++n;
  }
  for (int t = 0; t < K; ++t) out[t] = t < n ? (int32_t)bestG[t] : -1;
  *count = n;
}

int ko_candidates(const ko_model* m, const uint64_t* bin_keys, int64_t nb, int32_t* out, int32_t* count) {
  if (!m || (nb > 0 && (!bin_keys || !out || !count))) return KO_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < nb; ++i) candidates_of(m, bin_keys[i], out + i * m->p.k_cand, count + i);
  return KO_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* one GP at one query point                                                                        */

typedef struct {
  double u, d2, fp; /* UDF, squared nearest distance, scaled posterior mean f' */
  uint32_t flags;
} gp_val;

/* f' = sum_i alpha_i k'_i, d = nearest-sample distance (App. D scaling): RBF k'_i = exp(-lambda (r_i^2 - d^2)),
 * u = sqrt(-log f' / lambda + d^2); Matern 3/2 k'_i = (1 + lambda r_i) exp(-lambda (r_i - d)),
 * u = -log f' / lambda + d (the scaled inverses of the kernel table). */
static gp_val gp_value(const ko_model* m, int64_t g, const double* x) {
  const int dim = m->dim;
  const int64_t* ids = m->ts_id + m->ts_off[g];
  const int64_t N = m->ts_off[g + 1] - m->ts_off[g];
  const double lam = m->p.lambda;
  gp_val r = {0, INFINITY, 0, 0};
  for (int64_t i = 0; i < N; ++i) {
    double r2 = sqdist(x, m->x + ids[i] * dim, dim);
    if (r2 < r.d2) r.d2 = r2;
  }
  double fp = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double r2 = sqdist(x, m->x + ids[i] * dim, dim);
    fp += m->alpha[g][i] * kernel_scaled(&m->p, r2, r.d2, NULL);
  }
  r.fp = fp;
  if (fp > 0.0 && m->p.kernel == KO_KERNEL_MATERN32) {
    double u = -log(fp) / lam + sqrt(r.d2);
    if (u < 0.0) { r.flags |= KO_FLAG_CLAMPED; u = 0.0; }
    r.u = u;
  } else if (fp > 0.0) {
    double u2 = -log(fp) / lam + r.d2;
    if (u2 < 0.0) { r.flags |= KO_FLAG_CLAMPED; u2 = 0.0; }
    r.u = sqrt(u2);
  } else {
    r.flags |= KO_FLAG_FALLBACK;
    r.u = sqrt(r.d2);
  }
  return r;
}

/* Full outputs of GP g at x: gradient (Sec. IV-B.1), softmin variance (Sec. IV-B.3), GP variance
 * (posterior equation, evaluated through the scaled kernel vector as e^{-2 lambda d^2} |L^{-1} k'|^2)
 * and the sign.  Scratch arrays have length >= N_g. */
static void gp_full(const ko_model* m, int64_t g, const double* x, int has_sign, int8_t sign_in, double* r2,
                    double* kp, double* v, double* sdf, double* grad, double* var_sdf, double* var_f,
                    uint32_t* flags) {
  const int dim = m->dim;
  const int64_t* ids = m->ts_id + m->ts_off[g];
  const int64_t N = m->ts_off[g + 1] - m->ts_off[g];
  const double as = alpha_softmin(&m->p);
  const double* al = m->alpha[g];
  gp_val val = gp_value(m, g, x);
  *flags |= val.flags;

  /* gradient: grad f' = -c sum_i alpha_i w_i (x - x_i) (kernel_scaled); grad u = -grad f' / |grad f'|, the
   * direction of G = sum_i alpha_i w_i (x - x_i) */
  double Gv[3] = {0, 0, 0};
  for (int64_t i = 0; i < N; ++i) {
    const double* xi = m->x + ids[i] * dim;
    double w;
    r2[i] = sqdist(x, xi, dim);
    kp[i] = kernel_scaled(&m->p, r2[i], val.d2, &w);
    for (int j = 0; j < dim; ++j) Gv[j] += al[i] * w * (x[j] - xi[j]);
  }
  double gn = 0.0;
  for (int j = 0; j < dim; ++j) gn += Gv[j] * Gv[j];
  gn = sqrt(gn);

  /* sign */
  int s = 1;
  if (has_sign) {
    s = sign_in < 0 ? -1 : 1;
  } else if (m->p.sign_mode == 1 && m->nrm) {
    int64_t nn = 0; /* training sets are in ascending id order: the first minimum has the lowest id */
    for (int64_t i = 1; i < N; ++i) if (r2[i] < r2[nn]) nn = i;
    const double* xn = m->x + ids[nn] * dim;
    const double* nv = m->nrm + ids[nn] * dim;
    double dot = 0.0;
    for (int j = 0; j < dim; ++j) dot += nv[j] * (x[j] - xn[j]);
    s = dot >= 0.0 ? 1 : -1;
  }
  if (sdf) *sdf = s * val.u;
  if (grad) {
    if (gn > 0.0) {
      for (int j = 0; j < dim; ++j) grad[j] = s * Gv[j] / gn;
    } else {
      for (int j = 0; j < dim; ++j) grad[j] = 0.0;
      *flags |= KO_FLAG_ZERO_GRAD;
    }
  }

  /* softmin variance: z_i = |x - x_i|, s_i = e^{-a z_i} / sum_j e^{-a z_j}, h = s^T z,
   * V[u] = sum_i |grad_{x_i} h|^2 sigma_i^2 = sum_i s_i^2 (a (h - z_i) + 1)^2 sigma_i^2.
   * The common factor e^{a z_min} is divided out of numerator and denominator. */
  if (var_sdf) {
    double zmin = sqrt(val.d2), W = 0.0, hz = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      double z = sqrt(r2[i]);
      double w = exp(-as * (z - zmin));
      W += w;
      hz += w * z;
    }
    double h = hz / W, acc = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      double z = sqrt(r2[i]);
      double si = exp(-as * (z - zmin)) / W;
      double t = as * (h - z) + 1.0;
      acc += si * si * t * t * m->var[ids[i]];
    }
    *var_sdf = acc;
  }

  /* GP variance: V[f] = k(x,x) - k^T (K+Sigma)^{-1} k = 1 - |L^{-1} k|^2, with k = k' / gamma */
  if (var_f) {
    forward_subst(m->L[g], N, kp, v);
    double q = 0.0;
    for (int64_t i = 0; i < N; ++i) q += v[i] * v[i];
    double vf = 1.0 - kernel_unscale2(&m->p, val.d2) * q;
    *var_f = vf > 0.0 ? vf : 0.0;
  }
}

/* ------------------------------------------------------------------------------------------------ */
/* query                                                                                            */

typedef struct {
  int64_t nb;
  uint64_t* keys; /* unique bin keys, ascending */
  int32_t* cand;  /* nb x K */
  int32_t* ncand;
  int64_t* qbin;  /* per query: index into keys */
} bin_table;

static void free_bins(bin_table* t) { free(t->keys); free(t->cand); free(t->ncand); free(t->qbin); }

static int build_bins(const ko_model* m, const double* xq, int64_t Q, bin_table* t) {
  memset(t, 0, sizeof(*t));
  const int K = m->p.k_cand;
  uint64_t* qk = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(Q + 1));
  t->qbin = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Q + 1));
  if (!qk || !t->qbin) { free(qk); free_bins(t); return KO_ERR_MEM; }
  for (int64_t q = 0; q < Q; ++q) {
    int64_t c[3];
    if (bin_point(&m->p, xq + q * m->dim, c)) { free(qk); free_bins(t); return KO_ERR_ARG; }
    qk[q] = pack_key(c);
  }
  t->keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(Q + 1));
  if (!t->keys) { free(qk); free_bins(t); return KO_ERR_MEM; }
  if (Q) memcpy(t->keys, qk, sizeof(uint64_t) * Q);
  qsort(t->keys, (size_t)Q, sizeof(uint64_t), cmp_u64);
  int64_t nb = 0;
  for (int64_t i = 0; i < Q; ++i) if (i == 0 || t->keys[i] != t->keys[nb - 1]) t->keys[nb++] = t->keys[i];
  t->nb = nb;
  for (int64_t q = 0; q < Q; ++q) {
    int64_t lo = 0, hi = nb - 1;
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (t->keys[mid] < qk[q]) lo = mid + 1; else hi = mid;
    }
    t->qbin[q] = lo;
  }
  free(qk);
  t->cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nb * K + 1));
  t->ncand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nb + 1));
  if (!t->cand || !t->ncand) { free_bins(t); return KO_ERR_MEM; }
  return ko_candidates(m, t->keys, nb, t->cand, t->ncand);
}

static int64_t max_ts(const ko_model* m) {
  int64_t mx = 1;
  for (int64_t g = 0; g < m->G; ++g) if (m->ts_off[g + 1] - m->ts_off[g] > mx) mx = m->ts_off[g + 1] - m->ts_off[g];
  return mx;
}

/* min-fusion over the K candidates: u = min_k u_k; winner = first argmin in list order */
static int query_impl(const ko_model* m, const double* xq, int64_t Q, const int8_t* sign, const int32_t* forced,
                      double* sdf, double* grad, double* var_sdf, double* var_f, int32_t* winner, uint32_t* flags,
                      double* cand_u, int32_t* cand_id) {
  if (!m || Q < 0 || (Q > 0 && !xq)) return KO_ERR_ARG;
  const int dim = m->dim, K = m->p.k_cand;
  bin_table t;
  int rc = KO_OK;
  if (!forced) {
    rc = build_bins(m, xq, Q, &t);
    if (rc) return rc;
  } else {
    for (int64_t q = 0; q < Q; ++q)
      if (forced[q] < 0 || forced[q] >= m->G || m->status[forced[q]] != KO_CELL_OK) return KO_ERR_ARG;
  }
  const int64_t NM = max_ts(m);
  int fail = 0;
#pragma omp parallel
  {
    double* r2 = (double*)malloc(sizeof(double) * (size_t)NM);
    double* kp = (double*)malloc(sizeof(double) * (size_t)NM);
    double* v = (double*)malloc(sizeof(double) * (size_t)NM);
    if (!r2 || !kp || !v) fail = 1;
#pragma omp for schedule(dynamic, 64)
    for (int64_t q = 0; q < Q; ++q) {
      if (fail) continue;
      const double* x = xq + q * dim;
      uint32_t fl = 0;
      int64_t best = -1;
      if (forced) {
        best = forced[q];
      } else {
        const int32_t* cl = t.cand + t.qbin[q] * K;
        const int nc = t.ncand[t.qbin[q]];
        double bu = INFINITY, su = INFINITY;
        for (int k = 0; k < K; ++k) {
          if (cand_id) cand_id[q * K + k] = k < nc ? cl[k] : -1;
          if (cand_u) cand_u[q * K + k] = INFINITY;
        }
        for (int k = 0; k < nc; ++k) {
          gp_val gv = gp_value(m, cl[k], x);
          if (cand_u) cand_u[q * K + k] = gv.u;
          if (gv.u < bu) { su = bu; bu = gv.u; best = cl[k]; }
          else if (gv.u < su) { su = gv.u; }
        }
        if (nc >= 2 && su - bu <= 1e-5) fl |= KO_FLAG_NEAR_TIE;
      }
      if (best < 0) {
        fl |= KO_FLAG_NO_GP;
        if (sdf) sdf[q] = INFINITY;
        if (grad) for (int j = 0; j < dim; ++j) grad[q * dim + j] = 0.0;
        if (var_sdf) var_sdf[q] = 0.0;
        if (var_f) var_f[q] = 1.0;
      } else {
        gp_full(m, best, x, sign != NULL, sign ? sign[q] : 0, r2, kp, v, sdf ? sdf + q : NULL,
                grad ? grad + q * dim : NULL, var_sdf ? var_sdf + q : NULL, var_f ? var_f + q : NULL, &fl);
      }
      if (winner) winner[q] = (int32_t)best;
      if (flags) flags[q] = fl;
    }
    free(r2); free(kp); free(v);
  }
  if (!forced) free_bins(&t);
  return fail ? KO_ERR_MEM : rc;
}

static double* promote(const float* xq, int64_t n) {
  double* d = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  if (d) for (int64_t i = 0; i < n; ++i) d[i] = (double)xq[i];
  return d;
}

int ko_query(const ko_model* m, const float* xq, int64_t Q, const int8_t* sign, double* sdf, double* grad,
             double* var_sdf, double* var_f, int32_t* winner, uint32_t* flags, double* cand_u, int32_t* cand_id) {
  if (!m || Q < 0 || (Q > 0 && !xq)) return KO_ERR_ARG;
  double* x = promote(xq, Q * m->dim);
  if (!x) return KO_ERR_MEM;
  int rc = query_impl(m, x, Q, sign, NULL, sdf, grad, var_sdf, var_f, winner, flags, cand_u, cand_id);
  free(x);
  return rc;
}

int ko_query_f64(const ko_model* m, const double* xq, int64_t Q, const int8_t* sign, double* sdf, double* grad,
                 double* var_sdf, double* var_f, int32_t* winner, uint32_t* flags) {
  return query_impl(m, xq, Q, sign, NULL, sdf, grad, var_sdf, var_f, winner, flags, NULL, NULL);
}

int ko_eval_cell(const ko_model* m, const float* xq, int64_t Q, const int32_t* cell, const int8_t* sign,
                 double* sdf, double* grad, double* var_sdf, double* var_f, uint32_t* flags) {
  if (!m || Q < 0 || (Q > 0 && (!xq || !cell))) return KO_ERR_ARG;
  double* x = promote(xq, Q * m->dim);
  if (!x) return KO_ERR_MEM;
  int rc = query_impl(m, x, Q, sign, cell, sdf, grad, var_sdf, var_f, NULL, flags, NULL, NULL);
  free(x);
  return rc;
}

/* SDF-gradient variance (Sec. IV-B.3, App. C) of the queries xq on the given cells: with z_i = |x - x_i|,
 * v_i = (x - x_i) / z_i, softmin weights s_i = e^{-a z_i} / sum_j e^{-a z_j}, h = s^T z,
 * l_i = s_i (a s^T z - a z_i + 1), V = [v_1 .. v_N], g = V (a s s^T z - a diag(s) z + s) (the gradient of h),
 * the matrix of App. C
 *     M_i = a v_i (l_i (v_i - V s) + s_i (v_i - g))^T + (l_i / z_i) (v_i v_i^T - I),
 * whose k-th column is grad_{x_i} g_k, and V[grad_k u] = sum_i |M_i[:, k]|^2 sigma_i^2.  var_grad is Q x dim. */
int ko_var_grad(const ko_model* m, const float* xq, int64_t Q, const int32_t* cell, double* var_grad) {
  if (!m || Q < 0 || (Q > 0 && (!xq || !cell || !var_grad))) return KO_ERR_ARG;
  const int dim = m->dim;
  const double a = alpha_softmin(&m->p);
  for (int64_t q = 0; q < Q; ++q)
    if (cell[q] < 0 || cell[q] >= m->G || m->status[cell[q]] != KO_CELL_OK) return KO_ERR_ARG;
  const int64_t NM = max_ts(m);
  int fail = 0;
#pragma omp parallel
  {
    double* z = (double*)malloc(sizeof(double) * (size_t)NM);
    double* sw = (double*)malloc(sizeof(double) * (size_t)NM);
    double* vv = (double*)malloc(sizeof(double) * (size_t)NM * 3);
    if (!z || !sw || !vv) fail = 1;
#pragma omp for schedule(dynamic, 64)
    for (int64_t q = 0; q < Q; ++q) {
      if (fail) continue;
      double x[3] = {0, 0, 0};
      for (int j = 0; j < dim; ++j) x[j] = (double)xq[q * dim + j];
      const int64_t g = cell[q];
      const int64_t* ids = m->ts_id + m->ts_off[g];
      const int64_t N = m->ts_off[g + 1] - m->ts_off[g];
      double* out = var_grad + q * dim;
      int on_sample = 0;
      double zmin = INFINITY;
      for (int64_t i = 0; i < N; ++i) {
        const double* xi = m->x + ids[i] * dim;
        z[i] = sqrt(sqdist(x, xi, dim));
        if (z[i] == 0.0) on_sample = 1;
        for (int j = 0; j < dim; ++j) vv[i * 3 + j] = z[i] > 0.0 ? (x[j] - xi[j]) / z[i] : 0.0;
        if (z[i] < zmin) zmin = z[i];
      }
      if (on_sample) {
        for (int j = 0; j < dim; ++j) out[j] = INFINITY;
        continue;
      }
      /* softmin weights (the common factor e^{a zmin} cancels) and h = s^T z */
      double W = 0.0;
      for (int64_t i = 0; i < N; ++i) {
        sw[i] = exp(-a * (z[i] - zmin));
        W += sw[i];
      }
      double sz = 0.0;
      for (int64_t i = 0; i < N; ++i) {
        sw[i] /= W;
        sz += sw[i] * z[i];
      }
      /* V s and g = V (a s s^T z - a diag(s) z + s) */
      double Vs[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
      for (int64_t i = 0; i < N; ++i) {
        const double coef = a * sw[i] * sz - a * sw[i] * z[i] + sw[i];
        for (int j = 0; j < dim; ++j) {
          Vs[j] += vv[i * 3 + j] * sw[i];
          gv[j] += vv[i * 3 + j] * coef;
        }
      }
      for (int k = 0; k < dim; ++k) out[k] = 0.0;
      for (int64_t i = 0; i < N; ++i) {
        const double* v = vv + i * 3;
        const double li = sw[i] * (a * sz - a * z[i] + 1.0);
        double w[3];
        for (int j = 0; j < dim; ++j) w[j] = li * (v[j] - Vs[j]) + sw[i] * (v[j] - gv[j]);
        double M[3][3];
        for (int r = 0; r < dim; ++r)
          for (int c = 0; c < dim; ++c) M[r][c] = a * v[r] * w[c] + (li / z[i]) * (v[r] * v[c] - (r == c ? 1.0 : 0.0));
        const double s2 = m->var[ids[i]];
        for (int k = 0; k < dim; ++k) {
          double col = 0.0;
          for (int r = 0; r < dim; ++r) col += M[r][k] * M[r][k];
          out[k] += col * s2;
        }
      }
    }
    free(z); free(sw); free(vv);
  }
  return fail ? KO_ERR_MEM : KO_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* adjoint                                                                                          */

/* Reverse mode through the forward definitions above, for queries grouped by winner cell g, with d held
 * constant (u does not depend on the scale gamma, so this is exact):
 *   RBF        u^2 = -log f'/lambda + d^2:  dL/df' = -s dsdf / (2 lambda u f');
 *   Matern 3/2 u = -log f'/lambda + d:      dL/df' = -s dsdf / (lambda f');
 *   f' = sum_i alpha_i k'_i and grad_x k'_i = -c w_i r_i (kernel_scaled, r_i = x - x_i).
 *   grad output s G/|G| with G = sum_i alpha_i w_i r_i: cotangent on G is v = s (I - g g^T) dgrad / |G|, and
 *   dG/dx = sum_i alpha_i w_i (I - beta_i r_i r_i^T), beta_i = 2 lambda (RBF: grad w = -2 lambda w r) or
 *   lambda / |r_i| (Matern: grad w = -lambda w r / |r|).
 *   alpha = A^{-1} 1 with A_ij = k(|x_i - x_j|) + delta_ij sigma_i^2, grad_{x_m} A_mj = -c w_mj (x_m - x_j)
 *   (kernel_grad_w): with b = A^{-1} alpha_bar, dL/dx_m += sum_j c w_mj (b_m alpha_j + b_j alpha_m)(x_m - x_j).
 * The sign, sigma^2 and the winner choice are constants. */
static int backward_impl(const ko_model* m, const double* xq, int64_t Q, const int8_t* sign, const int32_t* winner_in,
                         const double* d_sdf, const double* d_grad, double* d_xq, double* d_x) {
  if (!m || Q < 0 || (Q > 0 && (!xq || !d_xq || !d_x || (!d_sdf && !d_grad)))) return KO_ERR_ARG;
  const int dim = m->dim;
  const double lam = m->p.lambda, cg = kernel_grad_c(&m->p);
  const int matern = m->p.kernel == KO_KERNEL_MATERN32;
  const int64_t G = m->G;
  int32_t* win = (int32_t*)malloc(sizeof(int32_t) * (size_t)(Q + 1));
  if (!win) return KO_ERR_MEM;
  if (winner_in) {
    for (int64_t q = 0; q < Q; ++q) {
      win[q] = winner_in[q];
      if (win[q] >= G || (win[q] >= 0 && m->status[win[q]] != KO_CELL_OK)) { free(win); return KO_ERR_ARG; }
    }
  } else {
    int rc = query_impl(m, xq, Q, sign, NULL, NULL, NULL, NULL, NULL, win, NULL, NULL, NULL);
    if (rc) { free(win); return rc; }
  }
  /* group queries by winner (counting sort; queries stay in ascending order inside a group) */
  int64_t* qoff = (int64_t*)calloc((size_t)(G + 2), sizeof(int64_t));
  int64_t* qlist = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Q + 1));
  double** xbar = (double**)calloc((size_t)(G + 1), sizeof(double*));
  if (!qoff || !qlist || !xbar) { free(win); free(qoff); free(qlist); free(xbar); return KO_ERR_MEM; }
  for (int64_t q = 0; q < Q; ++q) if (win[q] >= 0) qoff[win[q] + 1]++;
  for (int64_t g = 0; g < G; ++g) qoff[g + 1] += qoff[g];
  {
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(G + 1));
    if (!cur) { free(win); free(qoff); free(qlist); free(xbar); return KO_ERR_MEM; }
    memcpy(cur, qoff, sizeof(int64_t) * G);
    for (int64_t q = 0; q < Q; ++q) if (win[q] >= 0) qlist[cur[win[q]]++] = q;
    free(cur);
  }
  for (int64_t q = 0; q < Q; ++q)
    if (win[q] < 0) for (int j = 0; j < dim; ++j) d_xq[q * dim + j] = 0.0;

  int fail = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t g = 0; g < G; ++g) {
    if (qoff[g + 1] == qoff[g]) continue;
    const int64_t N = m->ts_off[g + 1] - m->ts_off[g];
    const int64_t* ids = m->ts_id + m->ts_off[g];
    const double* al = m->alpha[g];
    double* xb = (double*)calloc((size_t)(N * dim), sizeof(double));
    double* ab = (double*)calloc((size_t)N, sizeof(double));
    double* kp = (double*)malloc(sizeof(double) * (size_t)N);
    double* wv = (double*)malloc(sizeof(double) * (size_t)N);
    double* r = (double*)malloc(sizeof(double) * (size_t)(N * dim));
    double* y = (double*)malloc(sizeof(double) * (size_t)N);
    double* b = (double*)malloc(sizeof(double) * (size_t)N);
    if (!xb || !ab || !kp || !wv || !r || !y || !b) {
      fail = 1; free(xb); free(ab); free(kp); free(wv); free(r); free(y); free(b); continue;
    }
    for (int64_t t = qoff[g]; t < qoff[g + 1]; ++t) {
      const int64_t q = qlist[t];
      const double* x = xq + q * dim;
      double d2 = INFINITY;
      for (int64_t i = 0; i < N; ++i) {
        double r2 = 0.0;
        for (int j = 0; j < dim; ++j) {
          r[i * dim + j] = x[j] - m->x[ids[i] * dim + j];
          r2 += r[i * dim + j] * r[i * dim + j];
        }
        kp[i] = r2; /* temporarily r^2 */
        if (r2 < d2) d2 = r2;
      }
      int64_t nn = 0;
      for (int64_t i = 1; i < N; ++i) if (kp[i] < kp[nn]) nn = i;
      double fp = 0.0, Gv[3] = {0, 0, 0};
      for (int64_t i = 0; i < N; ++i) {
        kp[i] = kernel_scaled(&m->p, kp[i], d2, &wv[i]);
        fp += al[i] * kp[i];
        for (int j = 0; j < dim; ++j) Gv[j] += al[i] * wv[i] * r[i * dim + j];
      }
      /* sign, as in the forward pass */
      int s = 1;
      if (sign) {
        s = sign[q] < 0 ? -1 : 1;
      } else if (m->p.sign_mode == 1 && m->nrm) {
        double dot = 0.0;
        for (int j = 0; j < dim; ++j) dot += m->nrm[ids[nn] * dim + j] * r[nn * dim + j];
        s = dot >= 0.0 ? 1 : -1;
      }
      double xqb[3] = {0, 0, 0};
      const double ub = d_sdf ? s * d_sdf[q] : 0.0;
      if (fp > 0.0) {
        double fb;
        if (matern) {
          double u = -log(fp) / lam + sqrt(d2);
          fb = u > 0.0 ? -ub / (lam * fp) : 0.0;
        } else {
          double u2 = -log(fp) / lam + d2;
          fb = u2 > 0.0 ? -ub / (2.0 * lam * sqrt(u2) * fp) : 0.0;
        }
        for (int j = 0; j < dim; ++j) xqb[j] += fb * (-cg * Gv[j]);
        for (int64_t i = 0; i < N; ++i) {
          for (int j = 0; j < dim; ++j) xb[i * dim + j] += fb * cg * al[i] * wv[i] * r[i * dim + j];
          ab[i] += fb * kp[i];
        }
      } else if (d2 > 0.0) { /* u = |x - x_nn| */
        double d = sqrt(d2);
        for (int j = 0; j < dim; ++j) {
          xqb[j] += ub * r[nn * dim + j] / d;
          xb[nn * dim + j] -= ub * r[nn * dim + j] / d;
        }
      }
      if (d_grad) {
        double gn = 0.0;
        for (int j = 0; j < dim; ++j) gn += Gv[j] * Gv[j];
        gn = sqrt(gn);
        if (gn > 0.0) {
          double gh[3], gb[3], v[3], dot = 0.0;
          for (int j = 0; j < dim; ++j) { gh[j] = Gv[j] / gn; gb[j] = d_grad[q * dim + j]; dot += gh[j] * gb[j]; }
          for (int j = 0; j < dim; ++j) v[j] = s * (gb[j] - gh[j] * dot) / gn;
          for (int64_t i = 0; i < N; ++i) {
            const double* ri = r + i * dim;
            double rv = 0.0, rn = 0.0;
            for (int j = 0; j < dim; ++j) { rv += ri[j] * v[j]; rn += ri[j] * ri[j]; }
            double beta = 2.0 * lam;
            if (matern) beta = rn > 0.0 ? lam / sqrt(rn) : 0.0;
            for (int j = 0; j < dim; ++j) {
              double mv = al[i] * wv[i] * (v[j] - beta * ri[j] * rv); /* (dG/dx)_i v */
              xqb[j] += mv;
              xb[i * dim + j] -= mv;
            }
            ab[i] += wv[i] * rv;
          }
        }
      }
      for (int j = 0; j < dim; ++j) d_xq[q * dim + j] = xqb[j];
    }
    /* through alpha = A^{-1} 1 */
    forward_subst(m->L[g], N, ab, y);
    back_subst(m->L[g], N, y, b);
    for (int64_t i = 0; i < N; ++i) {
      const double* xi = m->x + ids[i] * dim;
      for (int64_t jj = 0; jj < N; ++jj) {
        if (jj == i) continue;
        const double* xj = m->x + ids[jj] * dim;
        double c = cg * kernel_grad_w(&m->p, sqdist(xi, xj, dim)) * (b[i] * al[jj] + b[jj] * al[i]);
        for (int j = 0; j < dim; ++j) xb[i * dim + j] += c * (xi[j] - xj[j]);
      }
    }
    xbar[g] = xb;
    free(ab); free(kp); free(wv); free(r); free(y); free(b);
  }
  if (!fail) {
    for (int64_t g = 0; g < G; ++g) {
      if (!xbar[g]) continue;
      const int64_t N = m->ts_off[g + 1] - m->ts_off[g];
      const int64_t* ids = m->ts_id + m->ts_off[g];
      for (int64_t i = 0; i < N; ++i)
        for (int j = 0; j < dim; ++j) d_x[ids[i] * dim + j] += xbar[g][i * dim + j];
    }
  }
  for (int64_t g = 0; g < G; ++g) free(xbar[g]);
  free(xbar); free(win); free(qoff); free(qlist);
  return fail ? KO_ERR_MEM : KO_OK;
}

int ko_backward(const ko_model* m, const float* xq, int64_t Q, const int8_t* sign, const int32_t* winner,
                const double* d_sdf, const double* d_grad, double* d_xq, double* d_x) {
  if (!m || Q < 0 || (Q > 0 && !xq)) return KO_ERR_ARG;
  double* x = promote(xq, Q * m->dim);
  if (!x) return KO_ERR_MEM;
  int rc = backward_impl(m, x, Q, sign, winner, d_sdf, d_grad, d_xq, d_x);
  free(x);
  return rc;
}

int ko_backward_f64(const ko_model* m, const double* xq, int64_t Q, const int8_t* sign, const int32_t* winner,
                    const double* d_sdf, const double* d_grad, double* d_xq, double* d_x) {
  return backward_impl(m, xq, Q, sign, winner, d_sdf, d_grad, d_xq, d_x);
}
