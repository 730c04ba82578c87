/*
 * ksdf_oracle.h -- interface of the CPU FP64 oracle for the Kernel-SDF back-end query.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, obviously-correct restatement of what the
 * paper's back-end computes.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or helper with the CUDA library under
 * paper_2603_29227_gb300/, and neither side includes the other.
 *
 * All floating-point arithmetic is IEEE binary64.  The library is built with -ffp-contract=off so that
 * no multiply-add is fused: the integer binning and the training-set box tests must be bit-exact.
 *
 * Paper references (Kernel-SDF, arXiv 2603.29227):
 *   Sec. III       SDF definition and eikonal property.
 *   Sec. IV-B.1    log-GP posterior mean, gradient and variance; min-fusion of the K nearest local GPs.
 *   Sec. IV-B.2    kernel table (RBF k(r)=exp(-r^2/2l^2), inverse r(f)=sqrt(-2l^2 log f); Matern 3/2
 *                  k(r)=(1+sqrt3 r/l)exp(-sqrt3 r/l), inverse r(f)=-l log f/sqrt3); scaled inverses.
 *   Sec. IV-B.3    softmin variance of the UDF.
 *   App. D         adaptive scaling (gamma = exp(d^2/2l^2) or exp(sqrt3 d/l), d = distance to the nearest sample).
 *   App. E         softmin limits (used by the tests as pins).
 *   App. F         min-fusion consistency (used by the tests as a magnitude pin).
 * RBF: lambda = 1/(2 l^2) as in App. I, so k(r) = exp(-lambda r^2) and u = sqrt(-log f / lambda).
 * Matern 3/2: lambda = sqrt3/l, so k(r) = (1 + lambda r) exp(-lambda r) and u = -log f / lambda.
 */
#ifndef KSDF_ORACLE_H
#define KSDF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dim;            /* 2 or 3 */
  double origin[3];   /* grid origin o (unused components ignored) */
  double cell;        /* cell edge h > 0 */
  double margin;      /* collection-box margin mu >= 0 */
  int n_max;          /* training-set cap per cell (rank selection above it) */
  int k_cand;         /* K nearest GP cells fused by min */
  double lambda;      /* RBF scale lambda = 1/(2 l^2) */
  double softmin_alpha; /* softmin temperature alpha of Sec. IV-B.3; <= 0 means "equal to lambda" */
  int sign_mode;      /* 0: sign from the caller (or +1 if none); 1: nearest-sample-normal stand-in */
  int kernel;         /* KO_KERNEL_RBF or KO_KERNEL_MATERN32 (kernel table of Sec. IV-B.2) */
} ko_params;

/* Kernels of the kernel table (Sec. IV-B.2) with lambda the scale of the exponent f = exp(-lambda u):
 *   RBF         k(r) = exp(-lambda r^2), lambda = 1/(2 l^2),  u(f) = sqrt(-log f / lambda);
 *   Matern 3/2  k(r) = (1 + lambda r) exp(-lambda r), lambda = sqrt(3)/l (the kernel scale sqrt(3)/lambda of
 *               Sec. IV-B.1), u(f) = -log f / lambda.
 * Scaled (App. D) with gamma = e^{lambda d^2} (RBF) or e^{lambda d} (Matern), d the nearest-sample distance:
 *   u = sqrt(-log f'/lambda + d^2) (RBF),  u = -log f'/lambda + d (Matern). */
enum { KO_KERNEL_RBF = 0, KO_KERNEL_MATERN32 = 1 };

typedef struct ko_model ko_model;

/* Return codes. */
enum { KO_OK = 0, KO_ERR_ARG = 1, KO_ERR_MEM = 2, KO_ERR_NOT_FITTED = 3 };

/* Per-query flag bits (same meaning as the library's). */
enum {
  KO_FLAG_FALLBACK = 1u,  /* winner's f' <= 0: u = distance to its nearest sample */
  KO_FLAG_NO_GP = 2u,     /* no candidate GP at all */
  KO_FLAG_NEAR_TIE = 4u,  /* second-best candidate u within 1e-5 m of the best */
  KO_FLAG_ZERO_GRAD = 8u, /* gradient of f' vanished: grad output is 0 */
  KO_FLAG_CLAMPED = 16u   /* -log f'/lambda + d^2 < 0, clamped to u = 0 */
};

/* Cell status. */
enum { KO_CELL_OK = 0, KO_CELL_EMPTY = 1, KO_CELL_NOT_PD = 2 };

int ko_set_threads(int n);           /* OpenMP thread count, returns the count in effect */
int ko_get_threads(void);

/* Bin points: key = pack(floor((x-o)/h)) as three 21-bit biased fields (cz,cy,cx). x is n x dim. */
int ko_bin(const ko_params* p, const double* x, int64_t n, uint64_t* keys);

/* Build cells, training sets, and fit every cell (Cholesky, alpha). var and normals may be NULL
 * (var NULL means sigma^2 = 0; normals NULL disables the sign stand-in). Copies all inputs. */
int ko_fit(const ko_params* p, const double* x, const double* var, const double* normals, int64_t S,
           ko_model** out);
void ko_free(ko_model* m);

int64_t ko_num_cells(const ko_model* m);
/* keys[G], status[G], ts_off[G+1] (training-set offsets); any pointer may be NULL */
int ko_cells(const ko_model* m, uint64_t* keys, int32_t* status, int64_t* ts_off);
/* training-set member ids, concatenated in cell order (length ts_off[G]) */
int ko_members(const ko_model* m, int64_t* ids);
/* alpha of cell g (length N_g), the Cholesky factor L (N_g x N_g row-major, upper part zero) */
int ko_cell_alpha(const ko_model* m, int64_t g, double* alpha);
int ko_cell_chol(const ko_model* m, int64_t g, double* L);

/* Candidate lists for bins (keys as from ko_bin): out[nb*K] cell ids (-1 padded), count[nb]. */
int ko_candidates(const ko_model* m, const uint64_t* bin_keys, int64_t nb, int32_t* out, int32_t* count);

/* Forward query. xq is Q x dim float32 (promoted to double). sign may be NULL. Outputs (any may be
 * NULL): sdf[Q], grad[Q*dim], var_sdf[Q], var_f[Q], winner[Q], flags[Q], cand_u[Q*K], cand_id[Q*K]. */
int ko_query(const ko_model* m, const float* xq, int64_t Q, const int8_t* sign, double* sdf, double* grad,
             double* var_sdf, double* var_f, int32_t* winner, uint32_t* flags, double* cand_u, int32_t* cand_id);

/* Same outputs, but evaluated with the given cell as the winner for each query (cell[q] >= 0). */
/* SDF-gradient variance (Sec. IV-B.3, App. C) of queries xq (Q x dim float32) on the cells cell[Q] (each an
 * OK cell): var_grad (Q x dim float64).  A query on a training sample gets +inf. */
int ko_var_grad(const ko_model* m, const float* xq, int64_t Q, const int32_t* cell, double* var_grad);

int ko_eval_cell(const ko_model* m, const float* xq, int64_t Q, const int32_t* cell, const int8_t* sign,
                 double* sdf, double* grad, double* var_sdf, double* var_f, uint32_t* flags);

/* Query with double-precision query points (for finite differences of the oracle itself). */
int ko_query_f64(const ko_model* m, const double* xq, int64_t Q, const int8_t* sign, double* sdf, double* grad,
                 double* var_sdf, double* var_f, int32_t* winner, uint32_t* flags);

/* Adjoint of sdf (and of the gradient output if d_grad != NULL) with respect to the query points and
 * the sample positions.  winner may be NULL (recomputed).  d_xq[Q*dim] is overwritten; d_x[S*dim] is
 * accumulated into.  xq is float32 like ko_query; ko_backward_f64 takes double query points. */
int ko_backward(const ko_model* m, const float* xq, int64_t Q, const int8_t* sign, const int32_t* winner,
                const double* d_sdf, const double* d_grad, double* d_xq, double* d_x);
int ko_backward_f64(const ko_model* m, const double* xq, int64_t Q, const int8_t* sign, const int32_t* winner,
                    const double* d_sdf, const double* d_grad, double* d_xq, double* d_x);

#ifdef __cplusplus
}
#endif
#endif
