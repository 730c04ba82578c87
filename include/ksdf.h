/*
 * ksdf.h -- C ABI of the GB300 Kernel-SDF back-end query library (libksdf.so).
 *
 * Kernel-SDF (arXiv 2603.29227) learns the signed distance d(x) = s(x) u(x) of a scene from surface
 * samples {x_i, sigma_i^2}.  Its back-end (Sec. IV-B) fits one log-GP per local region on the samples of
 * an enlarged collection box, with labels f(x_i) = 1 and the RBF kernel k(r) = exp(-lambda r^2)
 * (lambda = 1/(2 l^2), App. I), and answers a query x by min-fusing the K nearest local GPs:
 *
 *   f'(x)   = k'(x)^T (K + Sigma)^{-1} 1,   k'_i = exp(-lambda (|x - x_i|^2 - d^2))    (Sec. IV-B.1, App. D)
 *   u(x)    = min over the K GPs of sqrt(-log f'(x) / lambda + d^2)                    (kernel table, App. D)
 *   grad u  = -grad f' / |grad f'|                                                      (Sec. IV-B.1)
 *   V[u]    = sum_i s_i^2 (a (h - z_i) + 1)^2 sigma_i^2, softmin s, h = s^T z            (Sec. IV-B.3)
 *   V[f]    = 1 - k^T (K + Sigma)^{-1} k = 1 - e^{-2 lambda d^2} |L^{-1} k'|^2           (Sec. IV-B.1)
 *   V[grad_k u] = sum_i |grad_{x_i} g_k|^2 sigma_i^2, g = grad h (optional)          (Sec. IV-B.3, App. C)
 *
 * where d is the distance to the GP's nearest training sample.  The library implements that path on one
 * GPU: integer binning of samples and queries into a hash grid of cells of edge h, training-set
 * assembly, a batched FP64 Cholesky fit, candidate lists of the K nearest cells, the fused query kernels
 * and the adjoint.  Readings taken where the paper is silent are listed with the design notes; the main
 * ones: a "local GP" is a grid cell that holds at least one sample, its collection box is the cell grown
 * by a margin mu on every side (half open), a training set above n_max keeps ranks floor(j cnt / n_max),
 * and "the K nearest GPs" are the K valid cells nearest to the query's cell by squared lattice distance,
 * ties broken by the packed cell key (lexicographic (cz, cy, cx)).
 *
 * Conventions for every call:
 *   - Pointers are plain host or device pointers; the library checks which (cudaPointerGetAttributes).
 *     Device (or managed) arrays are used in place; host arrays are staged through the context's device
 *     workspace inside the call.  When any output array is in host memory the call synchronises the
 *     context's stream before it returns; otherwise every call is asynchronous on that stream.
 *   - Arrays are dense and row-major: points are n x dim (x, y[, z]) interleaved.
 *   - The caller owns every array it passes; the library keeps no pointer to them after the call returns
 *     (ksdf_fit copies what it needs into the model).  The context owns the fitted model and workspaces.
 *   - Errors are returned as ksdf_status; nothing is thrown across the ABI.  ksdf_last_error() gives a
 *     message.  Failures detected on the device (bad query values, capacity overflow, a wait that timed
 *     out) are accumulated in a device status word that ksdf_sync_status() reads and clears.
 *   - One context is used by one host thread at a time.
 */
#ifndef KSDF_H
#define KSDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KSDF_OK = 0,
  KSDF_ERR_ARG = 1,         /* invalid argument (NULL, size, parameter out of range, bad pointer) */
  KSDF_ERR_CUDA = 2,        /* a CUDA runtime call failed; see ksdf_last_error */
  KSDF_ERR_NOT_PD = 3,      /* reported by ksdf_fit when some cell's K + Sigma is not positive definite
                               in FP64 (those cells are excluded from every candidate list; the fit
                               still succeeds for the others) */
  KSDF_ERR_CAPACITY = 4,    /* a size exceeds a documented limit or the reserved capacity */
  KSDF_ERR_NOT_FITTED = 5,  /* query before a successful fit */
  KSDF_ERR_NONFINITE = 6,   /* NaN/Inf or out-of-grid coordinates in the input */
  KSDF_ERR_TIMEOUT = 7      /* a bounded device-side wait gave up (the kernel returned early) */
} ksdf_status;

/* Parameters of the method.  Field meanings follow the paper's notation. */
typedef struct {
  int dim;              /* n in {2, 3} (Sec. III) */
  double origin[3];     /* grid origin o; cell c covers [o + c h, o + (c+1) h) per axis */
  double cell;          /* cell edge h > 0 (one local GP per non-empty cell, Sec. IV-B.1) */
  double margin;        /* collection-box margin mu >= 0, mu < 8 h */
  int n_max;            /* training-set cap per cell, 1..512 */
  int k_cand;           /* K nearest GPs fused by min, 1..32 */
  double lambda;        /* RBF scale lambda = 1/(2 l^2) > 0 (App. I) */
  double softmin_alpha; /* softmin temperature of Sec. IV-B.3; <= 0 means lambda */
  int sign_mode;        /* 0: sign from the caller's array (all +1 when it is NULL);
                           1: when the caller passes no sign array, use a stand-in that is NOT the
                           paper's BHM sign: s = +1 iff n_nn . (x - x_nn) >= 0 for the winner GP's
                           nearest training sample x_nn and its normal n_nn (needs normals at fit) */
  int kernel;           /* KSDF_KERNEL_RBF (0) or KSDF_KERNEL_MATERN32 (1), the kernel table of Sec. IV-B.2 */
} ksdf_params;

/* Kernels (kernel table of Sec. IV-B.2), with `lambda` the scale of f = exp(-lambda u):
 *   KSDF_KERNEL_RBF       k(r) = exp(-lambda r^2) (lambda = 1/(2 l^2)), u = sqrt(-log f'/lambda + d^2);
 *   KSDF_KERNEL_MATERN32  k(r) = (1 + lambda r) exp(-lambda r) (lambda = sqrt(3)/l, the kernel scale sqrt(3)/lambda
 *                         of Sec. IV-B.1), u = -log f'/lambda + d;
 * f' is the posterior mean with the kernel vector scaled by gamma = e^{lambda d^2} or e^{lambda d} (App. D). */
enum { KSDF_KERNEL_RBF = 0, KSDF_KERNEL_MATERN32 = 1 };

/* out_mask bits for ksdf_query / ksdf_query_f64 (outputs whose bit is clear are not written and may be
 * NULL). */
enum {
  KSDF_OUT_SDF = 1u,
  KSDF_OUT_GRAD = 2u,
  KSDF_OUT_VAR_SDF = 4u,
  KSDF_OUT_VAR_F = 8u,
  KSDF_OUT_WINNER = 16u,
  KSDF_OUT_FLAGS = 32u,
  KSDF_OUT_ALL = 63u,     /* the six outputs above */
  KSDF_OUT_VAR_GRAD = 64u /* optional: the SDF-gradient variance (one more pass over the winner's samples) */
};

/* Per-query flag bits. */
enum {
  KSDF_FLAG_FALLBACK = 1u,   /* winner's f' <= 0: u is the distance to its nearest sample */
  KSDF_FLAG_NO_GP = 2u,      /* no valid GP cell exists: sdf = +inf, grad 0, var_sdf 0, var_f 1 */
  KSDF_FLAG_NEAR_TIE = 4u,   /* another candidate's u is within 1e-5 m of the winner's, or (mixed path) may
                                lie below it given the error bounds of the two FP32 evaluations: the binary64
                                path could pick that candidate (overlapping GPs of the same surface often agree
                                to far less than the FP32 error, so the flag is common) */
  KSDF_FLAG_ZERO_GRAD = 8u,  /* grad f' vanished: grad output 0 */
  KSDF_FLAG_CLAMPED = 16u,   /* -log f'/lambda + d^2 < 0 was clamped: u = 0 */
  KSDF_FLAG_INVALID = 32u    /* the query point was NaN/Inf or outside the grid: outputs NaN */
};

/* Cell status values (ksdf_get_cells). */
enum { KSDF_CELL_OK = 0, KSDF_CELL_EMPTY = 1, KSDF_CELL_NOT_PD = 2 };

typedef struct ksdf_ctx ksdf_ctx;

/* Create a context on the current CUDA device; `stream` is a cudaStream_t (NULL = legacy default).
 * Validates the parameters (KSDF_ERR_ARG).  Allocates only small bookkeeping buffers. */
ksdf_status ksdf_create(const ksdf_params* params, void* stream, ksdf_ctx** out);
ksdf_status ksdf_destroy(ksdf_ctx* ctx);
ksdf_status ksdf_set_stream(ksdf_ctx* ctx, void* stream);

/* Pre-size the workspaces for up to max_samples samples and max_queries queries per call, so that
 * later calls within those sizes allocate nothing. */
ksdf_status ksdf_reserve(ksdf_ctx* ctx, int64_t max_samples, int64_t max_queries);

/* Fit (Sec. IV-B.1): bin the S samples x (S x dim, float64) into cells, assemble every cell's training
 * set from its collection box, build A = K + diag(sigma^2) (var: S float32 sigma_i^2 >= 0, NULL = 0) in
 * FP64, factor A = L L^T in FP64 and solve alpha = A^{-1} 1 in FP64 (kept in FP64 and FP32); L is kept in
 * FP64 for the plain query and the adjoint, and L^{-1} is formed in FP32 from L for the mixed query's
 * variance contraction.  normals (S x dim
 * float32, may be NULL) feed the sign stand-in.  Replaces any previous model.  Synchronises the stream
 * (cell counts decide allocation sizes).  Returns KSDF_ERR_NONFINITE for NaN/Inf/out-of-grid samples
 * or a negative variance, KSDF_ERR_CAPACITY if a collection box holds more than 8192 samples before
 * the cap, KSDF_ERR_NOT_PD if some cell failed the factorisation (the model is still usable). */
ksdf_status ksdf_fit(ksdf_ctx* ctx, const double* x, const float* var, const float* normals, int64_t S);

/* Streaming update (Sec. IV-C: new surface samples arrive frame by frame and only the local GPs they touch
 * are retrained): append S_new samples (x_new S_new x dim float64, var_new S_new float32 or NULL = 0,
 * normals_new S_new x dim float32, required exactly when the model has normals) after the model's S
 * samples, which keep their ids, and refit.  The result is the model ksdf_fit would build from all
 * S + S_new samples; cells whose training set (members and their order) is unchanged take their factor,
 * L^{-1} and alpha from the previous model instead of being refitted.  *n_cells_refit (host, may be NULL)
 * receives the number of cells fitted.  With a refit budget (ksdf_set_schedule) the changed cells beyond it are
 * deferred and the model is no longer a fresh fit of all samples until they are fitted.  Synchronises the stream.
 * Errors as ksdf_fit; on an error the context has no model (KSDF_ERR_NOT_FITTED until the next ksdf_fit).
 * KSDF_ERR_NOT_FITTED without a model. */
ksdf_status ksdf_update(ksdf_ctx* ctx, const double* x_new, const float* var_new, const float* normals_new,
                        int64_t S_new, int64_t* n_cells_refit);

/* Streaming update with replacement: the GP training-data buffer update of Sec. IV-C / App. G.  When a region is
 * marched again, its surface points replace the ones it gave before.  drop (S bytes, host or device, S of the
 * current model; non-zero = remove) flags model samples to remove.  The samples that stay keep their order and
 * are renumbered 0..S_kept-1; the S_new new ones follow.  The result is the model ksdf_fit would build from the
 * kept samples followed by the new ones.  A cell whose training set is unchanged, in members and order, under the
 * new numbering takes its fit from the previous model.  A cell that lost a member is always fitted, even under a
 * refit budget.  Arguments, errors and synchronisation as ksdf_update; KSDF_ERR_ARG for a NULL drop or if no
 * sample would remain. */
ksdf_status ksdf_update_replace(ksdf_ctx* ctx, const uint8_t* drop, const double* x_new, const float* var_new,
                                const float* normals_new, int64_t S_new, int64_t* n_cells_refit);

/* Refit scheduling of ksdf_update (the training queue of Sec. IV-C / App. G).  Every cell carries a query counter
 * c0 -- each query that fuses the cell (the cell is one of its bin's K candidates) adds one, capped at 10000 --
 * and training marks c2 -- each update in which the cell's training set changed adds one.  With max_refit > 0 an
 * update fits at most max_refit cells: first every cell that must be fitted (new, or not fitted before), then the
 * changed cells by descending score c2 (1 + eta c0) (FP32, ties in cell order); the other changed cells are
 * deferred and keep the training set, factor and alpha of their last fit.  A fitted cell resets c2 to 0 and halves
 * c0.  With max_refit > 0, ksdf_update with S_new = 0 runs one more round over the deferred cells.  max_refit = 0
 * (the default) fits every changed cell, so that the model equals a fresh fit of all samples.  eta >= 0 (default
 * 1e-3).  KSDF_ERR_ARG for a negative max_refit or a non-finite or negative eta. */
ksdf_status ksdf_set_schedule(ksdf_ctx* ctx, int64_t max_refit, double eta);
/* The scheduling state of the model's G cells (host or device int32 arrays, any may be NULL): c0, c2, and refit
 * (1 if the last ksdf_fit / ksdf_update fitted the cell).  Synchronises the stream.  KSDF_ERR_NOT_FITTED without a
 * model. */
ksdf_status ksdf_get_schedule(ksdf_ctx* ctx, int32_t* c0, int32_t* c2, int32_t* refit);

/* Model serialisation (the serialised map of the paper's scalability experiment, whose size is set by the
 * stored GP surface samples): ksdf_save writes the context's parameters and the S samples the model was
 * fitted or updated from (positions float64, variances and normals float32, host byte order) to the file
 * `path`; ksdf_load reads such a file into a context created with the same parameters and fits it.  The
 * fit is deterministic, so the loaded model equals the saved one bit for bit.  File layout: the 8 bytes
 * "KSDFMAP1", int32 version 1, int32 dim, int32 has_normals, int32 kernel, the 11 parameters (dim, n_max,
 * k_cand, sign_mode as int32; origin[3], cell, margin, lambda, softmin_alpha as float64), int64 S, then
 * x (S x dim), var (S), normals (S x dim, when present).  Synchronises the stream.  Errors:
 * KSDF_ERR_NOT_FITTED (save without a model), KSDF_ERR_ARG (NULL path, a file that cannot be written or
 * read, a bad header, parameters that differ from the context's), and the errors of ksdf_fit (load). */
ksdf_status ksdf_save(ksdf_ctx* ctx, const char* path);
ksdf_status ksdf_load(ksdf_ctx* ctx, const char* path);

/* Autotuning of the batched fit's tile shape (the number of warps that factor one cell, per range of cell
 * sizes): times every candidate size-class table (ksdf_autotune_tables() of them) on the fitted model's own
 * cells -- each a full fit run twice, the second timed with CUDA events on the context's stream -- keeps the
 * fastest for the context's later fits and updates, and refits with it.  The model's numbers do not depend
 * on the table.  *table (may be NULL) receives the chosen index, fit_ms (may be NULL, ksdf_autotune_tables()
 * doubles) the measured fit times.  Synchronises the stream.  KSDF_ERR_NOT_FITTED without a model. */
ksdf_status ksdf_autotune(ksdf_ctx* ctx, int* table, double* fit_ms);
int ksdf_autotune_tables(void);

/* Autotuning of the query's tile shapes on the caller's own batch (Q points xq, Q x dim float32, sign Q int8 or
 * NULL; host or device): phase A's shared-memory budget for the candidates' samples (64, 128 or 256 chunks of 8
 * samples; a tile whose candidates hold more is processed in rounds) and the largest cell of phase B's 128-column
 * tensor-memory class (64, 96 or 128 samples; larger cells up to 256 take 256 columns).  Every pair
 * (ksdf_autotune_query_configs() of them, index = 3 x budget index + class index) runs the full query twice, the
 * second timed with CUDA events on the context's stream; the fastest is kept for the context's later queries.
 * The outputs do not depend on the choice.  *choice (may be NULL) gets the index, query_ms (may be NULL,
 * ksdf_autotune_query_configs() doubles) the times.  Synchronises the stream.  KSDF_ERR_NOT_FITTED without a
 * model, KSDF_ERR_ARG for Q <= 0. */
ksdf_status ksdf_autotune_query(ksdf_ctx* ctx, const float* xq, int64_t Q, const int8_t* sign, int* choice,
                                double* query_ms);
int ksdf_autotune_query_configs(void);

/* Diagnostic of failure detection (no counterpart in the paper): launches, on the context's stream, one CTA
 * that allocates tensor memory like the tensor-core query kernel and then waits on an mbarrier that nothing
 * completes (no copy or MMA is issued, so nothing is in flight), polling it at most `spins` times (1..2^24;
 * KSDF_ERR_ARG otherwise).  The wait gives up the way a production wait does: the device status word gets the
 * timeout bit, the tensor memory is released and the kernel returns, so the next ksdf_sync_status() returns
 * KSDF_ERR_TIMEOUT and the context stays usable.  Asynchronous; returns KSDF_OK once launched. */
ksdf_status ksdf_wait_diagnostic(ksdf_ctx* ctx, uint32_t spins);

/* Diagnostics: the scalar device routines of the fit (Sec. IV-B kernel matrix exp(-lambda r^2) and the
 * Cholesky pivots), evaluated on n inputs x (float64, host or device) into y (float64, host or device) so
 * that tests can hold them to their error bounds.  fn 0: 2^(-x / 2^16) from a binary64 argument; fn 1: the
 * same from the 40-bit fixed-point argument floor(x 2^40) (both 0 <= x < 2^22); fn 2: 1 / sqrt(x) for a
 * normal x > 0.  Inputs outside a routine's domain give NaN.  KSDF_ERR_ARG for an unknown fn or n < 0.
 * Synchronises the stream. */
ksdf_status ksdf_device_math(ksdf_ctx* ctx, int fn, const double* x, int64_t n, double* y);

/* Mixed-precision query: Q points xq (Q x dim float32); sign (Q int8, +1/-1, may be NULL).  FP32 SIMT
 * arithmetic in cell-local coordinates for the mean (compensated sum), gradient and softmin variance; the
 * GP variance contraction K' L^{-T} on the tensor cores in TF32 split three ways (hi*hi + hi*lo + lo*hi,
 * FP32 accumulation) for winner cells of up to 256 samples, in FP32 SIMT beyond.  Outputs (selected by
 * out_mask): sdf[Q], grad[Q x dim] (gradient of d = s grad u), var_sdf[Q] (V[u], Sec. IV-B.3),
 * var_f[Q] (V[f], Sec. IV-B.1), var_grad[Q x dim] (only with KSDF_OUT_VAR_GRAD: V[grad_k u] of Sec. IV-B.3 /
 * App. C, the surface-sample variances propagated through the softmin's gradient on the winner; +inf for a
 * query on a sample, 0 without a GP), winner[Q] (cell id of the fused GP, -1 if none; keep it for the
 * backward), flags[Q] (KSDF_FLAG_*).  Outputs not selected may be NULL. */
ksdf_status ksdf_query(ksdf_ctx* ctx, const float* xq, int64_t Q, const int8_t* sign, uint32_t out_mask, float* sdf,
                       float* grad, float* var_sdf, float* var_f, float* var_grad, int32_t* winner, uint32_t* flags);

/* The same query in FP64 end to end on the GPU (the plain path): xq and the outputs are float64. */
ksdf_status ksdf_query_f64(ksdf_ctx* ctx, const double* xq, int64_t Q, const int8_t* sign, uint32_t out_mask,
                           double* sdf, double* grad, double* var_sdf, double* var_f, double* var_grad,
                           int32_t* winner, uint32_t* flags);

/* Adjoint of the query (the differentiation path): given the cotangents d_sdf[Q] and
 * (optionally, may be NULL) d_grad[Q x dim] of the sdf and grad outputs, write d_xq[Q x dim] (overwritten)
 * and ADD the sample-position gradient into d_x[S x dim] (S of the last fit, ids in the fit's order).
 * winner is the array the forward query returned for the same xq and sign.  Per-cell recomputation:
 * nothing from the forward pass is stored.  The chain through alpha = A^{-1} 1 is taken with one FP64
 * triangular-solve pair per touched cell; sign, sigma^2, the winner choice and the scaling distance are
 * held constant (u does not depend on the scaling). */
ksdf_status ksdf_query_backward(ksdf_ctx* ctx, const float* xq, int64_t Q, const int8_t* sign, const int32_t* winner,
                                const float* d_sdf, const float* d_grad, float* d_xq, float* d_x);

/* Synchronise the stream, read and clear the device status word (KSDF_OK if no device failure). */
ksdf_status ksdf_sync_status(ksdf_ctx* ctx);
const char* ksdf_last_error(const ksdf_ctx* ctx);

/* ---- introspection of the fitted model (host outputs; synchronise the stream) ---- */

/* Number of samples S the model holds (after ksdf_fit, ksdf_update, ksdf_update_replace or ksdf_load); host output,
 * no synchronisation.  KSDF_ERR_NOT_FITTED without a model. */
ksdf_status ksdf_model_samples(ksdf_ctx* ctx, int64_t* S);

/* Number of cells G and of training-set members (sum of N_g). */
ksdf_status ksdf_model_size(ksdf_ctx* ctx, int64_t* n_cells, int64_t* n_members);
/* keys[G] (packed (cz,cy,cx) as three biased 21-bit fields, z most significant), status[G], ts_off[G+1],
 * members[n_members] (global sample ids, ascending within a cell).  Any pointer may be NULL. */
ksdf_status ksdf_get_cells(ksdf_ctx* ctx, uint64_t* keys, int32_t* status, int64_t* ts_off, int64_t* members);
/* alpha (n_members, float64) in training-set order; chol (sum N_g (N_g+1)/2, float64) the Cholesky factor
 * L of each cell as packed lower rows (row i at offset i (i+1)/2), cells in id order; linv (sum 32 nb (nb+1),
 * nb = ceil(N_g / 8), float32) L^{-1} of each cell in 8-row blocks: block R holds, for every column
 * j <= 8R+7, the eight values L^{-1}[8R+r][j], r = 0..7 (zero above the diagonal and past row N_g-1),
 * block R starting at 32 R (R+1).  Any pointer may be NULL. */
ksdf_status ksdf_get_fit(ksdf_ctx* ctx, double* alpha, double* chol, float* linv);
/* Packed keys of points (n x dim float64) and the candidate lists (n x K int32, -1 padded; count[n]) of the
 * cells those keys name.  Device or host arrays. */
ksdf_status ksdf_bin(ksdf_ctx* ctx, const double* x, int64_t n, uint64_t* keys);
ksdf_status ksdf_candidates(ksdf_ctx* ctx, const uint64_t* bin_keys, int64_t n, int32_t* cand, int32_t* count);

/* ---- measurement (no counterpart in the paper: instrumentation of this library) ---- */

/* Enable (1) or disable (0) per-stage timing: CUDA events are recorded on the context's stream around
 * each pipeline stage ("fit.index", "fit.assemble", "fit.cholesky", "query.group", "query.candidates",
 * "query.phaseA", "query.regroup", "query.phaseB", "backward.group", "backward.query", "backward.cell",
 * and the totals "fit", "query", "backward"; the FP64 query uses the prefix "query64").  Synchronises the
 * stream and clears the accumulated totals. */
ksdf_status ksdf_profile(ksdf_ctx* ctx, int enable);
/* Synchronise, fold the recorded events into per-stage totals and copy them out: names is a host buffer of
 * max_stages x 32 chars (NUL-terminated names), total_ms[max_stages] and calls[max_stages] the summed
 * device time and the number of timed calls per stage, *n_stages the number of stages known.  *launches
 * gets the number of kernels this library has launched since it was loaded (all contexts).  Any output
 * pointer may be NULL. */
ksdf_status ksdf_profile_read(ksdf_ctx* ctx, int max_stages, char* names, double* total_ms, int64_t* calls,
                              int* n_stages, int64_t* launches);

/* ---- fit of one local GP without any device allocation (the paper has no counterpart: this serves
 * callers that cannot allocate device memory) ----
 *
 * Who needs it: a real-time loop (a planner or controller that must not enter the CUDA allocator once it
 * runs, because an allocation can block for an unbounded time and may synchronise the device), or a
 * program whose device memory is all owned by another allocator.  Neither can create a context
 * (ksdf_create allocates), so this call takes no context and allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.
 *
 * What it computes: the same FP64 fit as ksdf_fit performs for one cell, within 1e-9 relative (ksdf_fit
 * evaluates kernel entries below 2.4e-16 in FP32 and uses its own exponential, so the two are not bit for bit
 * equal) -- A = K + diag(sigma^2) with K_ij = exp(-lambda |x_i - x_j|^2), A = L L^T, alpha = A^{-1} 1 (all
 * labels 1), and L^{-1} -- with params->dim and params->lambda; params->kernel must be KSDF_KERNEL_RBF (else
 * KSDF_ERR_ARG); the other fields are not used.
 *   x       device, N x dim float64 positions (read)
 *   var     device, N float32 sigma_i^2 >= 0 (read; NULL means 0)
 *   alpha   device, N float64 (written; zeros if A is not positive definite)
 *   linv    device, N (N+1) / 2 float64, L^{-1} as packed lower rows (written; unspecified if not PD)
 *   status  device, one int32: KSDF_CELL_OK, or KSDF_CELL_NOT_PD when a pivot is not finite, positive and
 *           normal, or when an input is NaN/Inf or a variance is negative (written by the kernel)
 *   stream  cudaStream_t the kernel is launched on (NULL = legacy default); the call is asynchronous
 * Every array must be device memory of the current device, or managed memory: host arrays and arrays of
 * another GPU give KSDF_ERR_ARG (copying them would need an allocation).  N must be 1..512: larger N gives
 * KSDF_ERR_CAPACITY.  KSDF_ERR_CUDA if the launch itself fails.
 * Scratch: a static 1,050,624-byte device array (the packed matrix for N = 512), which every GPU that
 * loads the library holds until the process exits.  All calls on a device share it and it keeps the last
 * call's contents (nothing in it needs to start at zero), so calls that overlap on the GPU -- on different
 * streams, or from different host threads, without ordering between them -- race and give wrong results.
 * The first call on each device resolves the array's device address (cudaGetSymbolAddress) and keeps it for
 * the life of the process; make that first call before any stream capture.  A cudaDeviceReset of that device
 * invalidates the kept address: do not use this entry point on a device after resetting it. */
ksdf_status ksdf_fit_gp_noalloc(const ksdf_params* params, const double* x, const float* var, int64_t N,
                                double* alpha, double* linv, int32_t* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif
