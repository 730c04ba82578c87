/*
 * ksdf_bhm.h -- C ABI of the GB300 Kernel-SDF front-end (in libksdf.so): the Bayesian Hilbert map (BHM)
 * occupancy field of Sec. IV-A of arXiv 2603.29227, its sign and threshold, and the surface points it hands to
 * the back-end of ksdf.h.
 *
 * The field is the log-odds l(x) = mu^T phi(x) of a logistic regression on RBF features (Sec. IV-A.1):
 *
 *   phi(x) = [k(x, x~_1), ..., k(x, x~_M), 1],  k(x, x~) = exp(-gamma |x - x~|^2),  features below phi_min dropped
 *
 * with hinge points x~_g = origin + g h on the integer lattice g in Z^3.  The weights w ~ N(mu, Sigma) have a
 * diagonal covariance (independent weights, Sec. IV-A.2) and are updated from each scan by the sequential
 * variational EM of App. A:
 *
 *   E-step  P_t = P_{t-1} + sum_k c(xi_k) phi_k^2,  mu_t = (P_{t-1} mu_{t-1} + sum_k (t_k - 1/2) phi_k) / P_t
 *           (P = diag(Sigma)^{-1}, c(xi) = |(1/2 - sigmoid(xi)) / xi| = tanh(xi/2) / (2 xi), 1/4 at xi = 0,
 *            t_k = 1 for a hit, 0 for a free-space sample)
 *   M-step  xi_k^2 = sum_m phi_km^2 / P_t,m + (mu_t^T phi_k)^2
 *
 * then the threshold tau <- (1 - alpha) tau + (alpha / K) sum_k l(x_k) over the scan's K hits
 * (eq. online_surf_logodds), the sign s(x) = +1 if l(x) < tau else -1 (eq. sign_prediction), and the surface
 * points of the tau level set with sigma_i^2 = beta (tau - l(x_i))^2 / |grad l(x_i)|^2
 * (eq. surface_point_uncertainty).
 *
 * Layout on the GPU (this library's design; it replaces the octree of local BHMs and their weight sync of
 * Sec. IV-A.2).  The lattice is cut into blocks of n_h^3 hinges; block B owns the hinges g with floor(g / n_h) = B
 * and a bias weight (the trailing 1 of phi, used by the points that lie in B).  A block becomes *active* when a
 * hit falls in it; the 26 blocks around an active block are *allocated* too, so every hinge within reach of a
 * sample has a weight.  Blocks live in a device hash table; every hinge weight exists once, so neighbouring
 * regions never disagree and there is nothing to sync.  A new weight starts at the prior N(0, prior_var).
 *
 * Definitions shared by every call (binary64 unless stated, each operation rounded, no contraction):
 *   lattice coordinate   u = (x - origin) / h per axis; |u| must stay below 2^16 (else KSDF_ERR_NONFINITE);
 *   block of a point     floor(floor(u) / n_h);
 *   feature kept         |u - g|^2 <= ln(1 / phi_min) / (gamma h^2) decided in fixed point: each fraction
 *                        u - floor(u) truncated to 2^-20, both sides of the comparison in units of 2^-40;
 *   samples of a ray     sensor p, hit x, L = |x - p|, sigma = free_step / L, u_p and u_x the lattice coordinates
 *                        of p and x, stepped in 2^-32 fixed point: U_p = rint(2^32 u_p), U_x = rint(2^32 u_x),
 *                        D = rint((U_x - U_p) sigma) per axis (round half to even), free samples u_j = (U_p + j D)
 *                        / 2^32 for j = 1 .. floor((L - free_gap) / free_step), kept when their block is active;
 *                        then the hit itself (at u_x);
 *   marching grid        spacing h / march_sub; cell nu = floor(march_sub u); node nu at lattice coordinate
 *                        nu / march_sub; an update marks the cells of its hits and their 26 neighbours; an edge
 *                        (node nu, axis a) joins nu and nu + e_a and is processed when one of its four adjacent
 *                        cells is marked; it gives a point when one node has l >= tau and the other l < tau, at
 *                        the linear interpolation of l along the edge; edge key = (nu_z + 2^19) << 42 |
 *                        (nu_y + 2^19) << 22 | (nu_x + 2^19) << 2 | a.
 * The GPU evaluates features and sums in binary32 and accumulates the EM statistics with binary32 atomics
 * (their order is not fixed), so its weights match a binary64 evaluation to about 1e-6 relative, not bit for
 * bit; the feature and sample sets, the blocks and the marked edges are decided exactly as above.
 *
 * Conventions as in ksdf.h: plain host or device pointers (host arrays are staged), errors as ksdf_status with
 * ksdf_bhm_last_error(), device-detected failures in a status word read by ksdf_bhm_sync_status(), one host
 * thread per context.  3D only.
 */
#ifndef KSDF_BHM_H
#define KSDF_BHM_H

#include <stdint.h>

#include "ksdf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double origin[3];     /* hinge lattice origin: hinge g at origin + g h */
  double hinge_spacing; /* h > 0 */
  int block_hinges;     /* n_h, hinges per block axis, 4..16; the feature window (2 r + 2 hinges per axis,
                           r = floor(sqrt(ln(1/phi_min) / (gamma h^2)))) must satisfy 2 r + 1 <= n_h and r <= 2 */
  double gamma;         /* RBF scale, k = exp(-gamma r^2), gamma = 1 / (2 l^2) (App. I gives l) */
  double phi_min;       /* feature threshold in (0, 1) (1e-3 in App. A) */
  double prior_var;     /* prior variance of a new weight, > 0 (prior mean 0) */
  int em_iters;         /* EM rounds per update, 1..4 (App. A: 1 to 2 suffice) */
  double xi_init;       /* initial variational parameter, >= 0 (App. A suggests 0 or 1) */
  double free_step;     /* spacing of the free-space samples along a ray, > 0 */
  double free_gap;      /* no free sample within this distance of the hit, >= 0 */
  double tau_alpha;     /* learning rate of tau, in (0, 1] */
  double tau_init;      /* initial tau */
  double beta;          /* scale of the surface-point variance, > 0 */
  int march_sub;        /* marching cells per hinge spacing: 1, 2, 4 or 8, with n_h march_sub <= 32 */
  int bias_feature;     /* 1: phi carries the trailing 1, one bias weight per block (Sec. IV-A.1); 0: no bias */
} ksdf_bhm_params;

typedef struct ksdf_bhm ksdf_bhm;

/* Create a map on the current device with room for max_blocks allocated blocks (each holds n_h^3 + 1 weights
 * of 20 bytes) and for max_marked blocks holding marched cells per update (each (n_h march_sub)^3 / 8 bytes;
 * 0 means max_blocks).  KSDF_ERR_ARG for invalid parameters.  stream: cudaStream_t (NULL = legacy default). */
ksdf_status ksdf_bhm_create(const ksdf_bhm_params* params, int64_t max_blocks, int64_t max_marked, void* stream,
                            ksdf_bhm** out);
ksdf_status ksdf_bhm_destroy(ksdf_bhm* m);
ksdf_status ksdf_bhm_set_stream(ksdf_bhm* m, void* stream);

/* One scan (Sec. IV-A.1 to IV-A.4): sensor position p (3 host doubles) and R hits (R x 3 float64, host or device).
 * Activates and allocates blocks, generates the samples, runs em_iters EM rounds, updates tau from the hits and
 * marks the marching cells of the hits.  Runs on the map's stream and synchronises it once, after counting the
 * samples (the count sizes the sample buffer).  Device-detected failures go to the
 * status word: a hit that is NaN/Inf or out of range (KSDF_ERR_NONFINITE; that hit is skipped), more blocks than
 * max_blocks or marked blocks than max_marked (KSDF_ERR_CAPACITY; the blocks beyond are not created or not
 * marched).  R = 0 is allowed (tau is then unchanged).  KSDF_ERR_ARG for a NULL p or R < 0. */
ksdf_status ksdf_bhm_update(ksdf_bhm* m, const double* p, const double* hits, int64_t R);

/* Surface points of the last update's marked cells (Sec. IV-A.4) in ascending edge key: x (cap x 3 float64),
 * var (cap float32 sigma_i^2), normals (cap x 3 float32, n = -grad l / |grad l|, App. B), keys (cap uint64 edge
 * keys); any output may be NULL.  Points where grad l = 0 are not emitted.  *n_out (host) gets the number of
 * points; when it exceeds cap nothing is written and KSDF_ERR_CAPACITY is returned.  Synchronises the stream. */
ksdf_status ksdf_bhm_march(ksdf_bhm* m, int64_t cap, double* x, float* var, float* normals, uint64_t* keys,
                           int64_t* n_out);

/* Which of n edge keys (host or device uint64, as ksdf_bhm_march returns them) the last update's marks process:
 * out[i] = 1 when one of the edge's four adjacent marching cells is marked, else 0 (n bytes, host or device).  A
 * caller that keeps the back-end's surface samples with their edge keys drops the flagged ones and appends the new
 * march (ksdf_update_replace): every processed edge then contributes its current point, or none (the GP buffer
 * update of Sec. IV-C).  Asynchronous unless out is host memory.  KSDF_ERR_ARG for n < 0 or a NULL array. */
ksdf_status ksdf_bhm_edges_marked(ksdf_bhm* m, const uint64_t* keys, int64_t n, uint8_t* out);

/* out_mask bits of ksdf_bhm_query */
enum { KSDF_BHM_LOGODDS = 1u, KSDF_BHM_SIGN = 2u, KSDF_BHM_GRAD = 4u, KSDF_BHM_PROB = 8u };

/* Prediction at Q points xq (Q x 3 float32): logodds[Q] = l(x), sign[Q] (int8, eq. sign_prediction with the
 * current tau), grad[Q x 3] = grad l(x), prob[Q] = sigmoid(l / sqrt(1 + pi/8 phi^T Sigma phi)) (App. B).  A point
 * that is NaN/Inf or out of range gets NaN outputs and sign +1 and sets KSDF_ERR_NONFINITE in the status word.
 * Outputs whose bit is clear may be NULL.  The sign array plugs into ksdf_query as its caller-supplied sign. */
ksdf_status ksdf_bhm_query(ksdf_bhm* m, const float* xq, int64_t Q, uint32_t out_mask, float* logodds, int8_t* sign,
                           float* grad, float* prob);

/* Introspection (host outputs; synchronise the stream).  ksdf_bhm_size: *n_blocks allocated blocks, the number of
 * samples (free + hits) and of kept hinge features (phi_m >= phi_min with an allocated weight, summed over the
 * samples; the bias not counted) of the last update; any pointer may be NULL.  ksdf_bhm_get: keys[n_blocks] the
 * packed block keys (as ksdf.h's cell keys: three biased 21-bit fields, z most significant), active[n_blocks]
 * (0/1), mu and prec[n_blocks x (n_h^3 + 1)] the weights' means and precisions (block slot order; within a block
 * the hinge (lx, ly, lz) at (lz n_h + ly) n_h + lx and the bias last).  Any pointer may be NULL. */
ksdf_status ksdf_bhm_size(ksdf_bhm* m, int64_t* n_blocks, int64_t* n_samples_last, int64_t* n_features_last);
ksdf_status ksdf_bhm_get(ksdf_bhm* m, uint64_t* keys, uint8_t* active, float* mu, float* prec);
ksdf_status ksdf_bhm_tau(ksdf_bhm* m, double* tau);

ksdf_status ksdf_bhm_sync_status(ksdf_bhm* m);
const char* ksdf_bhm_last_error(const ksdf_bhm* m);

#ifdef __cplusplus
}
#endif
#endif
