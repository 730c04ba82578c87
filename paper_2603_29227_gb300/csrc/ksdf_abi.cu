// ksdf_abi.cu -- the extern "C" entry points of libksdf.so (declared and documented in include/ksdf.h):
// argument checks, staging of host arrays through device workspaces, and dispatch to the fit, query and
// backward pipelines.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

#include "ksdf_internal.cuh"

namespace ksdf {

ksdf_status set_err(ksdf_ctx* c, ksdf_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

ksdf_status cuda_err(ksdf_ctx* c, cudaError_t e, const char* what) {
  return set_err(c, KSDF_ERR_CUDA, "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
}

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return cudaSuccess;
  if (b.p) {
    cudaError_t e = cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (e != cudaSuccess) return e;
  }
  size_t n = (bytes + 255) & ~size_t(255);
  cudaError_t e = cudaMalloc(&b.p, n);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return e;
  }
  b.bytes = n;
  return cudaSuccess;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

std::atomic<long long> g_launches{0};

static cudaEvent_t pool_event(ksdf_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

cudaEvent_t prof_begin(ksdf_ctx* c) {
  if (!c->prof) return nullptr;
  cudaEvent_t e = pool_event(c);
  if (e) cudaEventRecord(e, c->stream);
  return e;
}

void prof_end(ksdf_ctx* c, cudaEvent_t a, const char* name) {
  if (!c->prof || !a) return;
  cudaEvent_t b = pool_event(c);
  if (!b) return;
  cudaEventRecord(b, c->stream);
  c->pending.push_back({name, a, b});
}

static void prof_fold(ksdf_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) cudaGetLastError();
    size_t i = 0;
    while (i < c->stage_names.size() && c->stage_names[i] != p.name) ++i;
    if (i == c->stage_names.size()) {
      c->stage_names.push_back(p.name);
      c->stage_ms.push_back(0.0);
      c->stage_calls.push_back(0);
    }
    c->stage_ms[i] += ms;
    c->stage_calls[i] += 1;
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
}

cudaError_t fork_streams(ksdf_ctx* c) {
  cudaError_t e = cudaSuccess;
  if (!c->aux[0]) {
    for (int i = 0; i < ksdf_ctx::kNumAux && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&c->aux[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < ksdf_ctx::kNumAux && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming);
    for (int i = 0; i < ksdf_ctx::kNumAux && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&c->ev_mid[i], cudaEventDisableTiming);
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (int i = 0; i < ksdf_ctx::kNumAux && e == cudaSuccess; ++i)
      e = cudaStreamCreateWithPriority(&c->aux_hi[i], cudaStreamNonBlocking, greatest);
    for (int i = 0; i < ksdf_ctx::kNumAux && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&c->ev_join_hi[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  e = cudaEventRecord(c->ev_fork, c->stream);
  for (int i = 0; i < ksdf_ctx::kNumAux && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(c->aux[i], c->ev_fork, 0);
  for (int i = 0; i < ksdf_ctx::kNumAux && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(c->aux_hi[i], c->ev_fork, 0);
  return e;
}

cudaError_t join_streams(ksdf_ctx* c) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < ksdf_ctx::kNumAux && e == cudaSuccess; ++i) {
    e = cudaEventRecord(c->ev_join[i], c->aux[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join[i], 0);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join_hi[i], c->aux_hi[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join_hi[i], 0);
  }
  return e;
}

namespace {

bool on_device(const void* p) {
  if (!p) return true;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// stage an input array: device pointers pass through, host arrays are copied into stage[slot]
ksdf_status stage_in(ksdf_ctx* c, int slot, const void* p, size_t bytes, const void** out) {
  if (!p || on_device(p)) {
    *out = p;
    return KSDF_OK;
  }
  KSDF_CUDA(c, ensure(c->stage[slot], bytes));
  KSDF_CUDA(c, cudaMemcpyAsync(c->stage[slot].p, p, bytes, cudaMemcpyHostToDevice, c->stream));
  *out = c->stage[slot].p;
  return KSDF_OK;
}

struct OutStage {
  void* host = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
};

ksdf_status stage_out(ksdf_ctx* c, int slot, void* p, size_t bytes, bool copy_in, OutStage* o) {
  o->host = nullptr;
  o->dev = p;
  o->bytes = bytes;
  if (!p || on_device(p)) return KSDF_OK;
  KSDF_CUDA(c, ensure(c->stage[slot], bytes));
  o->host = p;
  o->dev = c->stage[slot].p;
  if (copy_in) KSDF_CUDA(c, cudaMemcpyAsync(o->dev, p, bytes, cudaMemcpyHostToDevice, c->stream));
  return KSDF_OK;
}

ksdf_status finish_out(ksdf_ctx* c, OutStage* o, int n) {
  bool any = false;
  for (int i = 0; i < n; ++i)
    if (o[i].host) {
      KSDF_CUDA(c, cudaMemcpyAsync(o[i].host, o[i].dev, o[i].bytes, cudaMemcpyDeviceToHost, c->stream));
      any = true;
    }
  if (any) KSDF_CUDA(c, cudaStreamSynchronize(c->stream));
  return KSDF_OK;
}

ksdf_status check_params(const ksdf_params* a) {
  if (!a) return KSDF_ERR_ARG;
  if (a->dim != 2 && a->dim != 3) return KSDF_ERR_ARG;
  if (!(a->cell > 0) || !(a->margin >= 0) || !(a->margin < 8 * a->cell)) return KSDF_ERR_ARG;
  if (a->n_max < 1 || a->n_max > kMaxNmax) return KSDF_ERR_ARG;
  if (a->k_cand < 1 || a->k_cand > kMaxK) return KSDF_ERR_ARG;
  if (!(a->lambda > 0) || !(a->lambda < 1e12)) return KSDF_ERR_ARG;
  for (int j = 0; j < 3; ++j)
    if (!(a->origin[j] == a->origin[j]) || a->origin[j] > 1e300 || a->origin[j] < -1e300) return KSDF_ERR_ARG;
  if (a->sign_mode != 0 && a->sign_mode != 1) return KSDF_ERR_ARG;
  if (a->kernel != KSDF_KERNEL_RBF && a->kernel != KSDF_KERNEL_MATERN32) return KSDF_ERR_ARG;
  return KSDF_OK;
}

}  // namespace
}  // namespace ksdf

using namespace ksdf;

extern "C" {

ksdf_status ksdf_create(const ksdf_params* params, void* stream, ksdf_ctx** out) {
  if (!out) return KSDF_ERR_ARG;
  *out = nullptr;
  if (check_params(params) != KSDF_OK) return KSDF_ERR_ARG;
  ksdf_ctx* c = new ksdf_ctx();
  c->abi = *params;
  c->p.dim = params->dim;
  for (int j = 0; j < 3; ++j) c->p.o[j] = j < params->dim ? params->origin[j] : 0.0;
  c->p.h = params->cell;
  {
    int e = 0;
    c->p.rh = std::frexp(params->cell, &e) == 0.5 ? std::ldexp(1.0, 1 - e) : 0.0;  // cell = 2^(e-1)
  }
  c->p.mu = params->margin;
  c->p.n_max = params->n_max;
  c->p.K = params->k_cand;
  c->p.lambda = params->lambda;
  c->p.alpha_s = params->softmin_alpha > 0 ? params->softmin_alpha : params->lambda;
  c->p.sign_mode = params->sign_mode;
  c->p.kernel = params->kernel;
  c->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = ensure(c->status_word, 16);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status_word.p, 0, 16, c->stream);
  if (e != cudaSuccess) {
    delete c;
    return KSDF_ERR_CUDA;
  }
  *out = c;
  return KSDF_OK;
}

static void release_model(Model& m) {
  DevBuf* bufs[] = {&m.key,   &m.status, &m.n,      &m.ts_off, &m.chol_off, &m.linv_off, &m.hkeys,
                    &m.hvals, &m.cell_order, &m.mf4, &m.md4,    &m.mvar,     &m.mnrm,     &m.mgid,
                    &m.mpad,  &m.chol64, &m.linv32,  &m.x,      &m.ltc_off,  &m.ltc,      &m.var_all,
                    &m.nrm_all, &m.bk_off, &m.bk_cells, &m.qc0,     &m.qc2,      &m.refit};
  for (DevBuf* b : bufs) release(*b);
}

ksdf_status ksdf_destroy(ksdf_ctx* c) {
  if (!c) return KSDF_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  release_model(c->m);
  release_model(c->m_prev);
  release(c->status_word);
  for (auto& b : c->ws) release(b);
  for (auto& b : c->stage) release(b);
  for (auto& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  for (int i = 0; i < ksdf_ctx::kNumAux; ++i) {
    if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
    if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
    if (c->ev_mid[i]) cudaEventDestroy(c->ev_mid[i]);
    if (c->aux_hi[i]) cudaStreamDestroy(c->aux_hi[i]);
    if (c->ev_join_hi[i]) cudaEventDestroy(c->ev_join_hi[i]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  delete c;
  return KSDF_OK;
}

ksdf_status ksdf_set_stream(ksdf_ctx* c, void* stream) {
  if (!c) return KSDF_ERR_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  return KSDF_OK;
}

ksdf_status ksdf_reserve(ksdf_ctx* c, int64_t max_samples, int64_t max_queries) {
  if (!c || max_samples < 0 || max_queries < 0) return KSDF_ERR_ARG;
  c->reserved_s = max_samples;
  c->reserved_q = max_queries;
  if (max_queries > 0) return query_reserve(c, max_queries, c->m.G > 0 ? c->m.G : 1);
  return KSDF_OK;
}

namespace ksdf {
namespace {

// replace: keep[i] = 1 for a sample that stays (int64, for the scan that numbers the kept samples)
__global__ void k_keep_flags(const uint8_t* drop, int64_t S, int64_t* keep) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < S) keep[i] = drop[i] ? 0 : 1;
}

// replace: the kept samples, compacted in their order (newid = exclusive scan of keep)
__global__ void k_compact_samples(const int64_t* keep, const int64_t* newid, int64_t S, int dim, const double* x,
                                  const float* var, const float* nrm, double* ux, float* uv, float* un) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S || !keep[i]) return;
  const int64_t j = newid[i];
  for (int a = 0; a < dim; ++a) ux[j * dim + a] = x[i * dim + a];
  uv[j] = var[i];
  if (nrm)
    for (int a = 0; a < dim; ++a) un[j * dim + a] = nrm[i * dim + a];
}

// replace: the current model's training sets in the new sample ids (a warp per cell); a cell that lost a member has
// no usable fit any more (status EMPTY), so the update fits it again and never keeps its old training set
__global__ void k_remap_members(const int64_t* ts_off, int64_t G, const int64_t* keep, const int64_t* newid,
                                int32_t* mgid, int32_t* status) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= G) return;
  bool lost = false;
  for (int64_t i = ts_off[g] + lane; i < ts_off[g + 1]; i += 32) {
    const int32_t id = mgid[i];
    if (keep[id]) {
      mgid[i] = (int32_t)newid[id];
    } else {
      mgid[i] = -1;
      lost = true;
    }
  }
  if (__any_sync(0xffffffffu, lost) && lane == 0) status[g] = KSDF_CELL_EMPTY;
}

ksdf_status update_impl(ksdf_ctx* c, const uint8_t* drop, const double* x_new, const float* var_new,
                        const float* normals_new, int64_t S_new, int64_t* n_cells_refit) {
  if (!c) return KSDF_ERR_ARG;
  if (!c->fitted) return set_err(c, KSDF_ERR_NOT_FITTED, "ksdf_update: no model to update (call ksdf_fit first)");
  if (S_new < 0 || (S_new > 0 && !x_new)) return set_err(c, KSDF_ERR_ARG, "ksdf_update: need x_new for S_new > 0");
  Model& m = c->m;
  if (S_new == 0 && !drop && c->sched_max <= 0) {  // nothing new, and no deferred cells without a budget
    if (n_cells_refit) *n_cells_refit = 0;
    return KSDF_OK;
  }
  if (S_new > 0 && (normals_new != nullptr) != m.has_normals)
    return set_err(c, KSDF_ERR_ARG, "ksdf_update: normals must be given exactly when the model has normals");
  const int dim = c->p.dim;
  const int64_t S_old = m.S;
  cudaStream_t st = c->stream;
  ksdf_status s;
  // the samples that stay: all of them, or those not flagged in `drop`, compacted in their order
  int64_t S0 = S_old;
  const int64_t* keep = nullptr;
  const int64_t* newid = nullptr;
  if (drop) {
    const void* dd;
    if ((s = stage_in(c, 5, drop, (size_t)S_old, &dd))) return s;
    // the keep flags and new ids live in the query's coarse-order workspace: nothing else uses it before the
    // refit below has consumed them
    KSDF_CUDA(c, ensure(c->ws[WS_BORD], sizeof(int64_t) * (2 * S_old + 2)));
    int64_t* kp = ptr<int64_t>(c->ws[WS_BORD]);
    int64_t* ni = kp + S_old;
    int64_t* tot = ni + S_old;
    if (S_old > 0) launch(k_keep_flags, ceil_div(S_old, 256), 256, 0, st, (const uint8_t*)dd, S_old, kp);
    KSDF_CUDA(c, scan_i64(kp, ni, S_old, tot, c->ws[WS_SCAN], st));
    KSDF_CUDA(c, cudaMemcpyAsync(&S0, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    KSDF_CUDA(c, cudaStreamSynchronize(st));
    keep = kp;
    newid = ni;
  }
  const int64_t S = S0 + S_new;
  if (S >= (1LL << 31)) return set_err(c, KSDF_ERR_CAPACITY, "ksdf_update: S must stay below 2^31");
  if (S <= 0) return set_err(c, KSDF_ERR_ARG, "ksdf_update_replace: no sample would remain");
  const void *dx, *dv, *dn;
  if ((s = stage_in(c, 0, x_new, sizeof(double) * S_new * dim, &dx))) return s;
  if ((s = stage_in(c, 1, var_new, sizeof(float) * S_new, &dv))) return s;
  if ((s = stage_in(c, 2, normals_new, sizeof(float) * S_new * dim, &dn))) return s;
  // the union: the model's (kept) samples first, in their order, then the new ones
  KSDF_CUDA(c, ensure(c->ws[WS_UX], sizeof(double) * S * dim));
  KSDF_CUDA(c, ensure(c->ws[WS_UV], sizeof(float) * S));
  double* ux = ptr<double>(c->ws[WS_UX]);
  float* uv = ptr<float>(c->ws[WS_UV]);
  float* un = nullptr;
  if (m.has_normals) {
    KSDF_CUDA(c, ensure(c->ws[WS_UN], sizeof(float) * S * dim));
    un = ptr<float>(c->ws[WS_UN]);
  }
  if (drop) {
    if (S_old > 0)
      launch(k_compact_samples, ceil_div(S_old, 256), 256, 0, st, keep, newid, S_old, dim, ptr<double>(m.x),
             ptr<float>(m.var_all), m.has_normals ? ptr<float>(m.nrm_all) : (const float*)nullptr, ux, uv, un);
    // the current model's training sets in the new ids, before it becomes the previous model
    launch(k_remap_members, ceil_div(m.G * 32, 256), 256, 0, st, ptr<int64_t>(m.ts_off), m.G, keep, newid,
           ptr<int32_t>(m.mgid), ptr<int32_t>(m.status));
  } else {
    KSDF_CUDA(c, cudaMemcpyAsync(ux, m.x.p, sizeof(double) * S0 * dim, cudaMemcpyDeviceToDevice, st));
    KSDF_CUDA(c, cudaMemcpyAsync(uv, m.var_all.p, sizeof(float) * S0, cudaMemcpyDeviceToDevice, st));
    if (m.has_normals)
      KSDF_CUDA(c, cudaMemcpyAsync(un, m.nrm_all.p, sizeof(float) * S0 * dim, cudaMemcpyDeviceToDevice, st));
  }
  if (S_new > 0)
    KSDF_CUDA(c, cudaMemcpyAsync(ux + S0 * dim, dx, sizeof(double) * S_new * dim, cudaMemcpyDeviceToDevice, st));
  if (dv) KSDF_CUDA(c, cudaMemcpyAsync(uv + S0, dv, sizeof(float) * S_new, cudaMemcpyDeviceToDevice, st));
  else if (S_new > 0) KSDF_CUDA(c, cudaMemsetAsync(uv + S0, 0, sizeof(float) * S_new, st));
  if (m.has_normals && S_new > 0)
    KSDF_CUDA(c, cudaMemcpyAsync(un + S0 * dim, dn, sizeof(float) * S_new * dim, cudaMemcpyDeviceToDevice, st));
  // the current model becomes the previous one; the new model reuses the buffers of the one before
  std::swap(c->m, c->m_prev);
  int64_t nref = 0;
  s = fit_model(c, ux, uv, un, S, &c->m_prev, &nref);
  if (n_cells_refit) *n_cells_refit = nref;
  return s;
}

}  // namespace
}  // namespace ksdf

ksdf_status ksdf_update(ksdf_ctx* c, const double* x_new, const float* var_new, const float* normals_new,
                        int64_t S_new, int64_t* n_cells_refit) {
  return ksdf::update_impl(c, nullptr, x_new, var_new, normals_new, S_new, n_cells_refit);
}

ksdf_status ksdf_model_samples(ksdf_ctx* c, int64_t* S) {
  if (!c || !S) return KSDF_ERR_ARG;
  if (!c->fitted) return set_err(c, KSDF_ERR_NOT_FITTED, "ksdf_model_samples: no model");
  *S = c->m.S;
  return KSDF_OK;
}

ksdf_status ksdf_update_replace(ksdf_ctx* c, const uint8_t* drop, const double* x_new, const float* var_new,
                                const float* normals_new, int64_t S_new, int64_t* n_cells_refit) {
  if (c && !drop) return set_err(c, KSDF_ERR_ARG, "ksdf_update_replace: need the drop flags (S bytes)");
  return ksdf::update_impl(c, drop, x_new, var_new, normals_new, S_new, n_cells_refit);
}

ksdf_status ksdf_set_schedule(ksdf_ctx* c, int64_t max_refit, double eta) {
  if (!c) return KSDF_ERR_ARG;
  if (max_refit < 0 || !(eta >= 0) || !(eta < 1e30))
    return set_err(c, KSDF_ERR_ARG, "ksdf_set_schedule: need max_refit >= 0 and a finite eta >= 0");
  c->sched_max = max_refit;
  c->sched_eta = (float)eta;
  return KSDF_OK;
}

ksdf_status ksdf_get_schedule(ksdf_ctx* c, int32_t* c0, int32_t* c2, int32_t* refit) {
  if (!c) return KSDF_ERR_ARG;
  if (!c->fitted) return set_err(c, KSDF_ERR_NOT_FITTED, "ksdf_get_schedule: no model");
  const int64_t G = c->m.G;
  int32_t* outs[3] = {c0, c2, refit};
  DevBuf* srcs[3] = {&c->m.qc0, &c->m.qc2, &c->m.refit};
  for (int k = 0; k < 3; ++k)
    if (outs[k]) KSDF_CUDA(c, cudaMemcpyAsync(outs[k], srcs[k]->p, sizeof(int32_t) * G, cudaMemcpyDefault, c->stream));
  KSDF_CUDA(c, cudaStreamSynchronize(c->stream));
  return KSDF_OK;
}

ksdf_status ksdf_autotune(ksdf_ctx* c, int* table, double* fit_ms) {
  if (!c) return KSDF_ERR_ARG;
  return autotune_fit(c, table, fit_ms);
}

int ksdf_autotune_tables(void) { return fit_table_count(); }

int ksdf_autotune_query_configs(void) { return query_tune_count(); }

ksdf_status ksdf_autotune_query(ksdf_ctx* c, const float* xq, int64_t Q, const int8_t* sign, int* choice,
                                double* query_ms) {
  if (!c) return KSDF_ERR_ARG;
  if (!c->fitted) return set_err(c, KSDF_ERR_NOT_FITTED, "ksdf_autotune_query: no model");
  if (Q <= 0 || !xq) return set_err(c, KSDF_ERR_ARG, "ksdf_autotune_query: need Q > 0 queries");
  const void *dq, *ds;
  ksdf_status s;
  if ((s = stage_in(c, 3, xq, sizeof(float) * Q * c->p.dim, &dq))) return s;
  if ((s = stage_in(c, 4, sign, sizeof(int8_t) * Q, &ds))) return s;
  std::vector<double> ms((size_t)query_tune_count(), 0.0);
  s = autotune_query(c, static_cast<const float*>(dq), Q, static_cast<const int8_t*>(ds), choice, ms.data());
  if (query_ms) std::memcpy(query_ms, ms.data(), sizeof(double) * ms.size());
  return s;
}

namespace {
constexpr char kMapMagic[8] = {'K', 'S', 'D', 'F', 'M', 'A', 'P', '1'};
struct MapParams {  // the parameters in a fixed layout (no padding): 4 int32 then 7 float64
  int32_t dim, n_max, k_cand, sign_mode;
  double origin[3], cell, margin, lambda, softmin_alpha;
};
MapParams map_params(const ksdf_params& a) {
  MapParams m;
  m.dim = a.dim;
  m.n_max = a.n_max;
  m.k_cand = a.k_cand;
  m.sign_mode = a.sign_mode;
  for (int j = 0; j < 3; ++j) m.origin[j] = a.origin[j];
  m.cell = a.cell;
  m.margin = a.margin;
  m.lambda = a.lambda;
  m.softmin_alpha = a.softmin_alpha;
  return m;
}
static_assert(sizeof(MapParams) == 4 * 4 + 7 * 8, "the map header's parameter block has no padding");
bool same_params(const MapParams& x, const MapParams& y) {
  bool eq = x.dim == y.dim && x.n_max == y.n_max && x.k_cand == y.k_cand && x.sign_mode == y.sign_mode &&
            x.cell == y.cell && x.margin == y.margin && x.lambda == y.lambda && x.softmin_alpha == y.softmin_alpha;
  for (int j = 0; j < 3; ++j) eq = eq && x.origin[j] == y.origin[j];
  return eq;
}
}  // namespace

ksdf_status ksdf_save(ksdf_ctx* c, const char* path) {
  if (!c || !path) return KSDF_ERR_ARG;
  if (!c->fitted) return set_err(c, KSDF_ERR_NOT_FITTED, "ksdf_save: no model");
  const Model& m = c->m;
  const int dim = c->p.dim;
  const int64_t S = m.S;
  std::vector<double> hx((size_t)S * dim);
  std::vector<float> hv((size_t)S), hn(m.has_normals ? (size_t)S * dim : 0);
  KSDF_CUDA(c, cudaMemcpyAsync(hx.data(), m.x.p, sizeof(double) * hx.size(), cudaMemcpyDeviceToHost, c->stream));
  KSDF_CUDA(c, cudaMemcpyAsync(hv.data(), m.var_all.p, sizeof(float) * hv.size(), cudaMemcpyDeviceToHost, c->stream));
  if (m.has_normals)
    KSDF_CUDA(c, cudaMemcpyAsync(hn.data(), m.nrm_all.p, sizeof(float) * hn.size(), cudaMemcpyDeviceToHost, c->stream));
  KSDF_CUDA(c, cudaStreamSynchronize(c->stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) return set_err(c, KSDF_ERR_ARG, "ksdf_save: cannot open %s for writing", path);
  const int32_t head[4] = {1, dim, m.has_normals ? 1 : 0, c->abi.kernel};
  const MapParams mp = map_params(c->abi);
  bool ok = std::fwrite(kMapMagic, 1, 8, f) == 8 && std::fwrite(head, sizeof(head), 1, f) == 1 &&
            std::fwrite(&mp, sizeof(mp), 1, f) == 1 && std::fwrite(&S, sizeof(S), 1, f) == 1 &&
            std::fwrite(hx.data(), sizeof(double), hx.size(), f) == hx.size() &&
            std::fwrite(hv.data(), sizeof(float), hv.size(), f) == hv.size() &&
            std::fwrite(hn.data(), sizeof(float), hn.size(), f) == hn.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return set_err(c, KSDF_ERR_ARG, "ksdf_save: write to %s failed", path);
  return KSDF_OK;
}

ksdf_status ksdf_load(ksdf_ctx* c, const char* path) {
  if (!c || !path) return KSDF_ERR_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_err(c, KSDF_ERR_ARG, "ksdf_load: cannot open %s", path);
  char magic[8];
  int32_t head[4];
  MapParams mp;
  int64_t S = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMapMagic, 8) == 0 &&
            std::fread(head, sizeof(head), 1, f) == 1 && head[0] == 1 && std::fread(&mp, sizeof(mp), 1, f) == 1 &&
            std::fread(&S, sizeof(S), 1, f) == 1;
  const int dim = c->p.dim;
  ok = ok && head[1] == dim && (head[2] == 0 || head[2] == 1) && head[3] == c->abi.kernel && S > 0 &&
       S < (1LL << 31) && same_params(mp, map_params(c->abi));
  std::vector<double> hx;
  std::vector<float> hv, hn;
  if (ok) {
    hx.resize((size_t)S * dim);
    hv.resize((size_t)S);
    hn.resize(head[2] ? (size_t)S * dim : 0);
    ok = std::fread(hx.data(), sizeof(double), hx.size(), f) == hx.size() &&
         std::fread(hv.data(), sizeof(float), hv.size(), f) == hv.size() &&
         std::fread(hn.data(), sizeof(float), hn.size(), f) == hn.size();
  }
  std::fclose(f);
  if (!ok) return set_err(c, KSDF_ERR_ARG, "ksdf_load: %s is not a map of this context's parameters", path);
  return ksdf_fit(c, hx.data(), hv.data(), head[2] ? hn.data() : nullptr, S);
}

ksdf_status ksdf_wait_diagnostic(ksdf_ctx* c, uint32_t spins) {
  if (!c) return KSDF_ERR_ARG;
  if (spins == 0 || spins > (1u << 24)) return set_err(c, KSDF_ERR_ARG, "ksdf_wait_diagnostic: spins must be 1..2^24");
  return wait_diagnostic(c, spins);
}

ksdf_status ksdf_device_math(ksdf_ctx* c, int fn, const double* x, int64_t n, double* y) {
  if (!c || fn < 0 || fn > 2 || n < 0 || (n > 0 && (!x || !y))) return KSDF_ERR_ARG;
  if (n == 0) return KSDF_OK;
  const void* dx;
  ksdf_status s;
  if ((s = stage_in(c, 0, x, sizeof(double) * n, &dx))) return s;
  OutStage o;
  if ((s = stage_out(c, 1, y, sizeof(double) * n, false, &o))) return s;
  if ((s = device_math(c, fn, static_cast<const double*>(dx), n, static_cast<double*>(o.dev)))) return s;
  if ((s = finish_out(c, &o, 1))) return s;
  KSDF_CUDA(c, cudaStreamSynchronize(c->stream));
  return KSDF_OK;
}

ksdf_status ksdf_fit(ksdf_ctx* c, const double* x, const float* var, const float* normals, int64_t S) {
  if (!c) return KSDF_ERR_ARG;
  if (S <= 0 || !x) return set_err(c, KSDF_ERR_ARG, "ksdf_fit: need S > 0 samples");
  const int dim = c->p.dim;
  const void *dx, *dv, *dn;
  ksdf_status s;
  if ((s = stage_in(c, 0, x, sizeof(double) * S * dim, &dx))) return s;
  if ((s = stage_in(c, 1, var, sizeof(float) * S, &dv))) return s;
  if ((s = stage_in(c, 2, normals, sizeof(float) * S * dim, &dn))) return s;
  return fit_model(c, static_cast<const double*>(dx), static_cast<const float*>(dv), static_cast<const float*>(dn), S);
}

static ksdf_status query_common(ksdf_ctx* c, const void* xq, bool f64, int64_t Q, const int8_t* sign,
                                uint32_t mask, void* sdf, void* grad, void* var_sdf, void* var_f, void* var_grad,
                                int32_t* winner, uint32_t* flags) {
  if (!c) return KSDF_ERR_ARG;
  if (!c->fitted) return set_err(c, KSDF_ERR_NOT_FITTED, "query before a successful fit");
  if (Q < 0 || (Q > 0 && !xq)) return set_err(c, KSDF_ERR_ARG, "query: bad Q or NULL points");
  if (Q >= (1LL << 31)) return set_err(c, KSDF_ERR_CAPACITY, "query: Q must be < 2^31");
  if (Q == 0) return KSDF_OK;  // empty arrays may carry NULL pointers
  mask &= KSDF_OUT_ALL | KSDF_OUT_VAR_GRAD;
  if (((mask & KSDF_OUT_SDF) && !sdf) || ((mask & KSDF_OUT_GRAD) && !grad) || ((mask & KSDF_OUT_VAR_SDF) && !var_sdf) ||
      ((mask & KSDF_OUT_VAR_F) && !var_f) || ((mask & KSDF_OUT_WINNER) && !winner) ||
      ((mask & KSDF_OUT_FLAGS) && !flags) || ((mask & KSDF_OUT_VAR_GRAD) && !var_grad))
    return set_err(c, KSDF_ERR_ARG, "query: an output selected by out_mask is NULL");
  if (Q == 0) return KSDF_OK;
  const int dim = c->p.dim;
  const size_t fs = f64 ? sizeof(double) : sizeof(float);
  const void *dxq, *dsg;
  ksdf_status s;
  if ((s = stage_in(c, 0, xq, fs * Q * dim, &dxq))) return s;
  if ((s = stage_in(c, 1, sign, sizeof(int8_t) * Q, &dsg))) return s;
  OutStage o[7];
  if ((s = stage_out(c, 2, (mask & KSDF_OUT_SDF) ? sdf : nullptr, fs * Q, false, &o[0]))) return s;
  if ((s = stage_out(c, 3, (mask & KSDF_OUT_GRAD) ? grad : nullptr, fs * Q * dim, false, &o[1]))) return s;
  if ((s = stage_out(c, 4, (mask & KSDF_OUT_VAR_SDF) ? var_sdf : nullptr, fs * Q, false, &o[2]))) return s;
  if ((s = stage_out(c, 5, (mask & KSDF_OUT_VAR_F) ? var_f : nullptr, fs * Q, false, &o[3]))) return s;
  if ((s = stage_out(c, 6, (mask & KSDF_OUT_WINNER) ? winner : nullptr, sizeof(int32_t) * Q, false, &o[4]))) return s;
  if ((s = stage_out(c, 7, (mask & KSDF_OUT_FLAGS) ? flags : nullptr, sizeof(uint32_t) * Q, false, &o[5]))) return s;
  if ((s = stage_out(c, 8, (mask & KSDF_OUT_VAR_GRAD) ? var_grad : nullptr, fs * Q * dim, false, &o[6]))) return s;
  s = run_query(c, dxq, f64, Q, static_cast<const int8_t*>(dsg), mask, o[0].dev, o[1].dev, o[2].dev, o[3].dev,
                o[6].dev, static_cast<int32_t*>(o[4].dev), static_cast<uint32_t*>(o[5].dev));
  if (s) return s;
  return finish_out(c, o, 7);
}

ksdf_status ksdf_query(ksdf_ctx* c, const float* xq, int64_t Q, const int8_t* sign, uint32_t out_mask, float* sdf,
                       float* grad, float* var_sdf, float* var_f, float* var_grad, int32_t* winner, uint32_t* flags) {
  return query_common(c, xq, false, Q, sign, out_mask, sdf, grad, var_sdf, var_f, var_grad, winner, flags);
}

ksdf_status ksdf_query_f64(ksdf_ctx* c, const double* xq, int64_t Q, const int8_t* sign, uint32_t out_mask,
                           double* sdf, double* grad, double* var_sdf, double* var_f, double* var_grad,
                           int32_t* winner, uint32_t* flags) {
  return query_common(c, xq, true, Q, sign, out_mask, sdf, grad, var_sdf, var_f, var_grad, winner, flags);
}

ksdf_status ksdf_query_backward(ksdf_ctx* c, const float* xq, int64_t Q, const int8_t* sign, const int32_t* winner,
                                const float* d_sdf, const float* d_grad, float* d_xq, float* d_x) {
  if (!c) return KSDF_ERR_ARG;
  if (!c->fitted) return set_err(c, KSDF_ERR_NOT_FITTED, "backward before a successful fit");
  if (Q < 0 || (Q > 0 && (!xq || !winner || !d_sdf || !d_xq || !d_x)))
    return set_err(c, KSDF_ERR_ARG, "ksdf_query_backward: NULL argument");
  if (Q == 0) return KSDF_OK;
  const int dim = c->p.dim;
  const int64_t S = c->m.S;
  const void *dxq, *dsg, *dw, *dds, *ddg;
  ksdf_status s;
  if ((s = stage_in(c, 0, xq, sizeof(float) * Q * dim, &dxq))) return s;
  if ((s = stage_in(c, 1, sign, Q, &dsg))) return s;
  if ((s = stage_in(c, 2, winner, sizeof(int32_t) * Q, &dw))) return s;
  if ((s = stage_in(c, 3, d_sdf, sizeof(float) * Q, &dds))) return s;
  if ((s = stage_in(c, 4, d_grad, sizeof(float) * Q * dim, &ddg))) return s;
  OutStage o[2];
  if ((s = stage_out(c, 5, d_xq, sizeof(float) * Q * dim, false, &o[0]))) return s;
  if ((s = stage_out(c, 6, d_x, sizeof(float) * S * dim, true, &o[1]))) return s;
  s = run_backward(c, static_cast<const float*>(dxq), Q, static_cast<const int8_t*>(dsg),
                   static_cast<const int32_t*>(dw), static_cast<const float*>(dds), static_cast<const float*>(ddg),
                   static_cast<float*>(o[0].dev), static_cast<float*>(o[1].dev));
  if (s) return s;
  return finish_out(c, o, 2);
}

ksdf_status ksdf_sync_status(ksdf_ctx* c) {
  if (!c) return KSDF_ERR_ARG;
  uint32_t w = 0;
  KSDF_CUDA(c, cudaMemcpyAsync(&w, c->status_word.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
  KSDF_CUDA(c, cudaStreamSynchronize(c->stream));
  KSDF_CUDA(c, cudaMemsetAsync(c->status_word.p, 0, sizeof(uint32_t), c->stream));
  if (w & ST_TIMEOUT) return set_err(c, KSDF_ERR_TIMEOUT, "a bounded device wait gave up");
  if (w & ST_CAPACITY) return set_err(c, KSDF_ERR_CAPACITY, "a device-side capacity was exceeded");
  if (w & ST_NONFINITE) return set_err(c, KSDF_ERR_NONFINITE, "NaN/Inf or out-of-grid query point(s)");
  return KSDF_OK;
}

const char* ksdf_last_error(const ksdf_ctx* c) { return c ? c->err.c_str() : "null context"; }

ksdf_status ksdf_profile(ksdf_ctx* c, int enable) {
  if (!c) return KSDF_ERR_ARG;
  KSDF_CUDA(c, cudaStreamSynchronize(c->stream));
  prof_fold(c);
  c->stage_names.clear();
  c->stage_ms.clear();
  c->stage_calls.clear();
  c->prof = enable != 0;
  return KSDF_OK;
}

ksdf_status ksdf_profile_read(ksdf_ctx* c, int max_stages, char* names, double* total_ms, int64_t* calls,
                              int* n_stages, int64_t* launches) {
  if (!c || max_stages < 0) return KSDF_ERR_ARG;
  KSDF_CUDA(c, cudaStreamSynchronize(c->stream));
  prof_fold(c);
  const int n = (int)c->stage_names.size();
  if (n_stages) *n_stages = n;
  for (int i = 0; i < n && i < max_stages; ++i) {
    if (names) {
      std::memset(names + 32 * i, 0, 32);
      std::strncpy(names + 32 * i, c->stage_names[i].c_str(), 31);
    }
    if (total_ms) total_ms[i] = c->stage_ms[i];
    if (calls) calls[i] = c->stage_calls[i];
  }
  if (launches) *launches = g_launches.load();
  return KSDF_OK;
}

ksdf_status ksdf_model_size(ksdf_ctx* c, int64_t* n_cells, int64_t* n_members) {
  if (!c) return KSDF_ERR_ARG;
  if (!c->fitted) return KSDF_ERR_NOT_FITTED;
  KSDF_CUDA(c, cudaStreamSynchronize(c->stream));
  if (n_cells) *n_cells = c->m.G;
  if (n_members) *n_members = c->m.M;
  return KSDF_OK;
}

ksdf_status ksdf_get_cells(ksdf_ctx* c, uint64_t* keys, int32_t* status, int64_t* ts_off, int64_t* members) {
  if (!c) return KSDF_ERR_ARG;
  if (!c->fitted) return KSDF_ERR_NOT_FITTED;
  Model& m = c->m;
  KSDF_CUDA(c, cudaStreamSynchronize(c->stream));
  if (keys) KSDF_CUDA(c, cudaMemcpy(keys, m.key.p, sizeof(uint64_t) * m.G, cudaMemcpyDefault));
  if (status) KSDF_CUDA(c, cudaMemcpy(status, m.status.p, sizeof(int32_t) * m.G, cudaMemcpyDefault));
  if (ts_off) KSDF_CUDA(c, cudaMemcpy(ts_off, m.ts_off.p, sizeof(int64_t) * (m.G + 1), cudaMemcpyDefault));
  if (members) {
    std::vector<int32_t> tmp((size_t)m.M);
    if (m.M) KSDF_CUDA(c, cudaMemcpy(tmp.data(), m.mgid.p, sizeof(int32_t) * m.M, cudaMemcpyDeviceToHost));
    std::vector<int64_t> t64(tmp.begin(), tmp.end());
    if (m.M) KSDF_CUDA(c, cudaMemcpy(members, t64.data(), sizeof(int64_t) * m.M, cudaMemcpyDefault));
  }
  return KSDF_OK;
}

ksdf_status ksdf_get_fit(ksdf_ctx* c, double* alpha, double* chol, float* linv) {
  if (!c) return KSDF_ERR_ARG;
  if (!c->fitted) return KSDF_ERR_NOT_FITTED;
  Model& m = c->m;
  KSDF_CUDA(c, cudaStreamSynchronize(c->stream));
  if (alpha && m.M) {
    std::vector<D4> tmp((size_t)m.M);
    KSDF_CUDA(c, cudaMemcpy(tmp.data(), m.md4.p, sizeof(D4) * m.M, cudaMemcpyDeviceToHost));
    std::vector<double> a((size_t)m.M);
    for (int64_t i = 0; i < m.M; ++i) a[i] = tmp[i].w;
    KSDF_CUDA(c, cudaMemcpy(alpha, a.data(), sizeof(double) * m.M, cudaMemcpyDefault));
  }
  if (chol && m.chol_total)
    KSDF_CUDA(c, cudaMemcpy(chol, m.chol64.p, sizeof(double) * m.chol_total, cudaMemcpyDefault));
  if (linv && m.linv_total)
    KSDF_CUDA(c, cudaMemcpy(linv, m.linv32.p, sizeof(float) * m.linv_total, cudaMemcpyDefault));
  return KSDF_OK;
}

ksdf_status ksdf_bin(ksdf_ctx* c, const double* x, int64_t n, uint64_t* keys) {
  if (!c || n < 0 || (n > 0 && (!x || !keys))) return KSDF_ERR_ARG;
  if (n == 0) return KSDF_OK;
  const void* dx;
  ksdf_status s;
  if ((s = stage_in(c, 0, x, sizeof(double) * n * c->p.dim, &dx))) return s;
  OutStage o;
  if ((s = stage_out(c, 1, keys, sizeof(uint64_t) * n, false, &o))) return s;
  if ((s = bin_points(c, static_cast<const double*>(dx), n, static_cast<uint64_t*>(o.dev)))) return s;
  return finish_out(c, &o, 1);
}

ksdf_status ksdf_candidates(ksdf_ctx* c, const uint64_t* bin_keys, int64_t n, int32_t* cand, int32_t* count) {
  if (!c || n < 0 || (n > 0 && (!bin_keys || !cand || !count))) return KSDF_ERR_ARG;
  if (!c->fitted) return KSDF_ERR_NOT_FITTED;
  if (n == 0) return KSDF_OK;
  const void* dk;
  ksdf_status s;
  if ((s = stage_in(c, 0, bin_keys, sizeof(uint64_t) * n, &dk))) return s;
  OutStage o[2];
  if ((s = stage_out(c, 1, cand, sizeof(int32_t) * n * c->p.K, false, &o[0]))) return s;
  if ((s = stage_out(c, 2, count, sizeof(int32_t) * n, false, &o[1]))) return s;
  if ((s = candidates_for_keys(c, static_cast<const uint64_t*>(dk), n, static_cast<int32_t*>(o[0].dev),
                               static_cast<int32_t*>(o[1].dev))))
    return s;
  return finish_out(c, o, 2);
}

}  // extern "C"
