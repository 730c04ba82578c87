// ksdf_noalloc.cu -- the fit of one local GP with no device allocation (ksdf_fit_gp_noalloc in ksdf.h).
//
// Some callers cannot call cudaMalloc: a real-time loop (a planner or controller that must not enter the
// CUDA allocator once it runs, because an allocation can block for an unbounded time and may synchronise
// the device), or a program whose device memory is entirely owned by another allocator, where a
// cudaMalloc outside that pool would fail or fragment it.  This entry point lets them fit one training
// set: they pass device arrays for the inputs and outputs, and the only scratch (the packed N x N kernel
// matrix and its Cholesky factor) lives in the file-scope array below.
#include <mutex>

#include "ksdf_internal.cuh"

namespace ksdf {
namespace {

constexpr int kNoAllocMaxN = 512;
constexpr int64_t kNoAllocTri = (int64_t)kNoAllocMaxN * (kNoAllocMaxN + 1) / 2;  // 131,328 doubles, 1,050,624 B

// Packed lower triangle of A = K + diag(sigma^2), overwritten by L.  Every GPU that loads the library holds
// this array until the process exits, and every call on that GPU shares it.  Nothing in it has to start at
// zero: each call writes every entry before it reads it.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocTri];

// Device address of g_noalloc_scratch per device, resolved on the first call on that device.  In host code
// the symbol itself is only a host-side stand-in, so it is never passed to a kernel.
constexpr int kMaxDevices = 256;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

__device__ inline int64_t tri_na(int i) { return (int64_t)i * (i + 1) / 2; }

// a usable Cholesky pivot: finite, positive and normal (the regular fit's rule)
__device__ inline bool pivot_usable(double d) {
  const long long b = __double_as_longlong(d);
  const int ex = (int)((b >> 52) & 0x7ff);
  return b > 0 && ex > 0 && ex < 2047;
}

// One CTA fits one training set: A, right-looking Cholesky in the scratch, alpha = A^{-1} 1 by two
// triangular solves, and L^{-1} (packed rows) written straight into the caller's output.
__global__ void __launch_bounds__(256) k_fit_gp_noalloc(const double* x, const float* var, int N, int dim,
                                                        double lambda, double* A, double* alpha, double* linv,
                                                        int32_t* status) {
  extern __shared__ double sm[];  // [3 N] coordinates, [N] right-hand side
  __shared__ int s_fail;
  double* sx = sm;
  double* sb = sm + 3 * N;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  // inputs: finite coordinates, finite non-negative variances (else the cell is reported not PD untouched)
  for (int i = tid; i < N; i += nthr) {
    bool ok = true;
    for (int j = 0; j < 3; ++j) {
      const double v = j < dim ? x[(int64_t)i * dim + j] : 0.0;
      ok &= isfinite(v);
      sx[3 * i + j] = v;
    }
    if (var) ok &= isfinite(var[i]) && var[i] >= 0.f;
    if (!ok) s_fail = 1;
  }
  __syncthreads();
  if (s_fail) {
    for (int i = tid; i < N; i += nthr) alpha[i] = 0.0;
    if (tid == 0) *status = KSDF_CELL_NOT_PD;
    return;
  }
  for (int i = warp; i < N; i += nwarp)
    for (int j = lane; j <= i; j += 32) {
      double dx = sx[3 * i] - sx[3 * j], dy = sx[3 * i + 1] - sx[3 * j + 1], dz = sx[3 * i + 2] - sx[3 * j + 2];
      double a = exp(-lambda * (dx * dx + dy * dy + dz * dz));
      if (i == j && var) a += (double)var[i];
      A[tri_na(i) + j] = a;
    }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (tid == 0) {
      double piv = A[tri_na(k) + k];
      if (!pivot_usable(piv)) s_fail = 1;
      else A[tri_na(k) + k] = sqrt(piv);
    }
    __syncthreads();
    if (s_fail) break;
    const double dkk = A[tri_na(k) + k];
    for (int i = k + 1 + tid; i < N; i += nthr) A[tri_na(i) + k] = A[tri_na(i) + k] / dkk;
    __syncthreads();
    for (int i = k + 1 + warp; i < N; i += nwarp) {
      const double lik = A[tri_na(i) + k];
      for (int j = k + 1 + lane; j <= i; j += 32) A[tri_na(i) + j] = fma(-lik, A[tri_na(j) + k], A[tri_na(i) + j]);
    }
    __syncthreads();
  }
  if (s_fail) {
    for (int i = tid; i < N; i += nthr) alpha[i] = 0.0;
    if (tid == 0) *status = KSDF_CELL_NOT_PD;
    return;
  }
  for (int i = tid; i < N; i += nthr) sb[i] = 1.0;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (tid == 0) sb[k] = sb[k] / A[tri_na(k) + k];
    __syncthreads();
    const double bk = sb[k];
    for (int i = k + 1 + tid; i < N; i += nthr) sb[i] = fma(-A[tri_na(i) + k], bk, sb[i]);
    __syncthreads();
  }
  for (int k = N - 1; k >= 0; --k) {
    if (tid == 0) sb[k] = sb[k] / A[tri_na(k) + k];
    __syncthreads();
    const double bk = sb[k];
    for (int i = tid; i < k; i += nthr) sb[i] = fma(-A[tri_na(k) + i], bk, sb[i]);
    __syncthreads();
  }
  for (int i = tid; i < N; i += nthr) alpha[i] = sb[i];
  double* X = linv;
  for (int i = warp; i < N; i += nwarp)
    for (int j = lane; j <= i; j += 32) X[tri_na(i) + j] = (i == j) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    const double dkk = A[tri_na(k) + k];
    for (int j = tid; j <= k; j += nthr) X[tri_na(k) + j] = X[tri_na(k) + j] / dkk;
    __syncthreads();
    for (int i = k + 1 + warp; i < N; i += nwarp) {
      const double lik = A[tri_na(i) + k];
      for (int j = lane; j <= k; j += 32) X[tri_na(i) + j] = fma(-lik, X[tri_na(k) + j], X[tri_na(i) + j]);
    }
    __syncthreads();
  }
  if (tid == 0) *status = KSDF_CELL_OK;
}

// memory the kernel may use on device `dev`: device memory of that device, or managed memory
bool usable_on(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // the failed query's own error, raised just above
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace
}  // namespace ksdf

extern "C" ksdf_status ksdf_fit_gp_noalloc(const ksdf_params* params, const double* x, const float* var, int64_t N,
                                           double* alpha, double* linv, int32_t* status, void* stream) {
  using namespace ksdf;
  if (!params || !x || !alpha || !linv || !status) return KSDF_ERR_ARG;
  if ((params->dim != 2 && params->dim != 3) || !(params->lambda > 0) || !(params->lambda < 1e12) ||
      params->kernel != KSDF_KERNEL_RBF)
    return KSDF_ERR_ARG;
  if (N < 1 || N > kNoAllocMaxN) return KSDF_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KSDF_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return KSDF_ERR_CAPACITY;
  // arrays of the current device (or managed) only: staging host arrays, or arrays of another GPU, would need
  // an allocation or peer access
  if (!usable_on(x, dev) || (var && !usable_on(var, dev)) || !usable_on(alpha, dev) || !usable_on(linv, dev) ||
      !usable_on(status, dev))
    return KSDF_ERR_ARG;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return KSDF_ERR_CUDA;
      }
      g_scratch_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  const size_t smem = sizeof(double) * 4 * (size_t)N;
  // launched through cudaLaunchKernel so that the status is this launch's own (an earlier, unrelated
  // asynchronous error is neither reported as this call's nor cleared)
  int n32 = (int)N, dim = params->dim;
  double lambda = params->lambda;
  void* args[] = {(void*)&x, (void*)&var, &n32, &dim, &lambda, &scratch, &alpha, &linv, &status};
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (cudaLaunchKernel((const void*)k_fit_gp_noalloc, dim3(1), dim3(256), args, smem,
                       static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return KSDF_ERR_CUDA;
  return KSDF_OK;
}
