// ksdf_peaks.cu -- libksdf_peaks.so: throughput probes of the execution units the Kernel-SDF kernels are
// bound by (declared in include/ksdf_peaks.h).  Measurement instrumentation only: nothing of the method is
// computed here and the product library does not link it.  Each probe launches one timed kernel after a
// warm-up launch, CUDA events on the caller's stream, and returns the achieved rate.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>

#include "../../../include/ksdf_peaks.h"

namespace {

char g_err[256] = "";

int fail(cudaError_t e, const char* what) {
  snprintf(g_err, sizeof(g_err), "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  return 2;
}

// FP64: four independent DFMA chains per thread
__global__ void k_dfma(int iters, double* sink) {
  double x0 = 1.0 + 1e-3 * threadIdx.x, x1 = x0 + 0.25, x2 = x0 + 0.5, x3 = x0 + 0.75;
  const double a = 0.999999, b = 1e-7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
  }
  if ((x0 + x1) + (x2 + x3) == 0.0) sink[0] = x0;  // never true; keeps the chains
}

// FP32: eight independent FFMA chains per thread
__global__ void k_ffma(int iters, float* sink) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.f + 1e-3f * threadIdx.x + 0.1f * k;
  const float a = 0.9999f, b = 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 0.f) sink[0] = s;
}

// packed FP32x2: eight independent fma.rn.f32x2 chains per thread (two FMAs per instruction)
__global__ void k_ffma2(int iters, float* sink) {
  unsigned long long x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float lo = 1.f + 1e-3f * threadIdx.x + 0.1f * k, hi = lo + 0.05f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(lo), "f"(hi));
  }
  unsigned long long a, b;
  asm("mov.b64 %0, {%1, %1};" : "=l"(a) : "f"(0.9999f));
  asm("mov.b64 %0, {%1, %1};" : "=l"(b) : "f"(1e-6f));
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(a), "l"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
    s += lo + hi;
  }
  if (s == 0.f) sink[0] = s;
}

// MUFU: eight independent ex2.approx chains per thread, x <- 2^-x (stays in (0.5, 1))
__device__ __forceinline__ float ex2n(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
  return y;
}
__global__ void k_ex2(int iters, float* sink) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 0.5f + 1e-4f * threadIdx.x + 0.01f * k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = ex2n(x[k]);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 0.f) sink[0] = s;
}

// tcgen05 kind::tf32: one CTA per SM; one thread issues back-to-back MMAs M = 128, N = 256, K = 8 on
// zero-filled shared-memory operands (K-major, no swizzle), accumulating in 256 TMEM columns; a commit to an
// mbarrier ends the chain and every wait is bounded (a wait that gives up sets *sink and the kernel returns
// after releasing the TMEM).
constexpr int kMmaM = 128, kMmaN = 256;
constexpr uint32_t kTmemCols = 256;
constexpr unsigned kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__global__ void __launch_bounds__(128) k_tf32(int iters, int* sink) {
  __shared__ __align__(1024) float sA[kMmaM * 8];
  __shared__ __align__(1024) float sB[kMmaN * 8];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x;
  for (int i = tid; i < kMmaM * 8; i += blockDim.x) sA[i] = 0.f;
  for (int i = tid; i < kMmaN * 8; i += blockDim.x) sB[i] = 0.f;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands visible to the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  bool ok = true;
  if (tid == 0) {
    // A: 128 rows x 2 K-quads (16 B per row and quad): quad stride 2048 B, 8-row group stride 128 B
    // B: 256 rows x 2 K-quads: quad stride 4096 B, 8-row group stride 128 B
    const uint64_t da = sdesc(su32(sA), 2048, 128), db = sdesc(su32(sB), 4096, 128);
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kMmaN >> 3) << 17) |
                           ((uint32_t)(kMmaM >> 4) << 24);
    for (int i = 0; i < iters; ++i) {
      const uint32_t acc = i > 0 ? 1u : 0u;
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
          "l"(da), "l"(db), "r"(idesc), "r"(acc)
          : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&bar))
                 : "memory");
    ok = false;
    for (unsigned it = 0; it < kSpinLimit && !ok; ++it) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(su32(&bar))
          : "memory");
      ok = done != 0;
    }
    if (!ok) atomicExch(sink, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <class F>
int time_launch(cudaStream_t st, F&& go, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return fail(e, "cudaEventCreate");
  go();  // warm-up
  cudaEventRecord(e0, st);
  go();
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess ? 0 : fail(e, "probe launch");
}

}  // namespace

extern "C" {

int ksdf_peaks_measure(int unit, void* stream, double* rate) {
  if (!rate) {
    snprintf(g_err, sizeof(g_err), "rate is NULL");
    return 1;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(e, "device query");
  void* sink = nullptr;
  if ((e = cudaMalloc(&sink, 64)) != cudaSuccess) return fail(e, "cudaMalloc");
  cudaMemsetAsync(sink, 0, 64, st);
  float ms = 0.f;
  int rc = 0;
  switch (unit) {
    case KSDF_PEAK_FP64_DFMA: {
      constexpr int kThreads = 512, kIters = 4096;
      rc = time_launch(st, [&] { k_dfma<<<sms, kThreads, 0, st>>>(kIters, (double*)sink); }, &ms);
      if (!rc) *rate = 2.0 * sms * kThreads * (double)kIters * 4 / (ms * 1e-3) / 1e12;
      break;
    }
    case KSDF_PEAK_FP32_FFMA: {
      constexpr int kThreads = 1024, kIters = 8192;
      rc = time_launch(st, [&] { k_ffma<<<2 * sms, kThreads, 0, st>>>(kIters, (float*)sink); }, &ms);
      if (!rc) *rate = 2.0 * sms * kThreads * (double)kIters * 8 / (ms * 1e-3) / 1e12;  // two CTAs per SM
      break;
    }
    case KSDF_PEAK_FP32X2_FFMA: {
      constexpr int kThreads = 1024, kIters = 4096;
      rc = time_launch(st, [&] { k_ffma2<<<2 * sms, kThreads, 0, st>>>(kIters, (float*)sink); }, &ms);
      if (!rc) *rate = 2.0 * sms * kThreads * (double)kIters * 16 / (ms * 1e-3) / 1e12;  // two CTAs per SM
      break;
    }
    case KSDF_PEAK_MUFU_EX2: {
      constexpr int kThreads = 1024, kIters = 2048;
      rc = time_launch(st, [&] { k_ex2<<<2 * sms, kThreads, 0, st>>>(kIters, (float*)sink); }, &ms);
      if (!rc) *rate = 2.0 * sms * kThreads * (double)kIters * 8 / (ms * 1e-3) / 1e12;
      break;
    }
    case KSDF_PEAK_TF32_TCGEN05: {
      constexpr int kIters = 8192;
      rc = time_launch(st, [&] { k_tf32<<<sms, 128, 0, st>>>(kIters, (int*)sink); }, &ms);
      int timed_out = 0;
      if (!rc && (e = cudaMemcpy(&timed_out, sink, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        rc = fail(e, "cudaMemcpy");
      if (!rc && timed_out) {
        snprintf(g_err, sizeof(g_err), "an MMA completion wait gave up");
        rc = 7;
      }
      if (!rc) *rate = 2.0 * kMmaM * kMmaN * 8.0 * kIters * sms / (ms * 1e-3) / 1e12;
      break;
    }
    default:
      snprintf(g_err, sizeof(g_err), "unknown unit %d", unit);
      rc = 1;
  }
  cudaStreamSynchronize(st);
  cudaFree(sink);
  return rc;
}

const char* ksdf_peaks_last_error(void) { return g_err; }

}  // extern "C"
