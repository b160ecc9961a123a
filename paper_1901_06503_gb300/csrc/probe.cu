// probe.cu -- arithmetic throughput probe: the fused multiply-add rate of the
// GPU's FP64, FP32 and packed two-lane FP32 pipes, measured with CUDA events.
//
// Not part of the method: the stencil kernels that are bound by arithmetic
// rather than memory (the FP64 leapfrog, the resident FP32 time loop) report
// their fraction of these measured rates instead of a nominal figure.  Each
// thread runs eight independent FMA chains (enough independent work to keep
// the pipe busy at any occupancy the grid reaches); nothing is read from or
// written to global memory except one word that is stored only when a chain
// lands on a value it never reaches, which keeps the chains live.
#include <string.h>

#include "internal.cuh"

namespace ffpat {

__device__ double g_probe_sink;

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_fma_rate(int iters, double seed) {
  const float s = (float)seed + 1e-3f * (float)(threadIdx.x & 31);
  if constexpr (KIND == 0) {
    double a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = seed + 1e-3 * (threadIdx.x + i);
    const double m = 1.0 - 1e-12, c = 1e-9;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) t += a[i];
    if (t == -1.0) g_probe_sink = t;
  } else if constexpr (KIND == 1) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = s + 1e-3f * i;
    const float m = 1.0f - 1e-7f, c = 1e-7f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, c);
    float t = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) t += a[i];
    if (t == -1.0f) g_probe_sink = t;
  } else {
    // two FP32 lanes per instruction (fma.rn.f32x2, as in the stencil kernels)
    unsigned long long a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      const float2 v = make_float2(s + 1e-3f * i, s - 1e-3f * i);
      memcpy(&a[i], &v, sizeof v);
    }
    const float2 mf = make_float2(1.0f - 1e-7f, 1.0f - 2e-7f), cf = make_float2(1e-7f, 2e-7f);
    unsigned long long m, c;
    memcpy(&m, &mf, sizeof m);
    memcpy(&c, &cf, sizeof c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int i = 0; i < kChains; ++i)
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(m), "l"(c));
    float t = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      float2 v;
      memcpy(&v, &a[i], sizeof v);
      t += v.x + v.y;
    }
    if (t == -1.0f) g_probe_sink = t;
  }
}

}  // namespace
}  // namespace ffpat

extern "C" int ffpat_debug_fma_rate(int32_t kind, double* flops_per_s, void* stream) {
  using namespace ffpat;
  if (kind < 0 || kind > 2 || !flops_per_s)
    return report(FFPAT_EINVAL, "ffpat_debug_fma_rate: kind %d outside 0..2 or null output", kind);
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return report(FFPAT_ECUDA, "ffpat_debug_fma_rate: device query failed");
  }
  // eight CTAs of 256 threads per SM (64 warps: every SM fully occupied)
  const int blocks = sms * 8;
  const int iters = kind == 0 ? 1024 : 16384;
  auto launch = [&](int it) {
    if (kind == 0)
      k_fma_rate<0><<<blocks, kThreads, 0, st>>>(it, 1.0);
    else if (kind == 1)
      k_fma_rate<1><<<blocks, kThreads, 0, st>>>(it, 1.0);
    else
      k_fma_rate<2><<<blocks, kThreads, 0, st>>>(it, 1.0);
    count_launch();
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return report(FFPAT_ECUDA, "ffpat_debug_fma_rate: cudaEventCreate failed");
  }
  launch(iters / 8);  // warm-up (clocks, instruction cache)
  double best = 0.0;
  int rc = FFPAT_OK;
  for (int rep = 0; rep < 3 && rc == FFPAT_OK; ++rep) {
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    const cudaError_t es = cudaEventSynchronize(e1);
    if (es != cudaSuccess) {
      cudaGetLastError();
      rc = report(FFPAT_ECUDA, "ffpat_debug_fma_rate: %s", cudaGetErrorString(es));
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    // one FMA is two floating-point operations per lane; the packed form has two lanes
    const double lanes = kind == 2 ? 2.0 : 1.0;
    const double flops = 2.0 * lanes * kChains * (double)iters * blocks * kThreads;
    if (ms > 0.0f) best = fmax(best, flops / (ms * 1e-3));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != FFPAT_OK) return rc;
  if ((rc = check_launch("ffpat_debug_fma_rate")) != FFPAT_OK) return rc;
  *flops_per_s = best;
  return FFPAT_OK;
}
