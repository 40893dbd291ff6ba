// ism_peak.cu -- ism_measure_peak: the FP32 (packed FFMA2) and FP64 FMA rates this GPU sustains, the
// denominators of the ALU rooflines of the propagation kernels (whose FP32/FP64 pipes, not HBM or the
// tensor cores, bound them).  Every SM runs independent FMA chains, enough per thread to hide the
// pipe latency, for a fixed number of iterations; the rate is the executed flops over the CUDA-event
// time of the launch.
#include <cuda_runtime.h>

#include <string>

#include "ism.h"
#include "ism_launch.h"

namespace {

constexpr int kChains = 8;        // independent FMA chains per thread
constexpr int kThreads = 512;     // per CTA
constexpr int kIters = 1 << 11;   // loop trips per launch (~0.3 s per FP32 launch on a GB300)

// The chains' results go nowhere; a guarded store into this array (never taken in practice) keeps the
// compiler from removing them, and needs no caller memory.
__device__ double g_sink[1024];

__global__ void __launch_bounds__(kThreads) k_peak_fp32(float seed) {
  float2 a[kChains];
  const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = make_float2(seed + threadIdx.x * 1e-6f + i, seed - i);
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], m, c);   // 4 flops per packed FMA
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
  if (s == 12345.678f) g_sink[blockIdx.x & 1023] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_fp64(double seed) {
  double a[kChains];
  const double m = 0.9999999, c = 1e-9;
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = seed + threadIdx.x * 1e-6 + i;
  for (int it = 0; it < kIters / 16; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);   // 2 flops per FMA
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == 12345.678) g_sink[blockIdx.x & 1023] = s;
}

}  // namespace

extern "C" int ism_measure_peak(int which, double* tflops) {
  if (!tflops || (which != 0 && which != 1)) return ism::set_error(ISM_EINVAL, "which must be 0 (FP32) or 1 (FP64)");
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = which == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_fp32, kThreads, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_fp64, kThreads, 0);
  if (e != cudaSuccess) return ism::set_error(ISM_ECUDA, (std::string("device query: ") + cudaGetErrorString(e)).c_str());
  const int blocks = sms * (per_sm < 1 ? 1 : per_sm);
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 0.f;
  for (int rep = 0; rep < 4; ++rep) {   // the first launch warms the clocks up; keep the best
    cudaEventRecord(a);
    if (which == 0) k_peak_fp32<<<blocks, kThreads>>>(1.0f + rep);
    else k_peak_fp64<<<blocks, kThreads>>>(1.0 + rep);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    if (e != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return ism::set_error(ISM_ECUDA, (std::string("peak launch: ") + cudaGetErrorString(e)).c_str());
  const double flops = which == 0 ? 4.0 * kChains * (double)kIters * kThreads * blocks
                                  : 2.0 * kChains * (double)(kIters / 16) * kThreads * blocks;
  *tflops = flops / (best * 1e-3) / 1e12;
  ism::clear_error();
  return ISM_OK;
}
