// Arithmetic peaks of the current device, measured: the denominators of the
// rooflines of the kernels bound by CUDA-core arithmetic (the FFT-form
// source-to-target kernels on FP32, the near field on FP32 and the rsqrt
// unit, the effective-mass weights on FP64). Each kernel runs independent
// dependent-FMA chains in every thread of a grid that fills every SM, long
// enough (several milliseconds) that launch overhead does not count.
#include <algorithm>

#include "hpm_internal.cuh"

namespace hpm {
namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) k_peak_ffma(int iters, float a, float b, float *sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.f) *sink = s;  // never true for these inputs; keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_peak_dfma(int iters, double a, double b, double *sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) *sink = s;
}

// reciprocal square roots: x <- rsqrt(x) + b stays in [b, 1/sqrt(b) + b]
__global__ void __launch_bounds__(kThreads) k_peak_rsqrt(int iters, float b, float *sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.f + (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = rsqrtf(x[c]) + b;
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.f) *sink = s;
}

// best of `reps` timed launches of `launch` (milliseconds)
template <class F>
hpm_status best_ms(F &&launch, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps, float *out) {
  launch();  // warm-up
  HPM_CUDA(cudaGetLastError());
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    HPM_CUDA(cudaEventRecord(e0, st));
    launch();
    HPM_CUDA(cudaGetLastError());
    HPM_CUDA(cudaEventRecord(e1, st));
    HPM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    HPM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  *out = best;
  return HPM_OK;
}

}  // namespace
}  // namespace hpm

using namespace hpm;

extern "C" hpm_status hpm_measure_alu_peaks(hpm_alu_peaks *out, void *stream) {
  if (!out) return HPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int nsm = sm_count();
  const int blocks = nsm * kBlocksPerSm;
  const double threads = (double)blocks * kThreads;
  void *sink = nullptr;
  HPM_TRY(lib_malloc_async(&sink, 64, st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hpm_status s = HPM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = HPM_ERR_CUDA;
  // iterations chosen for ~5-10 ms per launch on this part
  const int it32 = 16384, it64 = 256, itrs = 2048;
  float ms32 = 0.f, ms64 = 0.f, msr = 0.f;
  if (s == HPM_OK)
    s = best_ms([&] { k_peak_ffma<<<blocks, kThreads, 0, st>>>(it32, 0.99999f, 1e-6f, (float *)sink); }, st, e0, e1,
                3, &ms32);
  if (s == HPM_OK)
    s = best_ms([&] { k_peak_dfma<<<blocks, kThreads, 0, st>>>(it64, 0.9999999, 1e-9, (double *)sink); }, st, e0,
                e1, 3, &ms64);
  if (s == HPM_OK)
    s = best_ms([&] { k_peak_rsqrt<<<blocks, kThreads, 0, st>>>(itrs, 0.5f, (float *)sink); }, st, e0, e1, 3, &msr);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  if (s != HPM_OK) return s;
  const double per_thread32 = 2.0 * kChains * 16.0 * it32, per_thread64 = 2.0 * kChains * 16.0 * it64;
  out->fp32_tflops = threads * per_thread32 / (ms32 * 1e-3) / 1e12;
  out->fp64_tflops = threads * per_thread64 / (ms64 * 1e-3) / 1e12;
  out->rsqrt_gops = threads * kChains * 16.0 * itrs / (msr * 1e-3) / 1e9;
  out->ms_fp32 = ms32;
  out->ms_fp64 = ms64;
  out->ms_rsqrt = msr;
  out->sm_count = nsm;
  return HPM_OK;
}
