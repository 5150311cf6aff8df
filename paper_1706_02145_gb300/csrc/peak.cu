// Measured FMA issue peak of the current device: the denominator of the
// coupling kernels' roofline.  The coupling matvec is bound by plain FP32
// (FP64 for the refinement residuals) fused multiply-add issue, and neither
// peak is a datasheet constant worth trusting on this part (its FP64 rate is
// a small fraction of FP32), so it is measured: every thread runs 16
// independent FMA chains for a fixed number of iterations, on a grid of
// 4 x 256-thread CTAs per SM (32 warps per SM, 8 per scheduler), and the
// launch is timed with CUDA events on its own stream.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/celes.h"
#include "kernels.h"

namespace celes {
namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(int iters, T b, T c, T* __restrict__ out) {
  T a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = static_cast<T>(threadIdx.x + q) * static_cast<T>(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], b, c);
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}

// the packed two-lane FP32 FMA (__ffma2_rn, sm_100 and later): one
// instruction, two FMAs
__global__ void __launch_bounds__(kThreads) ffma2_chains_kernel(int iters, float b, float c, float* __restrict__ out) {
  float2 a[kChains / 2];
#pragma unroll
  for (int q = 0; q < kChains / 2; ++q)
    a[q] = make_float2(static_cast<float>(threadIdx.x + q) * 1e-3f, static_cast<float>(threadIdx.x - q) * 1e-3f);
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains / 2; ++q) a[q] = __ffma2_rn(a[q], bb, cc);
    // two packed FMAs per chain pair per iteration, so that the FMA count per
    // iteration equals the scalar kernel's
#pragma unroll
    for (int q = 0; q < kChains / 2; ++q) a[q] = __ffma2_rn(a[q], bb, cc);
  }
  float s = 0;
#pragma unroll
  for (int q = 0; q < kChains / 2; ++q) s += a[q].x + a[q].y;
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace celes

extern "C" int celes_fma_peak(int kind, double* tflops, double* ms_out) {
  using namespace celes;
  if (!tflops || kind < 0 || kind > 2) return CELES_EINVAL;
  const int sms = device_sms();
  const int blocks = 4 * sms;
  // FP64 issues at a small fraction of the FP32 rate: fewer iterations keep
  // each launch near 10-50 ms
  const int iters = kind == 0 ? 1 << 10 : 1 << 15;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* out = nullptr;
  int status = CELES_ECUDA;
  float best = 0.0f;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return CELES_ECUDA;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
  if (cudaMalloc(&out, static_cast<size_t>(blocks) * kThreads * sizeof(double)) != cudaSuccess) {
    status = CELES_ENOMEM;
    goto done;
  }
  // one warm-up launch, then the best of three timed launches
  for (int rep = 0; rep < 4; ++rep) {
    if (cudaEventRecord(e0, st) != cudaSuccess) goto done;
    if (kind == 0)
      fma_chains_kernel<double><<<blocks, kThreads, 0, st>>>(iters, 0.999999, 1e-7, static_cast<double*>(out));
    else if (kind == 1)
      fma_chains_kernel<float><<<blocks, kThreads, 0, st>>>(iters, 0.9999f, 1e-4f, static_cast<float*>(out));
    else
      ffma2_chains_kernel<<<blocks, kThreads, 0, st>>>(iters, 0.9999f, 1e-4f, static_cast<float*>(out));
    note_launch();
    if (cudaGetLastError() != cudaSuccess) goto done;
    if (cudaEventRecord(e1, st) != cudaSuccess) goto done;
    if (cudaEventSynchronize(e1) != cudaSuccess) goto done;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) goto done;
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  {
    const double fmas = static_cast<double>(blocks) * kThreads * iters * kChains;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    status = CELES_OK;
  }
done:
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return status;
}
