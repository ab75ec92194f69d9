// FP32 FMA throughput microbenchmark (psdf_measure_fp32_peak): the
// denominator of the FP32 roofline the benchmark reports for the PSDF
// kernels, measured on the GPU at hand instead of derived from unit counts.
//
// Every thread runs kChains independent multiply-add chains x <- x a + b
// (enough independent work per warp to hide the FMA latency), as scalar
// FP32 FMAs or as Blackwell's paired FP32 FMAs (two lanes of a float2 per
// instruction), over a grid that fills every SM.  Counted flops: 2 per FMA.
#include <algorithm>

#include "psdf_internal.h"

namespace psdf {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <bool PAIRED>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float *out, int iters, float a,
                                                                float b)
{
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float r = 0.f;
  if constexpr (PAIRED) {
    float2 x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = make_float2(1e-3f * (t & 7) + k, 0.5f * k);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
#pragma unroll
    for (int k = 0; k < kChains; ++k) r += x[k].x + x[k].y;
  } else {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (t & 7) + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
    }
#pragma unroll
    for (int k = 0; k < kChains; ++k) r += x[k];
  }
  out[t] = r;  // keeps the chains live
}

}  // namespace
}  // namespace psdf

using namespace psdf;

extern "C" int psdf_measure_fp32_peak(int32_t paired, int32_t iters, int32_t reps,
                                      double *tflops, double *best_ms, void *stream)
{
  if (!tflops || iters < 1 || reps < 1) return fail(PSDF_ERR_ARG, "bad argument");
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device attributes");
  const int blocks = sms * std::max(1, per_sm / kPeakThreads);
  const size_t n = (size_t)blocks * kPeakThreads;
  cudaStream_t st = (cudaStream_t)stream;
  float *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&out, n * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 1e30;
  auto kern = paired ? fma_peak_kernel<true> : fma_peak_kernel<false>;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // launch 0 warms up
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      kern<<<blocks, kPeakThreads, 0, st>>>(out, iters, 0.9999f, 1e-4f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0) best = std::min(best, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "psdf_measure_fp32_peak");
  const double flops = 2.0 * kChains * (paired ? 2.0 : 1.0) * (double)iters * (double)n;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (best_ms) *best_ms = best;
  return PSDF_OK;
}
