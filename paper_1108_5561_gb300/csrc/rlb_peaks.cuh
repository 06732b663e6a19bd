// rlb_peaks.cuh -- arithmetic-pipe peaks of the device, for the ALU rooflines
// of the stage kernels: FP32 fused multiply-add (FFMA), packed FP32 pairs
// (FFMA2, two multiply-adds per instruction) and FP64 (DFMA).
//
// Every thread runs K independent multiply-add chains (x <- x a + b), enough to
// cover the pipe latency, over a grid of 8 CTAs of 256 threads per SM; the
// chains converge to b / (1 - a) and stay normal.  A flop is counted as 2 per
// multiply-add (4 per FFMA2).  The result is written (to a file-scope device
// variable) only when it equals a value it cannot take, which keeps the chains
// live.
#pragma once

#include <cuda_runtime.h>

namespace rlbk {

__device__ double g_peak_sink;

constexpr int kPeakChains = 8, kPeakUnroll = 16;

__global__ void __launch_bounds__(256) peak_ffma_kernel(float a, float b, int iters) {
  float x[kPeakChains];
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kPeakUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kPeakChains; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) s += x[i];
  if (s == -1.f) g_peak_sink = s;
}

__global__ void __launch_bounds__(256) peak_ffma2_kernel(float a, float b, int iters) {
  float2 x[kPeakChains];
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) x[i] = make_float2(1e-3f * (float)(threadIdx.x + i), 2e-3f * (float)i);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kPeakUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kPeakChains; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) s += x[i].x + x[i].y;
  if (s == -1.f) g_peak_sink = s;
}

__global__ void __launch_bounds__(256) peak_dfma_kernel(double a, double b, int iters) {
  double x[kPeakChains];
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) x[i] = 1e-3 * (double)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kPeakUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kPeakChains; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) s += x[i];
  if (s == -1.0) g_peak_sink = s;
}

}  // namespace rlbk
