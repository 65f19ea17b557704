// Measurement helper with no counterpart in the paper: saturating loops of
// FP32 fused multiply-adds and of MUFU ex2, which the caller times to obtain
// the FP32-pipe and MUFU rates the GPU reaches at its current clocks (the
// denominators of the blend kernels' roofline).
#include "common.cuh"
#include "kernels.cuh"

namespace sixdgs {

constexpr int kProbeChains = 8;   // independent dependency chains per thread

__global__ void __launch_bounds__(256) fma_probe_kernel(float* out, int64_t iters, float c) {
  float x[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = fmaf(x[k], 0.99999f, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ex2_probe_kernel(float* out, int64_t iters, float c) {
  float x[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = -1e-3f * (float)(threadIdx.x + k);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = ex2_approx(x[k]) - c;   // stays in (-c, 1 - c]
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

void launch_peak_probe(int kind, int64_t iters, float* out, int blocks, cudaStream_t stream) {
  if (kind == 0)
    fma_probe_kernel<<<blocks, 256, 0, stream>>>(out, iters, 1e-4f);
  else
    ex2_probe_kernel<<<blocks, 256, 0, stream>>>(out, iters, 1.5f);
}

}  // namespace sixdgs
