// FP64 FMA throughput probe (henry_probe_fp64): the measured denominator of
// the FP64-pipe fraction that roofline reports give beside the HBM fraction.
#include <cuda_runtime.h>

#include "common.cuh"

namespace henry {

constexpr int kProbeBlocks = 152 * 8;
constexpr int kProbeBlock = 256;
constexpr int kProbeChains = 16;
constexpr int kProbeInner = 512;

// Sixteen independent dependency chains per thread keep the FP64 pipe busy
// (the latency of one FMA is hidden by the other fifteen); the multiplier and
// addend keep every value bounded, and the sum is stored so that nothing is
// eliminated.
__global__ void __launch_bounds__(kProbeBlock) k_probe_fp64(int reps, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = 1.0 + 1e-3 * (t + k);
  const double m = 0.999999, c = 1e-6;
  for (int r = 0; r < reps; ++r) {
#pragma unroll 8
    for (int i = 0; i < kProbeInner; ++i) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], m, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  out[t] = s;
}

cudaError_t probe_fp64(int reps, double* out, cudaStream_t s, double* tflops) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_probe_fp64<<<kProbeBlocks, kProbeBlock, 0, s>>>(1, out);   // warm-up
    cudaEventRecord(e0, s);
    k_probe_fp64<<<kProbeBlocks, kProbeBlock, 0, s>>>(reps, out);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double flop = 2.0 * kProbeChains * kProbeInner * (double)reps * kProbeBlocks * kProbeBlock;
  *tflops = flop / (ms * 1e-3) / 1e12;
  return cudaSuccess;
}

}  // namespace henry
