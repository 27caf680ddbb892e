// Constants and helpers shared by all kernels of libhenry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace henry {

constexpr int kNQ = 22;
constexpr int kStatusMaxit = 1;
constexpr int kStatusNonfinite = 2;
constexpr int kStatusBadInput = 4;
constexpr int kBlock = 256;
constexpr int kMaxCoarseUnknowns = 64;

#define HENRY_COUNT_LAUNCH(ctr)                                                        \
  do {                                                                                 \
    if (ctr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)                 \
      atomicAdd((unsigned long long*)(ctr), 1ULL);                                     \
  } while (0)

// Block sum of a double, result valid in thread 0. Fixed order.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
  return s;
}

// Tiling of the face-based residual kernel (see k_resjac).
struct ResTile {
  int TX, GR, R;    // columns per tile, row groups per block, rows per thread
  int ntx, nty;     // tiles per sample in x and y
};

// rmax: most rows a thread walks (more rows per thread: fewer blocks, fewer
// tile-edge recomputations of the south face; fewer: more parallelism for
// small batches). 0 selects the default, 8.
__host__ inline ResTile make_res_tile(int nx, int ny, int rmax = 0) {
  ResTile t;
  if (rmax <= 0) rmax = 8;
  t.TX = nx < kBlock ? nx : kBlock;
  t.GR = kBlock / t.TX;
  int rows = (ny + t.GR - 1) / t.GR;        // rows per thread if one tile covered all
  t.R = rows < rmax ? rows : rmax;
  t.ntx = (nx + t.TX - 1) / t.TX;
  t.nty = (ny + t.GR * t.R - 1) / (t.GR * t.R);
  return t;
}

}  // namespace henry
