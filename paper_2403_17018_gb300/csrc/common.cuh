// Constants and helpers shared by all kernels of libhenry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace henry {

constexpr int kNQ = 22;
constexpr int kStatusMaxit = 1;
constexpr int kStatusNonfinite = 2;
constexpr int kStatusBadInput = 4;
constexpr int kStatusStall = 8;      // a bounded wait for an asynchronous copy gave up
constexpr int kBlock = 256;
constexpr int kMaxCoarseUnknowns = 64;

#define HENRY_COUNT_LAUNCH(ctr)                                                        \
  do {                                                                                 \
    if (ctr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)                 \
      atomicAdd((unsigned long long*)(ctr), 1ULL);                                     \
  } while (0)

// ---------------------------------------------------------------------------
// One-dimensional bulk copies from global to shared memory by the TMA unit
// (cp.async.bulk), completing on an mbarrier in shared memory. A copy needs
// both addresses and its size to be multiples of 16 bytes (bulk_ok); callers
// copy anything else with plain loads. Waits are bounded by the global
// timer so that a copy that never lands cannot hang the block.
// ---------------------------------------------------------------------------
constexpr unsigned long long kBulkWaitNs = 200000000ull;   // 0.2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool bulk_ok(const void* dst, const void* src, size_t bytes) {
  return bytes > 0 && ((((uintptr_t)dst) | ((uintptr_t)src) | (uintptr_t)bytes) & 15) == 0;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also raises the barrier's expected transaction bytes.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of the barrier; false when kBulkWaitNs passed first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kBulkWaitNs) return false;
  return true;
}

// Stage the runs that runs(f) enumerates as f(destination in shared memory,
// source in global memory, bytes; every size a multiple of 4) with the
// whole block: one thread issues a TMA bulk copy for each 16-byte aligned
// run, all threads copy the others with plain loads; bar is an mbarrier in
// shared memory. Returns true once everything has landed. When a copy does
// not land within the bounded wait, sets kStatusStall in status[b], gives
// the copies in flight one more bounded wait and returns false (uniformly
// over the block: the caller returns; a block of a cluster first agrees
// with the others, see cluster_stage).
template <typename Runs>
__device__ __forceinline__ bool stage_runs(uint64_t* bar, Runs runs, int* status, int b) {
  unsigned tx = 0;
  runs([&](void* d, const void* src, unsigned bytes) { tx += bulk_ok(d, src, bytes) ? bytes : 0u; });
  if (threadIdx.x == 0 && tx > 0) {
    mbar_init(bar, 1);
    mbar_arrive_expect_tx(bar, tx);
    runs([&](void* d, const void* src, unsigned bytes) {
      if (bulk_ok(d, src, bytes)) bulk_g2s(d, src, bytes, bar);
    });
  }
  runs([&](void* d, const void* src, unsigned bytes) {
    if (bulk_ok(d, src, bytes)) return;
    uint32_t* dw = (uint32_t*)d;
    const uint32_t* sw = (const uint32_t*)src;
    for (unsigned e = threadIdx.x; e < bytes / 4; e += blockDim.x) dw[e] = sw[e];
  });
  __syncthreads();              // the barrier is initialised before anyone waits on it
  if (tx > 0 && !__syncthreads_and(mbar_wait_bounded(bar, 0))) {
    if (threadIdx.x == 0) status[b] |= kStatusStall;
    mbar_wait_bounded(bar, 0);
    return false;
  }
  return true;
}

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
