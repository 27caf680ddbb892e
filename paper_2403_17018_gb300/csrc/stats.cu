// MLMC level statistics on the device (arxiv 2403.17018, section 3: Def. of
// Y_l and V_l, Eq. A). Welford updates in sample order per thread, merged
// with Chan's pairwise formula in a fixed tree, so the result depends only on
// the batch contents and B.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "henry_device.cuh"

namespace henry {

constexpr int kStatThreads = 128;

struct Acc {
  double n;
  double mf[kNQ], m2f[kNQ], md[kNQ], m2d[kNQ];
};

__device__ __forceinline__ void chan_merge(double na, double& ma, double& m2a, double nb, double mb,
                                           double m2b) {
  const double n = na + nb;
  if (nb == 0.0) return;
  if (na == 0.0) { ma = mb; m2a = m2b; return; }
  const double d = mb - ma;
  ma = ma + d * (nb / n);
  m2a = m2a + m2b + d * d * (na * nb / n);
}

// One block. out[0] = n, then mean_f[6], m2_f[6], mean_d[6], m2_d[6].
__global__ void k_level_stats(unsigned long long* ctr, int B, const double* __restrict__ qf,
                              const double* __restrict__ qc, const int* __restrict__ status,
                              double* __restrict__ out) {
  HENRY_COUNT_LAUNCH(ctr);
  __shared__ Acc acc[kStatThreads];
  const int t = threadIdx.x;
  Acc a;
  a.n = 0.0;
  for (int k = 0; k < kNQ; ++k) a.mf[k] = a.m2f[k] = a.md[k] = a.m2d[k] = 0.0;
  for (int b = t; b < B; b += blockDim.x) {
    if (status && status[b] != 0) continue;
    a.n += 1.0;
    for (int k = 0; k < kNQ; ++k) {
      const double g = qf[(int64_t)b * kNQ + k];
      const double d = qc ? g - qc[(int64_t)b * kNQ + k] : g;
      double e = g - a.mf[k];
      a.mf[k] += e / a.n;
      a.m2f[k] += e * (g - a.mf[k]);
      e = d - a.md[k];
      a.md[k] += e / a.n;
      a.m2d[k] += e * (d - a.md[k]);
    }
  }
  acc[t] = a;
  __syncthreads();
  for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
    if (t < stride) {
      Acc& x = acc[t];
      const Acc& y = acc[t + stride];
      for (int k = 0; k < kNQ; ++k) {
        chan_merge(x.n, x.mf[k], x.m2f[k], y.n, y.mf[k], y.m2f[k]);
        chan_merge(x.n, x.md[k], x.m2d[k], y.n, y.md[k], y.m2d[k]);
      }
      x.n += y.n;
    }
    __syncthreads();
  }
  if (t == 0) {
    out[0] = acc[0].n;
    for (int k = 0; k < kNQ; ++k) {
      out[1 + k] = acc[0].mf[k];
      out[1 + kNQ + k] = acc[0].m2f[k];
      out[1 + 2 * kNQ + k] = acc[0].md[k];
      out[1 + 3 * kNQ + k] = acc[0].m2d[k];
    }
  }
}

// Per-cell Welford of c_l and c_l - P0 c_{l-1} over the batch, in sample
// order, continuing the running state held in device memory.
__global__ void k_field_stats(unsigned long long* ctr, int nx, int ny, int B,
                              const double* __restrict__ cf, const double* __restrict__ cc,
                              const int* __restrict__ status, int64_t* __restrict__ n,
                              double* __restrict__ mean_f, double* __restrict__ m2_f,
                              double* __restrict__ mean_d, double* __restrict__ m2_d) {
  HENRY_COUNT_LAUNCH(ctr);
  const int ncell = nx * ny;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  const int j = cell / nx, i = cell - j * nx;
  const int nxc = nx / 2, ncc = (nx / 2) * (ny / 2);
  const int ccell = (j >> 1) * nxc + (i >> 1);
  double cnt = (double)n[cell];
  double mf = mean_f[cell], sf = m2_f[cell], md = mean_d[cell], sd = m2_d[cell];
  for (int b = 0; b < B; ++b) {
    if (status && status[b] != 0) continue;
    const double g = cf[(int64_t)b * ncell + cell];
    const double d = cc ? g - cc[(int64_t)b * ncc + ccell] : g;
    cnt += 1.0;
    double e = g - mf;
    mf += e / cnt;
    sf += e * (g - mf);
    e = d - md;
    md += e / cnt;
    sd += e * (d - md);
  }
  n[cell] = (int64_t)cnt;
  mean_f[cell] = mf;
  m2_f[cell] = sf;
  mean_d[cell] = md;
  m2_d[cell] = sd;
}

// Per-cell exceedance counts (section 4: probability that the salt mass
// fraction at a location exceeds a threshold): count[cell] += number of
// valid samples b with c_b[cell] > threshold. One thread per cell, samples in
// order, integer counts (exact, independent of batching).
__global__ void k_field_exceed(unsigned long long* ctr, int ncell, int B,
                               const double* __restrict__ c, const int* __restrict__ status,
                               double threshold, int64_t* __restrict__ count) {
  HENRY_COUNT_LAUNCH(ctr);
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  int64_t k = 0;
  for (int b = 0; b < B; ++b) {
    if (status && status[b] != 0) continue;
    k += c[(int64_t)b * ncell + cell] > threshold ? 1 : 0;
  }
  count[cell] += k;
}

cudaError_t launch_field_exceed(unsigned long long* ctr, int ncell, int B, const double* c,
                                const int* status, double threshold, int64_t* count,
                                cudaStream_t s) {
  k_field_exceed<<<(ncell + 255) / 256, 256, 0, s>>>(ctr, ncell, B, c, status, threshold, count);
  return cudaGetLastError();
}

cudaError_t launch_level_stats(unsigned long long* ctr, int B, const double* qf, const double* qc,
                               const int* status, double* out, cudaStream_t s) {
  k_level_stats<<<1, kStatThreads, 0, s>>>(ctr, B, qf, qc, status, out);
  return cudaGetLastError();
}

cudaError_t launch_field_stats(unsigned long long* ctr, int nx, int ny, int B, const double* cf,
                               const double* cc, const int* status, int64_t* n, double* mean_f,
                               double* m2_f, double* mean_d, double* m2_d, cudaStream_t s) {
  const int ncell = nx * ny;
  k_field_stats<<<(ncell + 255) / 256, 256, 0, s>>>(ctr, nx, ny, B, cf, cc, status, n, mean_f,
                                                    m2_f, mean_d, m2_d);
  return cudaGetLastError();
}

}  // namespace henry
