// Temporally blocked legs of the multigrid V-cycle (red-black point-block
// Gauss-Seidel smoothing, section 2.3) on the batched levels.
//
// The per-operation path launches one kernel per half-sweep, one for the
// residual restriction and one for the prolongation: 2 nu1 + 1 launches on
// the way down a level and 2 nu2 + 1 on the way up, each a full pass over
// the level. On the levels whose operators stay in L2 those launches are
// latency-bound. Here each leg is one launch: a block owns a tile of one
// sample's cells plus a halo, holds the tile's unknowns in shared memory
// and performs all of the leg's half-sweeps on it, reading the operator
// rows and right-hand sides from global memory (L2). A half-sweep can only
// be trusted where every neighbour it read was trusted, so the trusted
// region shrinks by one cell per half-sweep on every side that is not a
// domain boundary; a halo of 2 nu cells (plus one for the residual of the
// down leg) keeps the tile's interior exact. Each block writes back only
// its interior, to a second buffer: a tile's halo is read before the leg
// while the neighbouring tiles finish theirs, so every leg reads one copy
// of the level's unknowns and writes the other (the down leg from the
// level's x to its second buffer, the up leg back). The arithmetic per cell
// is that of gs_point, resid_point and prolong_value in the same order, so
// the results are bitwise those of the per-operation path.
//
// Shared layout of a tile: [var][colour][row][m], the colour-split order of
// the global planes restricted to the tile (m = (i - ex0) / 2 with ex0
// even), so that a warp's own cells and each of its neighbour reads are
// consecutive words.
#pragma once

#include "kernels.cuh"

namespace henry {

// The tile's extended region [ex0, ex1) x [ey0, ey1) and its interior.
struct TbRegion {
  int i0, i1, j0, j1;      // interior
  int ex0, ex1, ey0, ey1;  // interior plus halo, clipped to the domain
  int hEX, EY;             // half width (cells per colour and row), rows
  __device__ __forceinline__ TbRegion(const Geom& G, const TbTile& t, int tile) {
    const int ty = tile / t.ntx, tx = tile - ty * t.ntx;
    i0 = tx * t.TX;
    j0 = ty * t.TY;
    i1 = i0 + t.TX < G.nx ? i0 + t.TX : G.nx;
    j1 = j0 + t.TY < G.ny ? j0 + t.TY : G.ny;
    const int hx = (t.H + 1) & ~1;
    ex0 = i0 - hx > 0 ? i0 - hx : 0;
    ex1 = i1 + hx < G.nx ? i1 + hx : G.nx;
    ey0 = j0 - t.H > 0 ? j0 - t.H : 0;
    ey1 = j1 + t.H < G.ny ? j1 + t.H : G.ny;
    hEX = (ex1 - ex0) >> 1;
    EY = ey1 - ey0;
  }
  // shared index of cell (i, j), variable v
  __device__ __forceinline__ int at(int v, int i, int j) const {
    return ((v * 2 + ((i + j) & 1)) * EY + (j - ey0)) * hEX + ((i - ex0) >> 1);
  }
};

// One half-sweep of colour c over the cells of the tile that are trusted
// after s half-sweeps (the extended region shrunk by s on every side that
// is not a domain boundary).
template <typename T, int P0>
__device__ __forceinline__ void tb_half_sweep(const Geom& G, const TbRegion& R, int c, int s,
                                              const T* __restrict__ Js, const T* __restrict__ bs,
                                              T* xs) {
  const int ncell = G.ncell(), half = G.half(), hx2 = G.nx >> 1;
  const int vx0 = R.ex0 == 0 ? 0 : R.ex0 + s, vx1 = R.ex1 == G.nx ? G.nx : R.ex1 - s;
  const int vy0 = R.ey0 == 0 ? 0 : R.ey0 + s, vy1 = R.ey1 == G.ny ? G.ny : R.ey1 - s;
  const int items = (vy1 - vy0) * R.hEX;
  auto nb = [&](int ii, int jj, T& vp, T& vc) {
    vp = xs[R.at(0, ii, jj)];
    vc = xs[R.at(1, ii, jj)];
  };
  for (int e = threadIdx.x; e < items; e += blockDim.x) {
    const int r = e / R.hEX, m = e - r * R.hEX;
    const int j = vy0 + r;
    const int i = R.ex0 + 2 * m + ((c + j) & 1);
    if (i < vx0 || i >= vx1) continue;
    const int cs = c * half + j * hx2 + (i >> 1);
    T xp, xc;
    gs_point<T, P0>(i, j, G.nx, G.ny, ncell, Js + cs, bs[cs], bs[ncell + cs], nb, xp, xc);
    xs[R.at(0, i, j)] = xp;
    xs[R.at(1, i, j)] = xc;
  }
}

// Copy the tile's interior unknowns back to the sample's global planes.
template <typename T>
__device__ __forceinline__ void tb_store_interior(const Geom& G, const TbRegion& R,
                                                  const T* xs, T* __restrict__ xg) {
  const int ncell = G.ncell(), half = G.half(), hx2 = G.nx >> 1;
  const int hw = (R.i1 - R.i0) >> 1, rows = R.j1 - R.j0;
  const int items = 2 * rows * hw;
  for (int e = threadIdx.x; e < items; e += blockDim.x) {
    const int c = e / (rows * hw);
    const int rr = e - c * rows * hw;
    const int r = rr / hw, m = rr - r * hw;
    const int j = R.j0 + r;
    const int i = R.i0 + 2 * m + ((c + j) & 1);
    const int cs = c * half + j * hx2 + (i >> 1);
    xg[cs] = xs[R.at(0, i, j)];
    xg[ncell + cs] = xs[R.at(1, i, j)];
  }
}

// Load the extended tile's unknowns from the sample's global planes
// (consecutive threads read consecutive words of one colour's row run);
// with PROLONG, black cells get x_f + P x_c (the red half-sweep that follows
// rewrites every red value without reading it).
template <typename T, bool PROLONG>
__device__ __forceinline__ void tb_load(const Geom& G, const TbRegion& R, const T* __restrict__ xg,
                                        const Geom& Gc, const T* __restrict__ xcs, T* xs) {
  const int ncell = G.ncell(), half = G.half(), hx2 = G.nx >> 1;
  const int items = 2 * R.EY * R.hEX;
  for (int e = threadIdx.x; e < items; e += blockDim.x) {
    const int c = e / (R.EY * R.hEX);
    const int rr = e - c * R.EY * R.hEX;
    const int r = rr / R.hEX, m = rr - r * R.hEX;
    const int j = R.ey0 + r;
    const int cs = c * half + j * hx2 + (R.ex0 >> 1) + m;
    T xp = xg[cs], xv = xg[ncell + cs];
    if (PROLONG && c == 1) {
      const int i = R.ex0 + 2 * m + ((1 + j) & 1);
      T vp, vc;
      prolong_value<T>(Gc, i, j, xcs, vp, vc);
      xp += vp;
      xv += vc;
    }
    xs[(c * R.EY + r) * R.hEX + m] = xp;
    xs[((2 + c) * R.EY + r) * R.hEX + m] = xv;
  }
}

// Down leg of level G: nu1 red-black sweeps on (J, b, x) starting from
// xin, the result to xout, then the finite-volume restriction of the
// residual to level Gc (b_c scaled by the coarse Dinv, x_c = 0), as
// restrict_cell. nu1 >= 1; the tile's halo is 2 nu1 + 1. Grid (tiles, B),
// kTbBlock threads. STAGED (one tile per sample): operator planes 4..23,
// b and x are first copied to shared memory by TMA bulk copies, in the
// sample's global colour-split layout, and every operation runs out of
// shared memory with the per-cell routines of the per-operation kernels; a
// copy that does not land within the bounded wait flags status[b]
// (kStatusStall) and leaves the sample.
template <typename T, bool STAGED>
__global__ void __launch_bounds__(kTbBlock)
k_tb_down(unsigned long long* ctr, Geom G, Geom Gc, int B, const int* __restrict__ active,
          TbTile t, int nu1, const T* __restrict__ J, const T* __restrict__ bvec,
          const T* __restrict__ xin, T* __restrict__ xout, const T* __restrict__ Jc,
          T* __restrict__ bc, T* __restrict__ xc, int* __restrict__ status) {
  HENRY_COUNT_LAUNCH(ctr);
  extern __shared__ __align__(16) unsigned char tb_sh[];
  const int b = blockIdx.y;
  if (!active[b]) return;
  const int ncell = G.ncell(), half = G.half(), ncc = Gc.ncell();
  const T* Js = J + (int64_t)b * kJP * ncell;
  const T* bs = bvec + (int64_t)b * 2 * ncell;
  const T* xg = xin + (int64_t)b * 2 * ncell;
  T* xo = xout + (int64_t)b * 2 * ncell;
  const T* Jcs = Jc + (int64_t)b * kJP * ncc;
  T* bcs = bc + (int64_t)b * 2 * ncc;
  T* xcs = xc + (int64_t)b * 2 * ncc;
  if (STAGED) {
    // the whole sample in shared memory, in its global layout: the
    // per-cell routines of the per-operation kernels apply unchanged
    uint64_t* bar = (uint64_t*)tb_sh;
    T* Jst = (T*)(tb_sh + 16);           // planes 4..23
    T* bst = Jst + 20 * ncell;
    T* xs = bst + 2 * ncell;
    auto runs = [&](auto&& f) {
      f(Jst, Js + 4 * ncell, (unsigned)(20 * ncell * sizeof(T)));
      f(bst, bs, (unsigned)(2 * ncell * sizeof(T)));
      f(xs, xg, (unsigned)(2 * ncell * sizeof(T)));
    };
    if (!stage_runs(bar, runs, status, b)) return;
    for (int s = 0; s < 2 * nu1; ++s) {
      for (int pos = threadIdx.x; pos < half; pos += blockDim.x)
        smooth_cell<T, 4>(G, s & 1, pos, Jst, bst, xs);
      __syncthreads();
    }
    for (int e = threadIdx.x; e < 2 * ncell; e += blockDim.x) xo[e] = xs[e];
    for (int cell = threadIdx.x; cell < ncc; cell += blockDim.x)
      restrict_cell<T, 4>(G, Gc, cell, Jst, bst, xs, Jcs, bcs, xcs, true);
    return;
  }
  const TbRegion R(G, t, blockIdx.x);
  T* xs = (T*)tb_sh;
  tb_load<T, false>(G, R, xg, Gc, nullptr, xs);
  __syncthreads();
  for (int s = 1; s <= 2 * nu1; ++s) {
    tb_half_sweep<T, 0>(G, R, (s - 1) & 1, s, Js, bs, xs);
    __syncthreads();
  }
  tb_store_interior<T>(G, R, xs, xo);
  // restriction: the coarse cells whose children are this tile's interior;
  // after a black half-sweep only the red children carry a residual
  const int cw = (R.i1 - R.i0) >> 1, ch = (R.j1 - R.j0) >> 1;
  auto nb = [&](int ii, int jj, T& vp, T& vc) {
    vp = xs[R.at(0, ii, jj)];
    vc = xs[R.at(1, ii, jj)];
  };
  for (int e = threadIdx.x; e < cw * ch; e += blockDim.x) {
    const int rj = e / cw;
    const int I = (R.i0 >> 1) + (e - rj * cw), Jr = (R.j0 >> 1) + rj;
    T sp = 0, sc = 0;
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
      if (c4 == 1 || c4 == 2) continue;
      const int i = 2 * I + (c4 & 1), j = 2 * Jr + (c4 >> 1);
      const int cs = cs_pos(i, j, G.nx, half);
      T rp, rc;
      resid_point<T>(i, j, G.nx, G.ny, ncell, Js + cs, bs[cs], bs[ncell + cs], xs[R.at(0, i, j)],
                     xs[R.at(1, i, j)], nb, rp, rc);
      sp += rp;
      sc += rc;
    }
    const int csc = cs_pos(I, Jr, Gc.nx, Gc.half());
    const T* d = Jcs + csc;
    bcs[csc] = d[0] * sp + d[ncc] * sc;
    bcs[ncc + csc] = d[2 * ncc] * sp + d[3 * ncc] * sc;
    xcs[csc] = (T)0;
    xcs[ncc + csc] = (T)0;
  }
}

// Up leg of level G: xin + P x_c on the black cells (the red half-sweep
// that follows rewrites every red value without reading it), then nu2
// red-black sweeps, the result to xout. nu2 >= 1; the tile's halo is
// 2 nu2. Grid (tiles, B), kTbBlock threads. STAGED as in k_tb_down, with
// operator planes 4..19.
template <typename T, bool STAGED>
__global__ void __launch_bounds__(kTbBlock)
k_tb_up(unsigned long long* ctr, Geom Gc, Geom G, int B, const int* __restrict__ active,
        TbTile t, int nu2, const T* __restrict__ xc, const T* __restrict__ J,
        const T* __restrict__ bvec, const T* __restrict__ xin, T* __restrict__ xout,
        int* __restrict__ status) {
  HENRY_COUNT_LAUNCH(ctr);
  extern __shared__ __align__(16) unsigned char tb_sh[];
  const int b = blockIdx.y;
  if (!active[b]) return;
  const int ncell = G.ncell(), half = G.half();
  const T* Js = J + (int64_t)b * kJP * ncell;
  const T* bs = bvec + (int64_t)b * 2 * ncell;
  const T* xg = xin + (int64_t)b * 2 * ncell;
  T* xo = xout + (int64_t)b * 2 * ncell;
  const T* xcs = xc + (int64_t)b * 2 * Gc.ncell();
  if (STAGED) {
    uint64_t* bar = (uint64_t*)tb_sh;
    T* Jst = (T*)(tb_sh + 16);           // planes 4..19
    T* bst = Jst + 16 * ncell;
    T* xs = bst + 2 * ncell;
    auto runs = [&](auto&& f) {
      f(Jst, Js + 4 * ncell, (unsigned)(16 * ncell * sizeof(T)));
      f(bst, bs, (unsigned)(2 * ncell * sizeof(T)));
      f(xs, xg, (unsigned)(2 * ncell * sizeof(T)));
    };
    if (!stage_runs(bar, runs, status, b)) return;
    for (int pos = threadIdx.x; pos < half; pos += blockDim.x)
      prolong_cell<T>(Gc, G, black_cell(G, pos), xcs, xs);
    __syncthreads();
    for (int s = 0; s < 2 * nu2; ++s) {
      for (int pos = threadIdx.x; pos < half; pos += blockDim.x)
        smooth_cell<T, 4>(G, s & 1, pos, Jst, bst, xs);
      __syncthreads();
    }
    for (int e = threadIdx.x; e < 2 * ncell; e += blockDim.x) xo[e] = xs[e];
    return;
  }
  const TbRegion R(G, t, blockIdx.x);
  T* xs = (T*)tb_sh;
  tb_load<T, true>(G, R, xg, Gc, xcs, xs);
  __syncthreads();
  for (int s = 1; s <= 2 * nu2; ++s) {
    tb_half_sweep<T, 0>(G, R, (s - 1) & 1, s, Js, bs, xs);
    __syncthreads();
  }
  tb_store_interior<T>(G, R, xs, xo);
}

// Clustered staged legs: a level whose sample does not fit one block's
// shared memory is split into CL strips of R = ny / CL rows (R even), one
// block of a thread-block cluster per strip. Each block stages its strip's
// operator planes (4..23 down, 4..19 up), b and x by TMA bulk copies, in the
// strip's own colour-split layout [plane][colour][row][m] (every run of a
// colour's rows is contiguous in the global planes); the unknowns of the row
// above and below the strip are read from the neighbouring blocks' shared
// memory (distributed shared memory), and every phase ends with a hardware
// cluster barrier, whose release/acquire order makes a phase's writes
// visible to the next phase's remote reads. Per cell the operations are
// those of gs_point, resid_point and prolong_value in the same order, so the
// results are bitwise those of the per-operation path. Grid B * CL, clusters
// of CL blocks, kTbBlock threads.
template <typename T>
struct StripX {
  const T* lo;   // the block below (rows j0 - 1), or null
  const T* me;
  const T* hi;   // the block above (row j0 + R), or null
  int j0, R, hs, hx2;
  __device__ __forceinline__ void operator()(int i, int j, T& vp, T& vc) const {
    const T* X = me;
    int r = j - j0;
    if (r < 0) { X = lo; r = R - 1; }
    else if (r >= R) { X = hi; r = 0; }
    const int idx = ((i + j) & 1) * hs + r * hx2 + (i >> 1);
    vp = X[idx];
    vc = X[2 * hs + idx];
  }
};

// Stage with the whole cluster: true when every block's copies landed (the
// decision is the same in every block of the cluster).
template <typename Runs>
__device__ __forceinline__ bool cluster_stage(uint64_t* bar, int* flag, Runs runs, int* status,
                                              int b) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const bool ok = stage_runs(bar, runs, status, b);
  if (threadIdx.x == 0) flag[0] = ok ? 1 : 0;
  cl.sync();
  if (threadIdx.x == 0) {
    int all = 1;
    for (unsigned r = 0; r < cl.num_blocks(); ++r) all &= *cl.map_shared_rank(flag, r);
    flag[1] = all;
  }
  cl.sync();   // every block has read every flag before any block may leave
  return flag[1] != 0;
}

template <typename T>
__global__ void __launch_bounds__(kTbBlock)
k_tbc_down(unsigned long long* ctr, Geom G, Geom Gc, int B, const int* __restrict__ active,
           int nu1, int CL, const T* __restrict__ J, const T* __restrict__ bvec,
           const T* __restrict__ xin, T* __restrict__ xout, const T* __restrict__ Jc,
           T* __restrict__ bc, T* __restrict__ xc, int* __restrict__ status) {
  HENRY_COUNT_LAUNCH(ctr);
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char tb_sh[];
  const int b = blockIdx.x / CL, rank = blockIdx.x - b * CL;
  if (!active[b]) return;                      // uniform over the cluster
  const int ncell = G.ncell(), half = G.half(), hx2 = G.nx >> 1;
  const int R = G.ny / CL, j0 = rank * R, hs = R * hx2;
  uint64_t* bar = (uint64_t*)tb_sh;
  int* flag = (int*)(tb_sh + 8);
  T* Jst = (T*)(tb_sh + 16);                   // planes 4..23, [plane][colour][row][m]
  T* bst = Jst + 40 * hs;
  T* xs = bst + 4 * hs;
  const T* Js = J + (int64_t)b * kJP * ncell;
  const T* bs = bvec + (int64_t)b * 2 * ncell;
  const T* xg = xin + (int64_t)b * 2 * ncell;
  auto runs = [&](auto&& f) {
    for (int q = 4; q < 24; ++q)
      for (int c = 0; c < 2; ++c)
        f(Jst + ((q - 4) * 2 + c) * hs, Js + (int64_t)q * ncell + c * half + j0 * hx2,
          (unsigned)(hs * sizeof(T)));
    for (int v = 0; v < 2; ++v)
      for (int c = 0; c < 2; ++c) {
        f(bst + (v * 2 + c) * hs, bs + v * ncell + c * half + j0 * hx2, (unsigned)(hs * sizeof(T)));
        f(xs + (v * 2 + c) * hs, xg + v * ncell + c * half + j0 * hx2, (unsigned)(hs * sizeof(T)));
      }
  };
  if (!cluster_stage(bar, flag, runs, status, b)) return;
  const StripX<T> nb{rank > 0 ? cl.map_shared_rank(xs, rank - 1) : nullptr, xs,
                     rank < CL - 1 ? cl.map_shared_rank(xs, rank + 1) : nullptr, j0, R, hs, hx2};
  for (int s = 0; s < 2 * nu1; ++s) {
    const int c = s & 1;
    for (int pos = threadIdx.x; pos < hs; pos += blockDim.x) {
      const int r = pos / hx2, m = pos - r * hx2, j = j0 + r;
      const int i = 2 * m + ((c + j) & 1), own = c * hs + pos;
      T xp, xv;
      gs_point<T, 4>(i, j, G.nx, G.ny, 2 * hs, Jst + own, bst[own], bst[2 * hs + own], nb, xp, xv);
      xs[own] = xp;
      xs[2 * hs + own] = xv;
    }
    cl.sync();
  }
  T* xo = xout + (int64_t)b * 2 * ncell;
  for (int e = threadIdx.x; e < 4 * hs; e += blockDim.x) {
    const int vc = e / hs, k = e - vc * hs;       // vc = v * 2 + c
    xo[(vc >> 1) * ncell + (vc & 1) * half + j0 * hx2 + k] = xs[e];
  }
  // restriction of the coarse rows j0/2 .. (j0 + R)/2 - 1 (red children)
  const int ncc = Gc.ncell();
  const T* Jcs = Jc + (int64_t)b * kJP * ncc;
  T* bcs = bc + (int64_t)b * 2 * ncc;
  T* xcs = xc + (int64_t)b * 2 * ncc;
  for (int e = threadIdx.x; e < hx2 * (R >> 1); e += blockDim.x) {
    const int rj = e / hx2;
    const int I = e - rj * hx2, Jr = (j0 >> 1) + rj;
    T sp = 0, sc = 0;
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
      if (c4 == 1 || c4 == 2) continue;
      const int i = 2 * I + (c4 & 1), j = 2 * Jr + (c4 >> 1);
      const int own = ((i + j) & 1) * hs + (j - j0) * hx2 + (i >> 1);
      T rp, rc;
      resid_point<T, 4>(i, j, G.nx, G.ny, 2 * hs, Jst + own, bst[own], bst[2 * hs + own], xs[own],
                        xs[2 * hs + own], nb, rp, rc);
      sp += rp;
      sc += rc;
    }
    const int csc = cs_pos(I, Jr, Gc.nx, Gc.half());
    const T* d = Jcs + csc;
    bcs[csc] = d[0] * sp + d[ncc] * sc;
    bcs[ncc + csc] = d[2 * ncc] * sp + d[3 * ncc] * sc;
    xcs[csc] = (T)0;
    xcs[ncc + csc] = (T)0;
  }
  cl.sync();   // no block leaves while another may still read its unknowns
}

template <typename T>
__global__ void __launch_bounds__(kTbBlock)
k_tbc_up(unsigned long long* ctr, Geom Gc, Geom G, int B, const int* __restrict__ active, int nu2,
         int CL, const T* __restrict__ xc, const T* __restrict__ J, const T* __restrict__ bvec,
         const T* __restrict__ xin, T* __restrict__ xout, int* __restrict__ status) {
  HENRY_COUNT_LAUNCH(ctr);
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char tb_sh[];
  const int b = blockIdx.x / CL, rank = blockIdx.x - b * CL;
  if (!active[b]) return;                      // uniform over the cluster
  const int ncell = G.ncell(), half = G.half(), hx2 = G.nx >> 1;
  const int R = G.ny / CL, j0 = rank * R, hs = R * hx2;
  uint64_t* bar = (uint64_t*)tb_sh;
  int* flag = (int*)(tb_sh + 8);
  T* Jst = (T*)(tb_sh + 16);                   // planes 4..19
  T* bst = Jst + 32 * hs;
  T* xs = bst + 4 * hs;
  const T* Js = J + (int64_t)b * kJP * ncell;
  const T* bs = bvec + (int64_t)b * 2 * ncell;
  const T* xg = xin + (int64_t)b * 2 * ncell;
  const T* xcs = xc + (int64_t)b * 2 * Gc.ncell();
  auto runs = [&](auto&& f) {
    for (int q = 4; q < 20; ++q)
      for (int c = 0; c < 2; ++c)
        f(Jst + ((q - 4) * 2 + c) * hs, Js + (int64_t)q * ncell + c * half + j0 * hx2,
          (unsigned)(hs * sizeof(T)));
    for (int v = 0; v < 2; ++v)
      for (int c = 0; c < 2; ++c) {
        f(bst + (v * 2 + c) * hs, bs + v * ncell + c * half + j0 * hx2, (unsigned)(hs * sizeof(T)));
        f(xs + (v * 2 + c) * hs, xg + v * ncell + c * half + j0 * hx2, (unsigned)(hs * sizeof(T)));
      }
  };
  if (!cluster_stage(bar, flag, runs, status, b)) return;
  // prolongation onto the strip's black cells
  for (int pos = threadIdx.x; pos < hs; pos += blockDim.x) {
    const int r = pos / hx2, m = pos - r * hx2, j = j0 + r;
    const int i = 2 * m + ((1 + j) & 1);
    T vp, vc;
    prolong_value<T>(Gc, i, j, xcs, vp, vc);
    xs[hs + pos] += vp;
    xs[3 * hs + pos] += vc;
  }
  cl.sync();
  const StripX<T> nb{rank > 0 ? cl.map_shared_rank(xs, rank - 1) : nullptr, xs,
                     rank < CL - 1 ? cl.map_shared_rank(xs, rank + 1) : nullptr, j0, R, hs, hx2};
  for (int s = 0; s < 2 * nu2; ++s) {
    const int c = s & 1;
    for (int pos = threadIdx.x; pos < hs; pos += blockDim.x) {
      const int r = pos / hx2, m = pos - r * hx2, j = j0 + r;
      const int i = 2 * m + ((c + j) & 1), own = c * hs + pos;
      T xp, xv;
      gs_point<T, 4>(i, j, G.nx, G.ny, 2 * hs, Jst + own, bst[own], bst[2 * hs + own], nb, xp, xv);
      xs[own] = xp;
      xs[2 * hs + own] = xv;
    }
    cl.sync();   // the last one also keeps every block until no remote read is left
  }
  T* xo = xout + (int64_t)b * 2 * ncell;
  for (int e = threadIdx.x; e < 4 * hs; e += blockDim.x) {
    const int vc = e / hs, k = e - vc * hs;
    xo[(vc >> 1) * ncell + (vc & 1) * half + j0 * hx2 + k] = xs[e];
  }
}

}  // namespace henry
