// Batched kernels of the Henry solver. Every kernel works on B independent
// samples at once; per-sample arrays are contiguous blocks ([B][...]).
// Multigrid vectors and matrices use the colour-split plane layout of
// cs_pos() so that each red-black half-sweep streams one contiguous half of
// every plane. FP64 state (p, c) uses the natural row-major layout.
//
// Samples whose `active` flag is 0 (converged in this time step, or failed)
// are skipped by every per-iteration kernel, so a sample's result does not
// depend on which other samples share its batch.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"
#include "henry_device.cuh"

namespace henry {

// Multigrid operators are stored row-scaled by the inverse of each cell's
// 2x2 diagonal block D: the equations of cell P read
//   x_P + sum_Q Dinv_P A_PQ x_Q = Dinv_P b_P,
// and every level keeps the scaled right-hand side bt = Dinv b. kJP = 24
// planes per cell: 0..3 Dinv_P, 4..19 the scaled off-diagonal blocks
// At_PQ = Dinv_P A_PQ (Q = W, E, S, N), 20..23 D_P itself. A point
// Gauss-Seidel update is then x_P = bt_P - sum_Q At_PQ x_Q: 16 operator
// values and 16 multiply-adds, no 2x2 product (the smoother is HBM-bound in
// FP32 on large grids and FP64-pipe-bound in FP64, so both count). The
// restriction forms the unscaled residual D_P (bt_P - x_P - sum At x_Q) and
// scales the coarse right-hand side by the coarse Dinv.
constexpr int kJP = 24;
template <typename T>
__device__ __forceinline__ void inv2(T a, T b, T c, T d, T& ia, T& ib, T& ic, T& id) {
  const T r = (T)1 / (a * d - b * c);
  ia = d * r;
  ib = -b * r;
  ic = -c * r;
  id = a * r;
}

// Store one cell's operator: Jc holds the unscaled blocks (0..3 diagonal,
// 4..19 W, E, S, N; each block (pp, pc, cp, cc), row = equation). Returns
// Dinv in d[0..3] for scaling the right-hand side.
template <typename T>
__device__ __forceinline__ void store_operator(T* __restrict__ Jb, int ncell, const T* Jc, T* d) {
#pragma unroll
  for (int m = 0; m < 4; ++m) Jb[(int64_t)(20 + m) * ncell] = Jc[m];
  inv2<T>(Jc[0], Jc[1], Jc[2], Jc[3], d[0], d[1], d[2], d[3]);
#pragma unroll
  for (int m = 0; m < 4; ++m) Jb[(int64_t)m * ncell] = d[m];
#pragma unroll
  for (int q = 1; q <= 4; ++q) {
    const T a = Jc[4 * q], b = Jc[4 * q + 1], c = Jc[4 * q + 2], e = Jc[4 * q + 3];
    Jb[(int64_t)(4 * q + 0) * ncell] = d[0] * a + d[1] * c;
    Jb[(int64_t)(4 * q + 1) * ncell] = d[0] * b + d[1] * e;
    Jb[(int64_t)(4 * q + 2) * ncell] = d[2] * a + d[3] * c;
    Jb[(int64_t)(4 * q + 3) * ncell] = d[2] * b + d[3] * e;
  }
}

// ---------------------------------------------------------------------------
// set-up kernels (once per solve)
// ---------------------------------------------------------------------------

// Random fields at cell centres (field_at: the configs' smooth fields, or
// the paper's Eq. poro_2levels; see henry.h for the formulas) and the
// inflow per row.
static __global__ void k_fields(unsigned long long* ctr, Phys P, Geom G, int B, int n_xi, int model,
                         const double* __restrict__ xi, const double* __restrict__ logk,
                         double* __restrict__ phi, double* __restrict__ K, double* __restrict__ qin,
                         int* __restrict__ status) {
  HENRY_COUNT_LAUNCH(ctr);
  const int64_t n = (int64_t)B * G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int b = (int)(idx / G.ncell());
  const int cell = (int)(idx - (int64_t)b * G.ncell());
  const int j = cell / G.nx, i = cell - j * G.nx;
  const double x = (i + 0.5) * G.hx, y = (j + 0.5) * G.hy;
  const double* z = xi + (int64_t)b * n_xi;
  double ph, k;
  field_at(P, model, n_xi, z, x, y, logk != nullptr, logk ? logk[idx] : 0.0, ph, k);
  phi[idx] = ph;
  K[idx] = k;
  if (i == 0) qin[(int64_t)b * G.ny + j] = inflow_at(P, model, n_xi, z, y);
  if (cell == 0) {
    bool ok = true;
    for (int m = 0; m < n_xi; ++m) ok = ok && isfinite(z[m]);
    status[b] = ok ? 0 : kStatusBadInput;
  }
}

// Coarse-grid fields for the rediscretised multigrid operators: arithmetic
// mean of the four children.
static __global__ void k_coarsen_fields(unsigned long long* ctr, Geom Gf, Geom Gc, int B,
                                 const double* __restrict__ phif, const double* __restrict__ Kf,
                                 double* __restrict__ phic, double* __restrict__ Kc) {
  HENRY_COUNT_LAUNCH(ctr);
  const int64_t n = (int64_t)B * Gc.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int b = (int)(idx / Gc.ncell());
  const int cell = (int)(idx - (int64_t)b * Gc.ncell());
  const int J = cell / Gc.nx, I = cell - J * Gc.nx;
  const int64_t f0 = (int64_t)b * Gf.ncell() + (2 * J) * Gf.nx + 2 * I;
  phic[idx] = 0.25 * (phif[f0] + phif[f0 + 1] + phif[f0 + Gf.nx] + phif[f0 + Gf.nx + 1]);
  Kc[idx] = 0.25 * (Kf[f0] + Kf[f0 + 1] + Kf[f0 + Gf.nx] + Kf[f0 + Gf.nx + 1]);
}

static __global__ void k_face_consts(unsigned long long* ctr, Phys P, Geom G, int B,
                              const double* __restrict__ phi, const double* __restrict__ K,
                              double* __restrict__ tx, double* __restrict__ dx,
                              double* __restrict__ ty, double* __restrict__ dy) {
  HENRY_COUNT_LAUNCH(ctr);
  const int64_t n = (int64_t)B * G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int b = (int)(idx / G.ncell());
  const int cell = (int)(idx - (int64_t)b * G.ncell());
  const int j = cell / G.nx, i = cell - j * G.nx;
  const int64_t o = (int64_t)b * G.ncell();
  face_constants(P, G, i, j, phi + o, K + o, tx[idx], dx[idx], ty[idx], dy[idx]);
}

// Initial state c = 0; the Newton guess for p is seawater hydrostatics,
// stored as the reduced pressure p' = p - rho0 g (Ly - y).
static __global__ void k_init_state(unsigned long long* ctr, Phys P, Geom G, int B, double* __restrict__ p,
                             double* __restrict__ c, int* __restrict__ iters,
                             int* __restrict__ step) {
  HENRY_COUNT_LAUNCH(ctr);
  const int64_t n = (int64_t)B * G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int b = (int)(idx / G.ncell());
  const int cell = (int)(idx - (int64_t)b * G.ncell());
  const int j = cell / G.nx;
  const double y = (j + 0.5) * G.hy;
  p[idx] = P.drho * P.g * (P.Ly - y);
  c[idx] = 0.0;
  if (cell == 0) iters[b] = 0;
  if (idx == 0) *step = 0;
}

// ---------------------------------------------------------------------------
// per time step
// ---------------------------------------------------------------------------
// Start of an implicit Euler step: c_old = c^{n-1} (with mo / so given, also
// the old-time storage terms of k_resid). With `extrapolate`, from
// the third step on (both u^{n-1} and u^{n-2} are solutions; the first
// step's pressure guess is not) the Newton initial guess is extrapolated
// linearly in time, u = 2 u^{n-1} - u^{n-2}, with c clamped to [0, 1]
// (p_prev keeps p^{n-2}, c_old c^{n-2} on entry). `step` counts completed
// steps (k_end_step increments it).
template <int D = 0>   // history arrays in use (hx.depth)
static __global__ void k_begin_step(unsigned long long* ctr, Geom G, int B, double* __restrict__ p,
                             double* __restrict__ c, double* __restrict__ p_prev,
                             double* __restrict__ c_old, const int* __restrict__ status,
                             int* __restrict__ active, int* __restrict__ it_step,
                             const int* __restrict__ step, int extrapolate,
                             const double* __restrict__ qin0, double* __restrict__ qin,
                             double tau, const double* __restrict__ phi = nullptr,
                             double vtau = 0.0, double rho0 = 0.0, double drho = 0.0,
                             double* __restrict__ mo = nullptr, double* __restrict__ so = nullptr,
                             double* __restrict__ vt_out = nullptr, GuessHist hx = {}) {
  HENRY_COUNT_LAUNCH(ctr);
  const int64_t n = (int64_t)B * G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  if (qin0 && idx < (int64_t)B * G.ny) {
    // Eq. e_recharge_of_param: inflow times (1 + sin(pi t / 40)), t in
    // seconds at the new time level t^(n+1) of this implicit step
    const double pi = 3.14159265358979323846;
    const double t = (*step + 1) * tau;
    qin[idx] = qin0[idx] * (1.0 + sin(pi * t / 40.0));
  }
  // Newton's initial guess for u^(n+1): the polynomial extrapolation in time
  // of order q through u^n, u^(n-1), ..., u^(n-q), i.e.
  //   u^(n+1) ~ sum_k (-1)^k C(q+1, k+1) u^(n-k)   (q = 1: 2u^n - u^(n-1)),
  // with q = min(extrapolate, step - 1, 1 + hx.depth): the initial state u^0
  // (before the first step's transient) is never used; c clamped to [0, 1].
  // c_old / p_prev hold u^(n-1) on entry and u^n (the old time level of this
  // step) on exit; hx holds u^(n-2) ... and is shifted by one step.
  const double cn = c[idx], pn = p[idx];
  double hc[1 + D], hp[1 + D];
  hc[0] = c_old[idx];
  hp[0] = p_prev[idx];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    hc[k + 1] = hx.c[k][idx];
    hp[k + 1] = hx.p[k][idx];
  }
  int q = extrapolate;
  if (q > *step - 1) q = *step - 1;
  if (q > 1 + D) q = 1 + D;
  if (q >= 1) {
    double w = q + 1.0;                 // C(q+1, 1)
    double ec = w * cn, ep = w * pn;
#pragma unroll
    for (int k = 1; k <= 1 + D; ++k) {
      if (k > q) break;
      w = -w * (q + 1 - k) / (k + 1);   // (-1)^k C(q+1, k+1)
      ec += w * hc[k - 1];
      ep += w * hp[k - 1];
    }
    c[idx] = fmin(fmax(ec, 0.0), 1.0);
    p[idx] = ep;
  }
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    hx.c[k][idx] = hc[k];
    hx.p[k][idx] = hp[k];
  }
  c_old[idx] = cn;
  p_prev[idx] = pn;
  if (mo) {
    // storage of the old time level, fixed for the whole step: (V phi / tau)
    // rho(c_old) and (V phi / tau) rho(c_old) c_old (k_resid)
    const double vt = vtau * phi[idx];
    const double m = vt * (rho0 + drho * cn);
    mo[idx] = m;
    so[idx] = m * cn;
    vt_out[idx] = vt;
  }
  const int b = (int)(idx / G.ncell());
  if (idx - (int64_t)b * G.ncell() == 0) {
    active[b] = (status[b] & (kStatusNonfinite | kStatusBadInput | kStatusStall)) ? 0 : 1;
    it_step[b] = 0;
  }
}

// Condition of the operator-rebuild block of a defect-correction iteration
// (graph loop with operator reuse): true when some sample asked for new
// operators (count published by k_check). When none did, the rebuild
// kernels, which would all skip every sample, are not launched.
static __global__ void k_set_rebuild(unsigned long long* ctr, const int* __restrict__ n_refresh,
                              cudaGraphConditionalHandle h) {
  HENRY_COUNT_LAUNCH(ctr);
  if (threadIdx.x == 0) cudaGraphSetConditional(h, *n_refresh > 0 ? 1u : 0u);
}

static __global__ void k_end_step(unsigned long long* ctr, int* __restrict__ step) {
  HENRY_COUNT_LAUNCH(ctr);
  if (threadIdx.x == 0) *step += 1;
}

// FP64 residual of the finest grid and its Jacobian in the multigrid type T,
// face by face. Tiling: a block covers TX columns x (GR * R) rows of one
// sample; thread t takes column t % TX and walks R rows of row group t / TX.
// Per cell the thread evaluates its east and north faces only: the west
// face comes from the left neighbour thread through shared memory (or is
// evaluated again at a tile edge) and the south face is the north face of
// the previous row, kept in registers (evaluated once per column at the
// bottom of a row group). Each face is evaluated with the canonical
// orientation, so both cells see bitwise the same flux.
// MG layout (NATURAL = false): writes b = -R, x = 0, J (colour-split), the
// face fluxes qx (east / right side) and qy (north), one partial sum of
// R_p^2 + R_c^2 per block. NATURAL = true: writes R [B][2][ncell] and J
// [B][20][ncell] in natural cell order (FP64), for tests. WANT_J = false:
// the residual outputs only (defect-correction iterations that reuse the
// operators). refresh (optional, per sample): samples with refresh[b] == 0
// are skipped.
template <typename T, bool NATURAL, bool WANT_J = true>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 8 ? 2 : 3)
k_resjac(unsigned long long* ctr, Phys P, Geom G, double vtau, int B, ResTile tl,
         const double* __restrict__ p, const double* __restrict__ c,
         const double* __restrict__ c_old, const double* __restrict__ phi,
         const double* __restrict__ K, const double* __restrict__ tx,
         const double* __restrict__ dx, const double* __restrict__ ty,
         const double* __restrict__ dy, const double* __restrict__ qin,
         const int* __restrict__ active, T* __restrict__ J, T* __restrict__ bvec,
         T* __restrict__ xvec, double* __restrict__ partial, double* __restrict__ qx,
         double* __restrict__ qy, const int* __restrict__ refresh) {
  HENRY_COUNT_LAUNCH(ctr);
  __shared__ double shF[2][kBlock];
  __shared__ T shD[8][kBlock];   // face derivatives (unused, and removed, when !WANT_J)
  __shared__ double shr[kBlock / 32];
  const int b = blockIdx.y;
  if (!NATURAL && (!active[b] || (refresh && !refresh[b]))) return;
  const int nx = G.nx, ny = G.ny, ncell = G.ncell(), half = G.half();
  const int t = threadIdx.x;
  const int col = t % tl.TX, rg = t / tl.TX;
  const int bx = blockIdx.x % tl.ntx, by = blockIdx.x / tl.ntx;
  const int i = bx * tl.TX + col;
  const int j0 = by * tl.GR * tl.R + rg * tl.R;
  const bool thr = rg < tl.GR && i < nx;
  const int64_t o = (int64_t)b * ncell;
  const double* pb_ = p + o;
  const double* cb_ = c + o;
  const double gdy = P.g * G.hy;
  const double A = G.hy;
  const double dcoL = 2.0 * A * P.D / G.hx;      // times phi_P
  const double tRf = 2.0 * A / (P.mu * G.hx);    // times K_P
  double v = 0.0;
  // south face of the first row (halo), as L = S, U = P
  double FmS = 0.0, FsS = 0.0;
  FaceD<T> dS;
  double pP = 0.0, cP = 0.0;
  if (thr && j0 < ny) {
    pP = pb_[j0 * nx + i];
    cP = cb_[j0 * nx + i];
    if (j0 > 0) {
      const int id = (j0 - 1) * nx + i;
      double q;
      face_flux<T, WANT_J, false, true>(P, pb_[id], cb_[id], pP, cP, ty[o + id], dy[o + id], gdy, q,
                                        FmS, FsS, dS);
    }
  }
  for (int r = 0; r < tl.R; ++r) {
    const int j = j0 + r;
    const bool cv = thr && j < ny;
    const int id = j * nx + i;
    double FmE = 0.0, FsE = 0.0, qE = 0.0;
    FaceD<T> dE;
    T dR[4];   // right side derivatives (dF/du_P)
    double phiP = 0.0, pN = 0.0, cN = 0.0;
    if (cv) {
      phiP = phi[o + id];
      if (i < nx - 1) {
        face_flux<T, WANT_J, false, false>(P, pP, cP, pb_[id + 1], cb_[id + 1], tx[o + id],
                                           dx[o + id], 0.0, qE, FmE, FsE, dE);
      } else {
        const double pbd = P.drho * P.g * (P.Ly - (j + 0.5) * G.hy);
        right_face<T, WANT_J, false>(P, pP, cP, tRf * K[o + id], dcoL * phiP, pbd, qE, FmE, FsE, dR);
      }
      shF[0][t] = FmE;
      shF[1][t] = FsE;
      if (WANT_J) {
        shD[0][t] = dE.mLp; shD[1][t] = dE.mLc; shD[2][t] = dE.mUp; shD[3][t] = dE.mUc;
        shD[4][t] = dE.sLp; shD[5][t] = dE.sLc; shD[6][t] = dE.sUp; shD[7][t] = dE.sUc;
      }
    }
    __syncthreads();
    if (cv) {
      // west face (L = W, U = P)
      double FmW = 0.0, FsW = 0.0;
      FaceD<T> dW;
      if (i > 0) {
        if (col > 0) {
          FmW = shF[0][t - 1];
          FsW = shF[1][t - 1];
          if (WANT_J) {
            dW.mLp = shD[0][t - 1]; dW.mLc = shD[1][t - 1]; dW.mUp = shD[2][t - 1]; dW.mUc = shD[3][t - 1];
            dW.sLp = shD[4][t - 1]; dW.sLc = shD[5][t - 1]; dW.sUp = shD[6][t - 1]; dW.sUc = shD[7][t - 1];
          }
        } else {
          double q;
          face_flux<T, WANT_J, false, false>(P, pb_[id - 1], cb_[id - 1], pP, cP, tx[o + id - 1],
                                             dx[o + id - 1], 0.0, q, FmW, FsW, dW);
        }
      }
      // north face (L = P, U = N)
      double FmN = 0.0, FsN = 0.0, qN = 0.0;
      FaceD<T> dN;
      if (j < ny - 1) {
        pN = pb_[id + nx];
        cN = cb_[id + nx];
        face_flux<T, WANT_J, false, true>(P, pP, cP, pN, cN, ty[o + id], dy[o + id], gdy, qN, FmN,
                                          FsN, dN);
      }
      // accumulation
      const double vt = vtau * phiP;
      const double rho = P.rho0 + P.drho * cP;
      const double cO = c_old[o + id];
      const double rho_o = P.rho0 + P.drho * cO;
      double Rp = vt * (rho - rho_o) + FmE + FmN - FmW - FmS;
      double Rc = vt * (rho * cP - rho_o * cO) + FsE + FsN - FsW - FsS;
      T Jc[20];
#pragma unroll
      for (int m = 0; m < 20; ++m) Jc[m] = (T)0;
      Jc[1] = (T)(vt * P.drho);
      Jc[3] = (T)(vt * (rho + P.drho * cP));
      if (i > 0) {
        Jc[0] -= dW.mUp; Jc[1] -= dW.mUc; Jc[2] -= dW.sUp; Jc[3] -= dW.sUc;
        Jc[4] = -dW.mLp; Jc[5] = -dW.mLc; Jc[6] = -dW.sLp; Jc[7] = -dW.sLc;
      } else {
        // left side: fixed freshwater inflow, diffusion to c = 0 at hx/2
        const double dco = dcoL * phiP;
        const double rb = 0.5 * (rho + P.rho0);
        Rp += -A * P.rho0 * qin[(int64_t)b * ny + j];
        Rc += dco * rb * cP;
        if (WANT_J) Jc[3] += (T)(dco * (0.5 * P.drho * cP + rb));
      }
      if (i < nx - 1) {
        Jc[0] += dE.mLp; Jc[1] += dE.mLc; Jc[2] += dE.sLp; Jc[3] += dE.sLc;
        Jc[8] = dE.mUp; Jc[9] = dE.mUc; Jc[10] = dE.sUp; Jc[11] = dE.sUc;
      } else {
        Jc[0] += dR[0]; Jc[1] += dR[1]; Jc[2] += dR[2]; Jc[3] += dR[3];
      }
      if (j > 0) {
        Jc[0] -= dS.mUp; Jc[1] -= dS.mUc; Jc[2] -= dS.sUp; Jc[3] -= dS.sUc;
        Jc[12] = -dS.mLp; Jc[13] = -dS.mLc; Jc[14] = -dS.sLp; Jc[15] = -dS.sLc;
      }
      if (j < ny - 1) {
        Jc[0] += dN.mLp; Jc[1] += dN.mLc; Jc[2] += dN.sLp; Jc[3] += dN.sLc;
        Jc[16] = dN.mUp; Jc[17] = dN.mUc; Jc[18] = dN.sUp; Jc[19] = dN.sUc;
      }
      if (NATURAL) {
        double* Rn = (double*)bvec + (int64_t)b * 2 * ncell;
        Rn[id] = Rp;
        Rn[ncell + id] = Rc;
        if (WANT_J && J) {
          T* Jn = J + (int64_t)b * 20 * ncell + id;
#pragma unroll
          for (int m = 0; m < 20; ++m) Jn[(int64_t)m * ncell] = Jc[m];
        }
      } else {
        const int cs = cs_pos(i, j, nx, half);
        const int64_t ob = (int64_t)b * 2 * ncell;
        T* Jb = J + (int64_t)b * kJP * ncell + cs;
        T d[4];   // Dinv of the operator the multigrid will use
        if (WANT_J) {
          store_operator<T>(Jb, ncell, Jc, d);
        } else {
#pragma unroll
          for (int m = 0; m < 4; ++m) d[m] = Jb[(int64_t)m * ncell];
        }
        const T mp = (T)(-Rp), mc = (T)(-Rc);
        bvec[ob + cs] = d[0] * mp + d[1] * mc;
        bvec[ob + ncell + cs] = d[2] * mp + d[3] * mc;
        xvec[ob + cs] = (T)0;
        xvec[ob + ncell + cs] = (T)0;
        qx[o + id] = qE;
        qy[o + id] = qN;
      }
      v += Rp * Rp + Rc * Rc;
      // the north face is the next row's south face
      FmS = FmN;
      FsS = FsN;
      dS = dN;
      pP = pN;
      cP = cN;
    }
    __syncthreads();
  }
  if (!NATURAL) {
    const double s = block_sum(v, shr);
    if (threadIdx.x == 0) partial[(int64_t)b * gridDim.x + blockIdx.x] = s;
  }
}

// FP64 residual of the finest grid alone, for the defect-correction
// iterations that keep their operators (operator reuse): the same discrete
// residual as k_resjac, arranged for GB300's narrow FP64 pipe, where every
// FP64 warp instruction costs the same pipe time whether one lane or 32
// are active (so the kernel avoids divergent FP64 work):
//  * per-cell constants: vt = V phi / tau and the old-time storage terms
//    mo = vt rho(c_old), so = mo c_old from k_begin_step, so the storage part
//    is a = vt rho, R_p = a - mo, R_c = a c - so;
//  * rho and rho c of a cell are formed once: the east neighbour's come from
//    the next lane (shuffle), the north neighbour's become the next row's;
//  * the west face is the east face of the previous lane; across a warp
//    edge both the neighbour's state and the face travel through shared
//    memory (two block barriers per row); only tile edges recompute;
//  * the right side is one more face, to the Dirichlet values (p_b, c = 1),
//    with the coefficients face_constants keeps in the last column;
//  * a face's mean density and its gravity term share c_L + c_U.
// Writes b = -Dinv R with the stored Dinv, x = 0, the face fluxes qx, qy
// and one partial sum of R_p^2 + R_c^2 per block; same tiling as k_resjac.
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_resid(unsigned long long* ctr, Phys P, Geom G, int B, ResTile tl,
        const double* __restrict__ p, const double* __restrict__ c,
        const double* __restrict__ vt, const double* __restrict__ mo,
        const double* __restrict__ so, const double* __restrict__ phi,
        const double* __restrict__ tx, const double* __restrict__ dx,
        const double* __restrict__ ty, const double* __restrict__ dy,
        const double* __restrict__ qin, const int* __restrict__ active, const T* __restrict__ J,
        T* __restrict__ bvec, T* __restrict__ xvec, double* __restrict__ partial,
        double* __restrict__ qx, double* __restrict__ qy) {
  HENRY_COUNT_LAUNCH(ctr);
  constexpr int kW = kBlock / 32;
  __shared__ double shS[4][kW];    // lane 0's p, c, rho, rho c for the previous warp's lane 31
  __shared__ double shF[2][kW];    // lane 31's east-face fluxes for the next warp's lane 0
  __shared__ double shr[kW];
  const int b = blockIdx.y;
  if (!active[b]) return;
  const int nx = G.nx, ny = G.ny, ncell = G.ncell(), half = G.half();
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int col = t % tl.TX, rg = t / tl.TX;
  const int bx = blockIdx.x % tl.ntx, by = blockIdx.x / tl.ntx;
  const int i = bx * tl.TX + col;
  const int j0 = by * tl.GR * tl.R + rg * tl.R;
  const bool thr = rg < tl.GR && i < nx;
  // where the east neighbour's state and the west face come from
  const bool east_in = thr && col < tl.TX - 1 && i < nx - 1;   // a thread of this tile
  const bool east_lane = east_in && lane < 31;
  const bool east_smem = east_in && lane == 31;
  const bool east_load = thr && col == tl.TX - 1 && i < nx - 1;  // tile edge
  const bool west_in = thr && col > 0;
  const bool west_lane = west_in && lane > 0;
  const bool west_smem = west_in && lane == 0;
  const bool west_load = thr && col == 0 && i > 0;               // tile edge
  const int64_t o = (int64_t)b * ncell;
  const double* pb_ = p + o;
  const double* cb_ = c + o;
  const double hd = 0.5 * P.drho;              // rho_bar = rho0 + hd (c_L + c_U)
  const double hdg = hd * P.g * G.hy;          // gravity term of a vertical face: hdg (c_L + c_U)
  // one face L -> U: mass and salt flux from both sides' p, c, rho, rho c
  auto face = [&](double pL, double cL, double rL, double rcL, double pU, double cU, double rU,
                  double rcU, double tf, double dco, bool vert, double& q, double& Fm,
                  double& Fs) {
    const double sc = cL + cU;
    const double rbar = fma(hd, sc, P.rho0);
    const double dp = pU - pL;
    q = -tf * (vert ? fma(hdg, sc, dp) : dp);
    const bool up = q >= 0.0;
    Fm = q * (up ? rL : rU);
    Fs = fma(q, up ? rcL : rcU, -(dco * rbar) * (cU - cL));
  };
  double v = 0.0;
  double pP = 0.0, cP = 0.0, rP = 0.0, rcP = 0.0, FmS = 0.0, FsS = 0.0;
  if (thr && j0 < ny) {
    pP = pb_[j0 * nx + i];
    cP = cb_[j0 * nx + i];
  }
  rP = fma(P.drho, cP, P.rho0);
  rcP = rP * cP;
  if (thr && j0 < ny && j0 > 0) {   // south face of the first row (every thread of a row group)
    const int id = (j0 - 1) * nx + i;
    const double pS = pb_[id], cS = cb_[id];
    const double rS = fma(P.drho, cS, P.rho0);
    double q;
    face(pS, cS, rS, rS * cS, pP, cP, rP, rcP, ty[o + id], dy[o + id], true, q, FmS, FsS);
  }
  for (int r = 0; r < tl.R; ++r) {
    const int j = j0 + r;
    const bool cv = thr && j < ny;
    const int id = j * nx + i;
    // east neighbour: the next lane's state, across a warp edge through
    // shared memory, at a tile edge from memory, at the right side the
    // seawater values
    if (lane == 0) { shS[0][w] = pP; shS[1][w] = cP; shS[2][w] = rP; shS[3][w] = rcP; }
    double pE = __shfl_down_sync(0xffffffffu, pP, 1);
    double cE = __shfl_down_sync(0xffffffffu, cP, 1);
    double rE = __shfl_down_sync(0xffffffffu, rP, 1);
    double rcE = __shfl_down_sync(0xffffffffu, rcP, 1);
    __syncthreads();
    if (east_smem) { pE = shS[0][w + 1]; cE = shS[1][w + 1]; rE = shS[2][w + 1]; rcE = shS[3][w + 1]; }
    if (!east_lane && !east_smem) {
      if (east_load && cv) {
        pE = pb_[id + 1];
        cE = cb_[id + 1];
      } else {   // the right side: reduced seawater pressure at this row, c = 1
        pE = P.drho * P.g * (P.Ly - (j + 0.5) * G.hy);
        cE = 1.0;
      }
      rE = fma(P.drho, cE, P.rho0);
      rcE = rE * cE;
    }
    double FmE = 0.0, FsE = 0.0, qE = 0.0;
    if (cv) face(pP, cP, rP, rcP, pE, cE, rE, rcE, tx[o + id], dx[o + id], false, qE, FmE, FsE);
    // west face: the previous lane's east face (across a warp edge through
    // shared memory; recomputed at a tile edge)
    if (lane == 31) { shF[0][w] = FmE; shF[1][w] = FsE; }
    double FmW = __shfl_up_sync(0xffffffffu, FmE, 1);
    double FsW = __shfl_up_sync(0xffffffffu, FsE, 1);
    __syncthreads();
    if (west_smem) { FmW = shF[0][w - 1]; FsW = shF[1][w - 1]; }
    if (!west_in) { FmW = 0.0; FsW = 0.0; }
    if (west_load && cv) {
      const double pW = pb_[id - 1], cW = cb_[id - 1];
      const double rW = fma(P.drho, cW, P.rho0);
      double q;
      face(pW, cW, rW, rW * cW, pP, cP, rP, rcP, tx[o + id - 1], dx[o + id - 1], false, q, FmW,
           FsW);
    }
    double pN = 0.0, cN = 0.0;
    double FmN = 0.0, FsN = 0.0, qN = 0.0;
    if (cv && j < ny - 1) {
      pN = pb_[id + nx];
      cN = cb_[id + nx];
    }
    const double rN = fma(P.drho, cN, P.rho0);
    const double rcN = rN * cN;
    if (cv && j < ny - 1) face(pP, cP, rP, rcP, pN, cN, rN, rcN, ty[o + id], dy[o + id], true, qN, FmN, FsN);
    if (cv) {
      const double a = vt[o + id] * rP;
      double Rp = (a - mo[o + id]) + FmE + FmN - FmW - FmS;
      double Rc = fma(a, cP, -so[o + id]) + FsE + FsN - FsW - FsS;
      if (i == 0) {   // left side: fresh-water inflow, diffusion to c = 0 at hx/2
        Rp += -G.hy * P.rho0 * qin[(int64_t)b * ny + j];
        Rc += ((2.0 * G.hy * P.D / G.hx) * phi[o + id]) * (0.5 * (rP + P.rho0)) * cP;
      }
      const int cs = cs_pos(i, j, nx, half);
      const int64_t ob = (int64_t)b * 2 * ncell;
      const T* Jb = J + (int64_t)b * kJP * ncell + cs;
      const T mp = (T)(-Rp), mc = (T)(-Rc);
      bvec[ob + cs] = Jb[0] * mp + Jb[(int64_t)ncell] * mc;
      bvec[ob + ncell + cs] = Jb[(int64_t)2 * ncell] * mp + Jb[(int64_t)3 * ncell] * mc;
      xvec[ob + cs] = (T)0;
      xvec[ob + ncell + cs] = (T)0;
      qx[o + id] = qE;
      qy[o + id] = qN;
      v = fma(Rp, Rp, fma(Rc, Rc, v));
    }
    FmS = FmN;
    FsS = FsN;
    pP = pN;
    cP = cN;
    rP = rN;
    rcP = rcN;
  }
  const double s = block_sum(v, shr);
  if (threadIdx.x == 0) partial[(int64_t)b * gridDim.x + blockIdx.x] = s;
}

// Per-sample convergence decision after k_resjac, one warp per sample:
// sums the sample's partials in a fixed order, scales the RMS residual to
// units of c per step, updates active / status / counters. A sample is
// converged when r <= max(rtol r0, atol), or when r <= max(stag_tol,
// stag_rel r0) and the last iteration reduced r by less than half (the
// residual has reached the FP64 rounding floor of the grid, which grows with
// resolution). Blocks add their
// count of still-active samples to acc[0]; the last block to finish
// (acc[1] counts finished blocks) publishes the total to *n_active, resets
// acc for the next launch and, when SET_COND, sets the while-loop condition
// of the enclosing CUDA graph. With refresh (operator reuse factor lag > 0)
// it also decides whether the next iteration rebuilds the Jacobian and the
// multigrid operators: after the step's initial residual (with *keep != 0
// only before the first iteration of the solve: the operators of the
// previous step are kept), later when the last iteration reduced the
// residual by less than a factor lag; acc[2] counts those samples and the
// last block publishes the count in n_active[1] (k_set_rebuild turns it
// into the condition of the rebuild).
template <bool SET_COND>
__global__ void k_check(unsigned long long* ctr, int B, int nchunk, int ncell,
                        const double* __restrict__ partial, double scale, double rtol,
                        double atol, int maxit, int* __restrict__ active,
                        int* __restrict__ it_step, double* __restrict__ res0,
                        double* __restrict__ res_last, int* __restrict__ status,
                        int* __restrict__ iters, int* __restrict__ n_active,
                        unsigned int* __restrict__ acc, double stag_tol,
                        cudaGraphConditionalHandle h, int* __restrict__ refresh, int lag,
                        double stag_rel = 0.0, const int* __restrict__ keep = nullptr) {
  HENRY_COUNT_LAUNCH(ctr);
  __shared__ int cnt, rcnt;
  __shared__ bool last;
  if (threadIdx.x == 0) cnt = rcnt = 0;
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + w;
  if (b < B && active[b]) {
    double s = 0.0;
    for (int k = l; k < nchunk; k += 32) s += partial[(int64_t)b * nchunk + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (l == 0) {
      const double r = sqrt(s / ncell) * scale;
      const int it = it_step[b];
      if (it == 0) res0[b] = r;
      const double prev = res_last[b];
      res_last[b] = r;
      if (!isfinite(r)) {
        status[b] |= kStatusNonfinite;
        active[b] = 0;
      } else if (r <= fmax(rtol * res0[b], atol) ||
                 (it > 0 && r <= fmax(stag_tol, stag_rel * res0[b]) && r > 0.5 * prev)) {
        active[b] = 0;
      } else if (it >= maxit) {
        status[b] |= kStatusMaxit;
        active[b] = 0;
      } else {
        const bool first = iters[b] == 0;   // no operators built yet in this solve
        it_step[b] = it + 1;
        iters[b] += 1;
        atomicAdd(&cnt, 1);
        if (refresh) {
          const bool kept = keep && *keep;
          const int rf = (it == 0 ? (!kept || first) : r * lag > prev) ? 1 : 0;
          refresh[b] = rf;
          if (rf) atomicAdd(&rcnt, 1);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (cnt) atomicAdd(&acc[0], (unsigned int)cnt);
    if (rcnt) atomicAdd(&acc[2], (unsigned int)rcnt);
    __threadfence();
    last = atomicAdd(&acc[1], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const unsigned int total = atomicExch(&acc[0], 0u);
    n_active[1] = (int)atomicExch(&acc[2], 0u);
    acc[1] = 0u;
    *n_active = (int)total;
    if (SET_COND) cudaGraphSetConditional(h, total > 0 ? 1u : 0u);
  }
}

// Linearisation point of level k-1 from level k: c averaged over the four
// children, face fluxes summed over the two fine faces that make up each
// coarse face (east faces of the right children, north faces of the top
// children; at the right side these are the boundary fluxes). Linearising
// every level about the same flux field keeps the upwind decisions of the
// coarse operators consistent with the finest one.
static __global__ void k_restrict_state(unsigned long long* ctr, Geom Gf, Geom Gc, int B,
                                 const int* __restrict__ active, const double* __restrict__ cf,
                                 const double* __restrict__ qxf, const double* __restrict__ qyf,
                                 double* __restrict__ cc, double* __restrict__ qxc,
                                 double* __restrict__ qyc, const int* __restrict__ refresh) {
  HENRY_COUNT_LAUNCH(ctr);
  const int64_t n = (int64_t)B * Gc.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int b = (int)(idx / Gc.ncell());
  if (!active[b] || (refresh && !refresh[b])) return;
  const int cell = (int)(idx - (int64_t)b * Gc.ncell());
  const int J = cell / Gc.nx, I = cell - J * Gc.nx;
  const int nx = Gf.nx;
  const int64_t f0 = (int64_t)b * Gf.ncell() + (2 * J) * nx + 2 * I;
  cc[idx] = 0.25 * (cf[f0] + cf[f0 + 1] + cf[f0 + nx] + cf[f0 + nx + 1]);
  qxc[idx] = qxf[f0 + 1] + qxf[f0 + nx + 1];
  qyc[idx] = qyf[f0 + nx] + qyf[f0 + nx + 1];
}

// Jacobian of a coarse multigrid level from its own state and fields.
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_jac(unsigned long long* ctr, Phys P, Geom G, double vtau, int B, const int* __restrict__ active,
      const double* __restrict__ p, const double* __restrict__ c, const double* __restrict__ phi,
      const double* __restrict__ K, const double* __restrict__ tx, const double* __restrict__ dx,
      const double* __restrict__ ty, const double* __restrict__ dy, const double* __restrict__ qx,
      const double* __restrict__ qy, T* __restrict__ J, const int* __restrict__ refresh) {
  HENRY_COUNT_LAUNCH(ctr);
  const int ncell = G.ncell();
  const int64_t n = (int64_t)B * ncell;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int b = (int)(idx / ncell);
  if (!active[b] || (refresh && !refresh[b])) return;
  const int cell = (int)(idx - (int64_t)b * ncell);
  const int j = cell / G.nx, i = cell - j * G.nx;
  const int64_t o = (int64_t)b * ncell;
  CellIn in;
  gather_cell(G, i, j, p + o, c + o, phi + o, K + o, tx + o, dx + o, ty + o, dy + o, in);
  in.c_old = in.c;
  in.qin = 0.0;
  const int id = cell;
  in.qE = qx[o + id];
  in.qN = in.hasN ? qy[o + id] : 0.0;
  in.qW = in.hasW ? qx[o + id - 1] : 0.0;
  in.qS = in.hasS ? qy[o + id - G.nx] : 0.0;
  double Rp, Rc;
  T Jc[20];
  cell_residual<T, true, true>(P, G, vtau, in, Rp, Rc, Jc);
  T* Jb = J + (int64_t)b * kJP * ncell + cs_pos(i, j, G.nx, G.half());
  T d[4];
  store_operator<T>(Jb, ncell, Jc, d);
}

// Explicit inverse of the coarsest system (the direct coarse solve of the
// multigrid, section 2.3), one block per sample: in-place Gauss-Jordan
// elimination with partial pivoting by rows. Per pivot k, three phases
// separated by barriers: warp 0 picks the pivot row and records the
// multipliers of column k, the pivot row is swapped in and divided by the
// pivot, and every other element is updated by its own thread. The column
// interchanges that undo the row pivots (last pivot first) are folded into
// the output index. Unknown order 2*cell + var, cell natural; the inverse is
// stored transposed, Ainv^T[v][u] at v*n + u, so that the coarse solve
// x = Ainv b reads it with lanes over u. The arithmetic is the multigrid
// type T (the coarse solve is part of the preconditioner): one n^3
// elimination per operator rebuild turns each coarse solve into one
// parallel matrix-vector product instead of 2n dependent substitution
// steps. Shared memory (dynamic): coarse_inv_smem_bytes<T>(n).
template <typename T>
__host__ __device__ inline size_t coarse_inv_smem_bytes(int n) {
  return ((size_t)n * (n + 1) + n + 2) * sizeof(T) + 2 * (size_t)n * sizeof(int);
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
k_coarse_inv(unsigned long long* ctr, Geom G, int B, const int* __restrict__ active,
             const T* __restrict__ J, T* __restrict__ AinvT, const int* __restrict__ refresh) {
  HENRY_COUNT_LAUNCH(ctr);
  extern __shared__ __align__(16) unsigned char inv_sh[];
  const int b = blockIdx.x;
  if (!active[b] || (refresh && !refresh[b])) return;
  const int nc = G.ncell(), n = 2 * nc, half = G.half(), ld = n + 1;
  T* A = (T*)inv_sh;
  T* fcol = A + n * ld;                 // multipliers of column k, after the swap
  T* rinv_sh = fcol + n;                // 1 / pivot
  int* pv = (int*)(rinv_sh + 2);        // pivot row of each step
  int* qcol = pv + n;                   // output column -> eliminated column
  const int l = threadIdx.x & 31;
  const T* Jb = J + (int64_t)b * kJP * nc;
  for (int e = threadIdx.x; e < n * ld; e += blockDim.x) A[e] = (T)0;
  __syncthreads();
  for (int cell = threadIdx.x; cell < nc; cell += blockDim.x) {
    const int j = cell / G.nx, i = cell - j * G.nx;
    const int cs = cs_pos(i, j, G.nx, half);
    const int nb[5] = {cell, i > 0 ? cell - 1 : -1, i < G.nx - 1 ? cell + 1 : -1,
                       j > 0 ? cell - G.nx : -1, j < G.ny - 1 ? cell + G.nx : -1};
    // the scaled system: identity diagonal blocks, At off the diagonal
    A[(2 * cell) * ld + 2 * cell] = (T)1;
    A[(2 * cell + 1) * ld + 2 * cell + 1] = (T)1;
    for (int q = 1; q < 5; ++q) {
      if (nb[q] < 0) continue;
      for (int e = 0; e < 2; ++e)
        for (int v = 0; v < 2; ++v)
          A[(2 * cell + e) * ld + 2 * nb[q] + v] = Jb[(int64_t)(4 * q + 2 * e + v) * nc + cs];
    }
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      // pivot: largest |A[r][k]|, r >= k, lowest index on ties
      T bv = (T)-1;
      int br = k;
      for (int r = k + l; r < n; r += 32) {
        const T v = fabs(A[r * ld + k]);
        if (v > bv) { bv = v; br = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int orr = __shfl_down_sync(0xffffffffu, br, o);
        if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
      }
      br = __shfl_sync(0xffffffffu, br, 0);
      // column k of the rows after the swap of rows k and br
      for (int r = l; r < n; r += 32) fcol[r] = r == k ? (T)0 : A[(r == br ? k : r) * ld + k];
      if (l == 0) {
        const T d = A[br * ld + k];
        pv[k] = br;
        rinv_sh[0] = d != (T)0 ? (T)1 / d : (T)0;
      }
    }
    __syncthreads();
    const int br = pv[k];
    const T rinv = rinv_sh[0];
    for (int col = threadIdx.x; col < n; col += blockDim.x) {
      // swap rows k and br; the new pivot row divided by the pivot, its own
      // column becoming 1 / pivot
      const T a = A[br * ld + col];
      if (br != k) A[br * ld + col] = A[k * ld + col];
      A[k * ld + col] = (col == k ? (T)1 : a) * rinv;
    }
    __syncthreads();
    // every other row: subtract f times the pivot row, its column k
    // becoming -f / pivot
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int row = e / n, col = e - row * n;
      if (row == k) continue;
      const T v = col == k ? (T)0 : A[row * ld + col];
      A[row * ld + col] = fma(-fcol[row], A[k * ld + col], v);
    }
    __syncthreads();
  }
  // column c of the inverse is column q(c) of the eliminated matrix, with
  // the interchanges (k, pv[k]) applied to c for k = 0, 1, ..., n-1
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    int x = c;
    for (int k = 0; k < n; ++k) x = x == k ? pv[k] : (x == pv[k] ? k : x);
    qcol[c] = x;
  }
  __syncthreads();
  T* out = AinvT + (int64_t)b * kMaxCoarseUnknowns * kMaxCoarseUnknowns;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int v = e / n, u = e - v * n;
    out[e] = A[u * ld + qcol[v]];
  }
}

// ---------------------------------------------------------------------------
// multigrid building blocks on one sample's arrays (J: [kJP][ncell], b, x:
// [2][ncell], colour-split planes). Used by the batched kernels below, with
// global-memory bases, and by k_vcycle_small, with shared-memory copies.
// ---------------------------------------------------------------------------

// Point-block Gauss-Seidel update of cell (i, j) on the row-scaled system:
// x_P = bt_P - sum_Q At_PQ x_Q (= D_P^{-1} (b_P - sum_Q A_PQ x_Q)). Jb points
// at the cell's colour-split position of plane 0 (planes ncell apart);
// nb(i', j', vp, vc) reads a neighbour's two unknowns, so that the batched,
// shared-memory and temporally blocked smoothers all perform the same
// operations in the same order (their results are bitwise equal). Each
// product is subtracted on its own so that it compiles to one FMA (the FP64
// form of the smoother is bound by GB300's FP64 pipe).
template <typename T, int P0 = 0, typename NB>
__device__ __forceinline__ void gs_point(int i, int j, int nx, int ny, int ncell,
                                         const T* __restrict__ Jb, T bp, T bc, NB nb, T& xp,
                                         T& xc) {
  // Jb points at plane P0 (a copy that starts at plane P0 > 0, e.g. in
  // shared memory); plane q is at (q - P0) * ncell
  T rp = bp, rc = bc;
  T vp, vc;
  if (i > 0) {
    nb(i - 1, j, vp, vc);
    rp -= Jb[(4 - P0) * ncell] * vp;
    rp -= Jb[(5 - P0) * ncell] * vc;
    rc -= Jb[(6 - P0) * ncell] * vp;
    rc -= Jb[(7 - P0) * ncell] * vc;
  }
  if (i < nx - 1) {
    nb(i + 1, j, vp, vc);
    rp -= Jb[(8 - P0) * ncell] * vp;
    rp -= Jb[(9 - P0) * ncell] * vc;
    rc -= Jb[(10 - P0) * ncell] * vp;
    rc -= Jb[(11 - P0) * ncell] * vc;
  }
  if (j > 0) {
    nb(i, j - 1, vp, vc);
    rp -= Jb[(12 - P0) * ncell] * vp;
    rp -= Jb[(13 - P0) * ncell] * vc;
    rc -= Jb[(14 - P0) * ncell] * vp;
    rc -= Jb[(15 - P0) * ncell] * vc;
  }
  if (j < ny - 1) {
    nb(i, j + 1, vp, vc);
    rp -= Jb[(16 - P0) * ncell] * vp;
    rp -= Jb[(17 - P0) * ncell] * vc;
    rc -= Jb[(18 - P0) * ncell] * vp;
    rc -= Jb[(19 - P0) * ncell] * vc;
  }
  xp = rp;
  xc = rc;
}

// Unscaled residual b - A x at cell (i, j) from the row-scaled system:
// D_P (bt_P - x_P - sum_Q At_PQ x_Q); Jc, nb as in gs_point, (x0p, x0c) the
// cell's own unknowns.
template <typename T, int P0 = 0, typename NB>
__device__ __forceinline__ void resid_point(int i, int j, int nx, int ny, int ncell,
                                            const T* __restrict__ Jc, T bp, T bc, T x0p, T x0c,
                                            NB nb, T& rp, T& rc) {
  rp = bp - x0p;
  rc = bc - x0c;
  T vp, vc;
  if (i > 0) {
    nb(i - 1, j, vp, vc);
    rp -= Jc[(4 - P0) * ncell] * vp;
    rp -= Jc[(5 - P0) * ncell] * vc;
    rc -= Jc[(6 - P0) * ncell] * vp;
    rc -= Jc[(7 - P0) * ncell] * vc;
  }
  if (i < nx - 1) {
    nb(i + 1, j, vp, vc);
    rp -= Jc[(8 - P0) * ncell] * vp;
    rp -= Jc[(9 - P0) * ncell] * vc;
    rc -= Jc[(10 - P0) * ncell] * vp;
    rc -= Jc[(11 - P0) * ncell] * vc;
  }
  if (j > 0) {
    nb(i, j - 1, vp, vc);
    rp -= Jc[(12 - P0) * ncell] * vp;
    rp -= Jc[(13 - P0) * ncell] * vc;
    rc -= Jc[(14 - P0) * ncell] * vp;
    rc -= Jc[(15 - P0) * ncell] * vc;
  }
  if (j < ny - 1) {
    nb(i, j + 1, vp, vc);
    rp -= Jc[(16 - P0) * ncell] * vp;
    rp -= Jc[(17 - P0) * ncell] * vc;
    rc -= Jc[(18 - P0) * ncell] * vp;
    rc -= Jc[(19 - P0) * ncell] * vc;
  }
  const T sp = rp, sc = rc;
  rp = Jc[(20 - P0) * ncell] * sp + Jc[(21 - P0) * ncell] * sc;
  rc = Jc[(22 - P0) * ncell] * sp + Jc[(23 - P0) * ncell] * sc;
}

// Reader of a sample's unknowns in the colour-split layout.
template <typename T>
struct CsReader {
  const T* x;
  int ncell, hx2, half, nx;
  __device__ __forceinline__ void operator()(int i, int j, T& vp, T& vc) const {
    const int q = cs_pos(i, j, nx, half);
    vp = x[q];
    vc = x[ncell + q];
  }
};

// Point-block Gauss-Seidel update of the cell at colour-split position
// `pos` of colour `colour` on one sample's arrays (colour-split layout; J
// from plane P0 on).
template <typename T, int P0 = 0>
__device__ __forceinline__ void smooth_cell(const Geom& G, int colour, int pos,
                                            const T* __restrict__ J, const T* __restrict__ b,
                                            T* __restrict__ x) {
  const int half = G.half(), ncell = G.ncell(), hx2 = G.nx >> 1;
  const int j = pos / hx2, k = pos - j * hx2;
  const int i = 2 * k + ((j + colour) & 1);
  const int own = colour * half + pos;
  const T* xo = x + (1 - colour) * half;   // the other colour's half of each plane
  T xp, xc;
  gs_point<T, P0>(i, j, G.nx, G.ny, ncell, J + own, b[own], b[ncell + own],
              [&](int ii, int jj, T& vp, T& vc) {
                const int q = jj * hx2 + (ii >> 1);
                vp = xo[q];
                vc = xo[ncell + q];
              },
              xp, xc);
  x[own] = xp;
  x[ncell + own] = xc;
}

// Unscaled residual b - A x at cell (i, j) (colour-split layout; Jb from
// plane P0 on).
template <typename T, int P0 = 0>
__device__ __forceinline__ void residual_cell(const Geom& G, int i, int j, const T* __restrict__ Jb,
                                              const T* __restrict__ b, const T* __restrict__ x,
                                              T& rp, T& rc) {
  const int ncell = G.ncell(), half = G.half(), nx = G.nx;
  const int cs = cs_pos(i, j, nx, half);
  resid_point<T, P0>(i, j, nx, G.ny, ncell, Jb + cs, b[cs], b[ncell + cs], x[cs], x[ncell + cs],
                 CsReader<T>{x, ncell, nx >> 1, half, nx}, rp, rc);
}

// Coarse cell `cell` of level k-1: b_c = sum over the four children of
// (b - A x) on level k (finite-volume restriction), stored scaled by the
// coarse Dinv (planes 0..3 of Jc), x_c = 0. red_only: the last operation on
// level k was a black half-sweep, which leaves the residual of every black
// cell zero up to rounding, so only the two red children (i + j even) are
// evaluated.
template <typename T, int P0 = 0>
__device__ __forceinline__ void restrict_cell(const Geom& Gf, const Geom& Gc, int cell,
                                              const T* __restrict__ Jf, const T* __restrict__ bf,
                                              const T* __restrict__ xf, const T* __restrict__ Jc,
                                              T* __restrict__ bc, T* __restrict__ xc,
                                              bool red_only) {
  const int J = cell / Gc.nx, I = cell - J * Gc.nx;
  const int ncc = Gc.ncell();
  T sp = 0, sc = 0;
#pragma unroll
  for (int c4 = 0; c4 < 4; ++c4) {
    if (red_only && (c4 == 1 || c4 == 2)) continue;
    const int i = 2 * I + (c4 & 1), j = 2 * J + (c4 >> 1);
    T rp, rc;
    residual_cell<T, P0>(Gf, i, j, Jf, bf, xf, rp, rc);
    sp += rp;
    sc += rc;
  }
  const int csc = cs_pos(I, J, Gc.nx, Gc.half());
  const T* d = Jc + csc;
  bc[csc] = d[0] * sp + d[ncc] * sc;
  bc[ncc + csc] = d[2 * ncc] * sp + d[3 * ncc] * sc;
  xc[csc] = (T)0;
  xc[ncc + csc] = (T)0;
}

// Natural index of the black cell at colour-split position `pos`.
__device__ __forceinline__ int black_cell(const Geom& G, int pos) {
  const int hx2 = G.nx >> 1;
  const int j = pos / hx2, k = pos - j * hx2;
  return j * G.nx + 2 * k + ((j + 1) & 1);
}

// Bilinear correction (vp, vc) of fine cell (i, j) from the coarse
// unknowns xc (colour-split layout of Gc).
template <typename T>
__device__ __forceinline__ void prolong_value(const Geom& Gc, int i, int j,
                                              const T* __restrict__ xc, T& vp, T& vc) {
  const int I = i >> 1, J = j >> 1;
  int I2 = I + ((i & 1) ? 1 : -1), J2 = J + ((j & 1) ? 1 : -1);
  I2 = I2 < 0 ? 0 : (I2 >= Gc.nx ? Gc.nx - 1 : I2);
  J2 = J2 < 0 ? 0 : (J2 >= Gc.ny ? Gc.ny - 1 : J2);
  const int ncc = Gc.ncell(), hc = Gc.half();
  const int a0 = cs_pos(I, J, Gc.nx, hc), a1 = cs_pos(I2, J, Gc.nx, hc);
  const int a2 = cs_pos(I, J2, Gc.nx, hc), a3 = cs_pos(I2, J2, Gc.nx, hc);
  const T w0 = (T)0.5625, w1 = (T)0.1875, w3 = (T)0.0625;
  vp = w0 * xc[a0] + w1 * (xc[a1] + xc[a2]) + w3 * xc[a3];
  vc = w0 * xc[ncc + a0] + w1 * (xc[ncc + a1] + xc[ncc + a2]) + w3 * xc[ncc + a3];
}

// Fine cell `cell` of level k: x_f += P x_c, cell-centred bilinear
// interpolation (9/16, 3/16, 3/16, 1/16), constant extrapolation at the
// domain boundary. When post-smoothing follows, only black cells are
// corrected: the red half-sweep that comes next overwrites every red value
// without reading it (a point update reads its neighbours only), so the
// result is the same.
template <typename T>
__device__ __forceinline__ void prolong_cell(const Geom& Gc, const Geom& Gf, int cell,
                                             const T* __restrict__ xc, T* __restrict__ xf) {
  const int j = cell / Gf.nx, i = cell - j * Gf.nx;
  T vp, vc;
  prolong_value<T>(Gc, i, j, xc, vp, vc);
  const int cs = cs_pos(i, j, Gf.nx, Gf.half()), ncf = Gf.ncell();
  xf[cs] += vp;
  xf[ncf + cs] += vc;
}

// Coarsest-grid solve x = Ainv b with the stored transposed inverse (see
// k_coarse_inv) by one warp, lanes over unknowns; y is an n-vector of
// scratch in shared memory.
template <typename T>
__device__ __forceinline__ void coarse_solve_warp(const Geom& G, const T* __restrict__ AinvT,
                                                  const T* __restrict__ b, T* __restrict__ x, T* y,
                                                  int l) {
  const int nc = G.ncell(), n = 2 * nc, half = G.half();
  for (int u = l; u < n; u += 32) {
    const int cell = u >> 1, v = u & 1;
    const int j = cell / G.nx, i = cell - j * G.nx;
    y[u] = b[v * nc + cs_pos(i, j, G.nx, half)];
  }
  __syncwarp();
  for (int u = l; u < n; u += 32) {
    T acc = (T)0;
    for (int v = 0; v < n; ++v) acc = fma(AinvT[v * n + u], y[v], acc);
    const int cell = u >> 1, var = u & 1;
    const int j = cell / G.nx, i = cell - j * G.nx;
    x[var * nc + cs_pos(i, j, G.nx, half)] = acc;
  }
}

// ---------------------------------------------------------------------------
// batched multigrid kernels (one thread per cell of all B samples)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_coarse_solve(unsigned long long* ctr, Geom G, int B, const int* __restrict__ active,
                               const T* __restrict__ AinvT, const T* __restrict__ bvec,
                               T* __restrict__ xvec) {
  HENRY_COUNT_LAUNCH(ctr);
  __shared__ T ysh[kBlock / 32][kMaxCoarseUnknowns];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + w;
  if (b >= B || !active[b]) return;
  const int64_t ob = (int64_t)b * 2 * G.ncell();
  coarse_solve_warp<T>(G, AinvT + (int64_t)b * kMaxCoarseUnknowns * kMaxCoarseUnknowns, bvec + ob,
                       xvec + ob, ysh[w], l);
}

// One red (colour 0) or black (colour 1) half-sweep of point-block
// Gauss-Seidel on every sample.
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_smooth(unsigned long long* ctr, Geom G, int B, int colour, const int* __restrict__ active,
         const T* __restrict__ J, const T* __restrict__ bvec, T* __restrict__ xvec) {
  HENRY_COUNT_LAUNCH(ctr);
  const int half = G.half(), ncell = G.ncell();
  const int64_t n = (int64_t)B * half;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int b = (int)(idx / half);
  if (!active[b]) return;
  const int pos = (int)(idx - (int64_t)b * half);
  const int64_t ob = (int64_t)b * 2 * ncell;
  smooth_cell<T>(G, colour, pos, J + (int64_t)b * kJP * ncell, bvec + ob, xvec + ob);
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
k_resid_restrict(unsigned long long* ctr, Geom Gf, Geom Gc, int B, const int* __restrict__ active,
                 const T* __restrict__ Jf, const T* __restrict__ bf, const T* __restrict__ xf,
                 const T* __restrict__ Jc, T* __restrict__ bc, T* __restrict__ xc, int red_only) {
  HENRY_COUNT_LAUNCH(ctr);
  const int ncc = Gc.ncell(), ncf = Gf.ncell();
  const int64_t n = (int64_t)B * ncc;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int b = (int)(idx / ncc);
  if (!active[b]) return;
  const int cell = (int)(idx - (int64_t)b * ncc);
  restrict_cell<T>(Gf, Gc, cell, Jf + (int64_t)b * kJP * ncf, bf + (int64_t)b * 2 * ncf,
                   xf + (int64_t)b * 2 * ncf, Jc + (int64_t)b * kJP * ncc, bc + (int64_t)b * 2 * ncc,
                   xc + (int64_t)b * 2 * ncc, red_only != 0);
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
k_prolong(unsigned long long* ctr, Geom Gc, Geom Gf, int B, const int* __restrict__ active,
          const T* __restrict__ xc, T* __restrict__ xf, int black_only) {
  HENRY_COUNT_LAUNCH(ctr);
  const int ncf = Gf.ncell(), ncc = Gc.ncell();
  const int per = black_only ? Gf.half() : ncf;   // cells corrected per sample
  const int64_t n = (int64_t)B * per;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int b = (int)(idx / per);
  if (!active[b]) return;
  const int u = (int)(idx - (int64_t)b * per);
  const int cell = black_only ? black_cell(Gf, u) : u;
  prolong_cell<T>(Gc, Gf, cell, xc + (int64_t)b * 2 * ncc, xf + (int64_t)b * 2 * ncf);
}

// ---------------------------------------------------------------------------
// fused V-cycles on the small multigrid levels 0..ks (at most kSmallCells
// cells per sample on level ks): one block per sample; J, b and x of these
// levels and the coarsest inverse are staged in shared memory and every
// phase of the cycle is separated by __syncthreads(). Level ks takes b from
// and returns x to global memory (x_ks is read as the initial guess).
// Each staged array is one contiguous run per sample, so the staging is a
// handful of TMA bulk copies issued by one thread (plain loads only for a
// run that is not 16-byte aligned); the first 16 bytes of the dynamic shared
// memory hold their mbarrier.
// ---------------------------------------------------------------------------
constexpr int kSmallCells = 512;   // largest level the shared-memory kernel accepts
constexpr int kMaxLevels = 12;

template <typename T>
struct SmallMG {
  int ks;                           // top small level
  Geom g[kMaxLevels];
  T* J[kMaxLevels];                 // global bases (sample 0)
  T* b[kMaxLevels];
  T* x[kMaxLevels];
};

template <typename T>
__host__ __device__ inline size_t small_smem_bytes(const SmallMG<T>& M) {
  size_t cells = 0;
  for (int k = 0; k <= M.ks; ++k) cells += (size_t)M.g[k].ncell();
  const int n = 2 * M.g[0].ncell();
  return 16 + cells * (kJP + 4) * sizeof(T) + (size_t)n * n * sizeof(T) + n * sizeof(T) + 64;
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
k_vcycle_small(unsigned long long* ctr, SmallMG<T> M, int B, const int* __restrict__ active,
               const T* __restrict__ AinvT, int nu1, int nu2, int ncycles,
               int* __restrict__ status) {
  HENRY_COUNT_LAUNCH(ctr);
  extern __shared__ __align__(16) unsigned char smem[];
  const int bs = blockIdx.x;
  if (!active[bs]) return;
  const int ks = M.ks;
  T* J[kMaxLevels];
  T* bv[kMaxLevels];
  T* xv[kMaxLevels];
  uint64_t* bar = (uint64_t*)smem;
  T* p = (T*)(smem + 16);
  for (int k = 0; k <= ks; ++k) {
    const int nc = M.g[k].ncell();
    J[k] = p; p += kJP * nc;
    bv[k] = p; p += 2 * nc;
    xv[k] = p; p += 2 * nc;
  }
  const int n = 2 * M.g[0].ncell();
  T* A = (T*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  T* y = A + n * n;
  // stage J of all small levels, b and x of the top one and the coarsest
  // inverse: each is one run (destination, source, bytes), sizes multiples of 4
  auto runs = [&](auto&& f) {
    for (int k = 0; k <= ks; ++k) {
      const int nc = M.g[k].ncell();
      f(J[k], M.J[k] + (int64_t)bs * kJP * nc, (unsigned)(kJP * nc * sizeof(T)));
    }
    const int nc = M.g[ks].ncell();
    f(bv[ks], M.b[ks] + (int64_t)bs * 2 * nc, (unsigned)(2 * nc * sizeof(T)));
    f(xv[ks], M.x[ks] + (int64_t)bs * 2 * nc, (unsigned)(2 * nc * sizeof(T)));
    f(A, AinvT + (int64_t)bs * kMaxCoarseUnknowns * kMaxCoarseUnknowns,
      (unsigned)(n * n * sizeof(T)));
  };
  // a copy that did not land in time leaves x_ks untouched (sample flagged)
  if (!stage_runs(bar, runs, status, bs)) return;
  for (int cyc = 0; cyc < ncycles; ++cyc) {
    for (int k = ks; k >= 1; --k) {
      const Geom& G = M.g[k];
      for (int s = 0; s < nu1; ++s)
        for (int col = 0; col < 2; ++col) {
          for (int pos = threadIdx.x; pos < G.half(); pos += blockDim.x)
            smooth_cell<T>(G, col, pos, J[k], bv[k], xv[k]);
          __syncthreads();
        }
      for (int cell = threadIdx.x; cell < M.g[k - 1].ncell(); cell += blockDim.x)
        restrict_cell<T>(G, M.g[k - 1], cell, J[k], bv[k], xv[k], J[k - 1], bv[k - 1],
                         xv[k - 1], nu1 > 0);
      __syncthreads();
    }
    if (threadIdx.x < 32) coarse_solve_warp<T>(M.g[0], A, bv[0], xv[0], y, threadIdx.x);
    __syncthreads();
    for (int k = 1; k <= ks; ++k) {
      const Geom& G = M.g[k];
      if (nu2 > 0)
        for (int pos = threadIdx.x; pos < G.half(); pos += blockDim.x)
          prolong_cell<T>(M.g[k - 1], G, black_cell(G, pos), xv[k - 1], xv[k]);
      else
        for (int cell = threadIdx.x; cell < G.ncell(); cell += blockDim.x)
          prolong_cell<T>(M.g[k - 1], G, cell, xv[k - 1], xv[k]);
      __syncthreads();
      for (int s = 0; s < nu2; ++s)
        for (int col = 0; col < 2; ++col) {
          for (int pos = threadIdx.x; pos < G.half(); pos += blockDim.x)
            smooth_cell<T>(G, col, pos, J[k], bv[k], xv[k]);
          __syncthreads();
        }
    }
  }
  const int nc = M.g[ks].ncell();
  T* dx = M.x[ks] + (int64_t)bs * 2 * nc;
  for (int e = threadIdx.x; e < 2 * nc; e += blockDim.x) dx[e] = xv[ks][e];
}

// Defect-correction update of the FP64 state: u += x (finest level).
template <typename T>
__global__ void k_update(unsigned long long* ctr, Geom G, int B, const int* __restrict__ active,
                         const T* __restrict__ xvec, double* __restrict__ p, double* __restrict__ c) {
  HENRY_COUNT_LAUNCH(ctr);
  const int ncell = G.ncell();
  const int64_t n = (int64_t)B * ncell;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int b = (int)(idx / ncell);
  if (!active[b]) return;
  const int cell = (int)(idx - (int64_t)b * ncell);
  const int j = cell / G.nx, i = cell - j * G.nx;
  const int cs = cs_pos(i, j, G.nx, G.half());
  const int64_t ob = (int64_t)b * 2 * ncell;
  p[idx] += (double)xvec[ob + cs];
  c[idx] += (double)xvec[ob + ncell + cs];
}

// ---------------------------------------------------------------------------
// quantities of interest (section 4): one block per sample
// ---------------------------------------------------------------------------
constexpr double kFreshC = 0.012178;   // fresh-water threshold of Eq. integral_fw
constexpr double kBoxHalf = 0.1;        // half-width of the boxes of Eq. integral_box

__device__ __forceinline__ double bilinear(const Geom& G, const double* c, double x, double y) {
  const double fx = x / G.hx - 0.5, fy = y / G.hy - 0.5;
  int i0 = (int)floor(fx), j0 = (int)floor(fy);
  i0 = i0 < 0 ? 0 : (i0 > G.nx - 2 ? G.nx - 2 : i0);
  j0 = j0 < 0 ? 0 : (j0 > G.ny - 2 ? G.ny - 2 : j0);
  const double tx = fmin(fmax(fx - i0, 0.0), 1.0), ty = fmin(fmax(fy - j0, 0.0), 1.0);
  const int id = j0 * G.nx + i0;
  return (1 - tx) * (1 - ty) * c[id] + tx * (1 - ty) * c[id + 1] + (1 - tx) * ty * c[id + G.nx] +
         tx * ty * c[id + G.nx + 1];
}

static __global__ void __launch_bounds__(kBlock)
k_qoi(unsigned long long* ctr, Phys P, Geom G, int B, const double* __restrict__ p,
      const double* __restrict__ c, const double* __restrict__ phi, double* __restrict__ q,
      double* __restrict__ c_out, double* __restrict__ p_out, int qstride) {
  HENRY_COUNT_LAUNCH(ctr);
  __shared__ double sh[kBlock / 32];
  const int b = blockIdx.x;
  const int ncell = G.ncell();
  const int64_t o = (int64_t)b * ncell;
  double s0 = 0, s1 = 0, s2 = 0, fw = 0;
  double box[15];
#pragma unroll
  for (int m = 0; m < 15; ++m) box[m] = 0.0;
  // box columns and rows of Eq. integral_box around the points of Eq.
  // 12points (frame y in [0, 1]), half-width 0.1, clipped to the domain
  const double bx[5] = {0.90, 1.15, 1.40, 1.65, 1.90};
  const double by[3] = {0.05, 0.25, 0.50};
  for (int cell = threadIdx.x; cell < ncell; cell += blockDim.x) {
    const double cv = c[o + cell];
    const double rho = P.rho0 + P.drho * cv;
    const int j = cell / G.nx, i = cell - j * G.nx;
    const double x = (i + 0.5) * G.hx;
    s0 += cv * rho;
    s1 += phi[o + cell] * rho * cv;
    s2 += cv * (P.Lx - x);
    fw += cv <= kFreshC ? 1.0 : 0.0;
    const double xl = i * G.hx, yl = j * G.hy;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double oy = fmax(fmin(yl + G.hy, by[r] + kBoxHalf) - fmax(yl, by[r] - kBoxHalf), 0.0);
      if (oy == 0.0) continue;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const double ox = fmax(fmin(xl + G.hx, bx[k] + kBoxHalf) - fmax(xl, bx[k] - kBoxHalf), 0.0);
        box[5 * r + k] += cv * rho * oy * ox;
      }
    }
    if (c_out) c_out[o + cell] = cv;
    if (p_out) p_out[o + cell] = p[o + cell] + P.rho0 * P.g * (P.Ly - (j + 0.5) * G.hy);
  }
  const double V = G.hx * G.hy;
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  fw = block_sum(fw, sh);
#pragma unroll
  for (int m = 0; m < 15; ++m) box[m] = block_sum(box[m], sh);
  if (threadIdx.x == 0) {
    double* qb = q + (int64_t)b * qstride;   // [B][...][kNQ]: sample stride qstride
    qb[0] = s0 * V;
    qb[1] = s1 * V;
    qb[2] = s2 * V;
    qb[3] = bilinear(G, c + o, 1.40, 0.05);
    qb[4] = bilinear(G, c + o, 1.65, 0.25);
    qb[5] = bilinear(G, c + o, 1.90, 0.50);
    qb[6] = fw * V;
#pragma unroll
    for (int m = 0; m < 15; ++m) qb[7 + m] = box[m];
  }
}

// p -> p' = p - rho0 g (Ly - y) for the natural-layout entry point.
static __global__ void k_reduce_pressure(Phys P, Geom G, int B, const double* __restrict__ p,
                                  double* __restrict__ pr) {
  const int64_t n = (int64_t)B * G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int cell = (int)(idx % G.ncell());
  const int j = cell / G.nx;
  pr[idx] = p[idx] - P.rho0 * P.g * (P.Ly - (j + 0.5) * G.hy);
}

// ---------------------------------------------------------------------------
// V-cycles on levels 0..kc by one thread-block cluster per sample: the CL
// blocks of a cluster split every phase's cells among them and are
// separated by hardware cluster barriers (the blocks of a cluster are
// co-scheduled, so the barrier cannot wait on a block that never runs).
// Operators and vectors stay in global memory (L2 resident at these sizes);
// the barrier's release/acquire semantics at cluster scope make each phase's
// global writes visible to the whole cluster in the next phase.
// Level kc takes b from and returns x to global memory like the batched
// kernels; x_kc is read as the initial guess.
// ---------------------------------------------------------------------------
constexpr int kMaxCluster = 8;

template <typename T>
__global__ void __launch_bounds__(kBlock)
k_vcycle_cluster(unsigned long long* ctr, SmallMG<T> M, int B, const int* __restrict__ active,
                 const T* __restrict__ AinvT, int nu1, int nu2,
                 int ncycles, int CL) {
  HENRY_COUNT_LAUNCH(ctr);
  namespace cg = cooperative_groups;
  __shared__ T ysh[kMaxCoarseUnknowns];
  const int b = blockIdx.x / CL;
  const int rank = blockIdx.x - b * CL;
  if (b >= B || !active[b]) return;           // uniform over the cluster
  cg::cluster_group cl = cg::this_cluster();
  auto sync = [&]() {
    if (CL > 1) cl.sync(); else __syncthreads();
  };
  const int nthr = CL * blockDim.x;
  const int gid = rank * blockDim.x + threadIdx.x;
  const int kc = M.ks;
  T* J[kMaxLevels];
  T* bv[kMaxLevels];
  T* xv[kMaxLevels];
  for (int k = 0; k <= kc; ++k) {
    const int64_t nc = M.g[k].ncell();
    J[k] = M.J[k] + (int64_t)b * kJP * nc;
    bv[k] = M.b[k] + (int64_t)b * 2 * nc;
    xv[k] = M.x[k] + (int64_t)b * 2 * nc;
  }
  const T* A = AinvT + (int64_t)b * kMaxCoarseUnknowns * kMaxCoarseUnknowns;
  for (int cyc = 0; cyc < ncycles; ++cyc) {
    for (int k = kc; k >= 1; --k) {
      const Geom& G = M.g[k];
      for (int sw = 0; sw < nu1; ++sw)
        for (int col = 0; col < 2; ++col) {
          for (int pos = gid; pos < G.half(); pos += nthr) smooth_cell<T>(G, col, pos, J[k], bv[k], xv[k]);
          sync();
        }
      for (int cell = gid; cell < M.g[k - 1].ncell(); cell += nthr)
        restrict_cell<T>(G, M.g[k - 1], cell, J[k], bv[k], xv[k], J[k - 1], bv[k - 1],
                         xv[k - 1], nu1 > 0);
      sync();
    }
    if (rank == 0 && threadIdx.x < 32) coarse_solve_warp<T>(M.g[0], A, bv[0], xv[0], ysh, threadIdx.x);
    sync();
    for (int k = 1; k <= kc; ++k) {
      const Geom& G = M.g[k];
      if (nu2 > 0)
        for (int pos = gid; pos < G.half(); pos += nthr)
          prolong_cell<T>(M.g[k - 1], G, black_cell(G, pos), xv[k - 1], xv[k]);
      else
        for (int cell = gid; cell < G.ncell(); cell += nthr)
          prolong_cell<T>(M.g[k - 1], G, cell, xv[k - 1], xv[k]);
      sync();
      for (int sw = 0; sw < nu2; ++sw)
        for (int col = 0; col < 2; ++col) {
          for (int pos = gid; pos < G.half(); pos += nthr) smooth_cell<T>(G, col, pos, J[k], bv[k], xv[k]);
          sync();
        }
    }
  }
}

// ---------------------------------------------------------------------------
// BiCGStab on the row-scaled finest-level system At x = bt, right-
// preconditioned by one multigrid V-cycle (van der Vorst's algorithm; the
// paper's linear solver is a Krylov method preconditioned by geometric
// multigrid, section 2.3). Vectors are [B][2][ncell] in the multigrid type
// and colour-split layout; per-sample scalars in S[B][kKryS] (FP64):
//   0 rho, 1 alpha, 2 omega, 3 beta, 4..6 dot products.
// Samples that are inactive are skipped by every kernel.
// ---------------------------------------------------------------------------
constexpr int kKryS = 8;

// (At y)_P = y_P + sum_Q At_PQ y_Q at cell (i, j).
template <typename T>
__device__ __forceinline__ void scaled_apply_cell(const Geom& G, int i, int j,
                                                  const T* __restrict__ Jb,
                                                  const T* __restrict__ y, T& ap, T& ac) {
  const int ncell = G.ncell(), half = G.half(), nx = G.nx;
  const int cs = cs_pos(i, j, nx, half);
  const T* Jc = Jb + cs;
  const T* yp = y;
  const T* yc = y + ncell;
  ap = yp[cs];
  ac = yc[cs];
  T vp, vc;
  if (i > 0) {
    const int q = cs_pos(i - 1, j, nx, half);
    vp = yp[q]; vc = yc[q];
    ap += Jc[4 * ncell] * vp; ap += Jc[5 * ncell] * vc;
    ac += Jc[6 * ncell] * vp; ac += Jc[7 * ncell] * vc;
  }
  if (i < nx - 1) {
    const int q = cs_pos(i + 1, j, nx, half);
    vp = yp[q]; vc = yc[q];
    ap += Jc[8 * ncell] * vp; ap += Jc[9 * ncell] * vc;
    ac += Jc[10 * ncell] * vp; ac += Jc[11 * ncell] * vc;
  }
  if (j > 0) {
    const int q = cs_pos(i, j - 1, nx, half);
    vp = yp[q]; vc = yc[q];
    ap += Jc[12 * ncell] * vp; ap += Jc[13 * ncell] * vc;
    ac += Jc[14 * ncell] * vp; ac += Jc[15 * ncell] * vc;
  }
  if (j < G.ny - 1) {
    const int q = cs_pos(i, j + 1, nx, half);
    vp = yp[q]; vc = yc[q];
    ap += Jc[16 * ncell] * vp; ap += Jc[17 * ncell] * vc;
    ac += Jc[18 * ncell] * vp; ac += Jc[19 * ncell] * vc;
  }
}

// out = At y, one thread per cell of every active sample.
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_kry_matvec(unsigned long long* ctr, Geom G, int B, const int* __restrict__ active,
             const T* __restrict__ J, const T* __restrict__ y, T* __restrict__ out) {
  HENRY_COUNT_LAUNCH(ctr);
  const int ncell = G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * ncell) return;
  const int b = (int)(idx / ncell);
  if (!active[b]) return;
  const int cell = (int)(idx - (int64_t)b * ncell);
  const int j = cell / G.nx, i = cell - j * G.nx;
  const int64_t o = (int64_t)b * 2 * ncell;
  T ap, ac;
  scaled_apply_cell<T>(G, i, j, J + (int64_t)b * kJP * ncell, y + o, ap, ac);
  const int cs = cs_pos(i, j, G.nx, G.half());
  out[o + cs] = ap;
  out[o + ncell + cs] = ac;
}

// Partial sums of up to two dot products (a1, b1) and (a2, b2) over one
// sample's 2 ncell entries, in FP64: grid (chunks, B), each block sums
// kBlock * 4 consecutive entries; partial[k][b][chunk].
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_kry_dot(unsigned long long* ctr, int n2, int B, const int* __restrict__ active,
          const T* __restrict__ a1, const T* __restrict__ b1, const T* __restrict__ a2,
          const T* __restrict__ b2, double* __restrict__ partial) {
  HENRY_COUNT_LAUNCH(ctr);
  __shared__ double sh[kBlock / 32];
  const int b = blockIdx.y;
  if (!active[b]) return;
  const int64_t o = (int64_t)b * n2;
  const int base = blockIdx.x * kBlock * 4;
  double s1 = 0.0, s2 = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = base + k * kBlock + threadIdx.x;
    if (e < n2) {
      s1 += (double)a1[o + e] * (double)b1[o + e];
      if (a2) s2 += (double)a2[o + e] * (double)b2[o + e];
    }
  }
  s1 = block_sum(s1, sh);
  if (a2) s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    partial[(int64_t)b * gridDim.x + blockIdx.x] = s1;
    if (a2) partial[((int64_t)B + b) * gridDim.x + blockIdx.x] = s2;
  }
}

// Per-sample BiCGStab scalars, one thread per sample (fixed-order sums of
// the dot partials). stage 0: rho_new = (rh, r), beta = (rho_new / rho)
// (alpha / omega), rho = rho_new; stage 1: alpha = rho / (rh, v); stage 2:
// omega = (t, s) / (t, t). A zero denominator gives a zero coefficient (the
// outer defect correction, whose residual is the FP64 one, carries on).
static __global__ void k_kry_scalars(unsigned long long* ctr, int B, int nchunk, int stage,
                              const int* __restrict__ active, const double* __restrict__ partial,
                              double* __restrict__ S) {
  HENRY_COUNT_LAUNCH(ctr);
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  double d1 = 0.0, d2 = 0.0;
  for (int k = 0; k < nchunk; ++k) {
    d1 += partial[(int64_t)b * nchunk + k];
    if (stage == 2) d2 += partial[((int64_t)B + b) * nchunk + k];
  }
  double* s = S + (int64_t)b * kKryS;
  if (stage == 0) {
    const double den = s[0] * s[2];
    s[3] = den != 0.0 ? (d1 / s[0]) * (s[1] / s[2]) : 0.0;
    s[0] = d1;
  } else if (stage == 1) {
    s[1] = d1 != 0.0 ? s[0] / d1 : 0.0;
  } else {
    s[2] = d2 != 0.0 ? d1 / d2 : 0.0;
  }
}

// Vector updates of one BiCGStab iteration, one thread per entry of every
// active sample. op 0 (start): r = rh = bt, p = v = xk = 0, scalars 1.
// op 1: p = r + beta (p - omega v); b = p, x = 0 (preconditioner input).
// op 2: xk += alpha y (y = x); r -= alpha v; b = r, x = 0.
// op 3: xk += omega z (z = x); r -= omega t.
// op 4: x = xk (the correction handed to the state update).
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_kry_update(unsigned long long* ctr, int n2, int B, int op, const int* __restrict__ active,
             double* __restrict__ S, T* __restrict__ r, T* __restrict__ rh, T* __restrict__ p,
             T* __restrict__ v, T* __restrict__ t, T* __restrict__ xk, T* __restrict__ bvec,
             T* __restrict__ xvec) {
  HENRY_COUNT_LAUNCH(ctr);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * n2) return;
  const int b = (int)(idx / n2);
  if (!active[b]) return;
  const double* s = S + (int64_t)b * kKryS;
  switch (op) {
    case 0: {
      const T bt = bvec[idx];
      r[idx] = bt; rh[idx] = bt; p[idx] = (T)0; v[idx] = (T)0; xk[idx] = (T)0;
      if (idx - (int64_t)b * n2 == 0) {
        double* w = S + (int64_t)b * kKryS;
        w[0] = w[1] = w[2] = 1.0;
      }
      break;
    }
    case 1: {
      const T beta = (T)s[3], omega = (T)s[2];
      const T pn = r[idx] + beta * (p[idx] - omega * v[idx]);
      p[idx] = pn; bvec[idx] = pn; xvec[idx] = (T)0;
      break;
    }
    case 2: {
      const T alpha = (T)s[1];
      xk[idx] += alpha * xvec[idx];
      const T sn = r[idx] - alpha * v[idx];
      r[idx] = sn; bvec[idx] = sn; xvec[idx] = (T)0;
      break;
    }
    case 3: {
      const T omega = (T)s[2];
      xk[idx] += omega * xvec[idx];
      r[idx] -= omega * t[idx];
      break;
    }
    default:
      xvec[idx] = xk[idx];
  }
}

// ---------------------------------------------------------------------------
// discrete adjoint through the implicit Euler steps (section 2.3 time
// discretisation): with R^n(u^n, u^{n-1}) = 0 and Q = Q(u^r),
//   J_r^T lam_r = dQ/du^r,   J_n^T lam_n = -(dR^{n+1}/du^n)^T lam_{n+1},
//   dQ/dtheta = -sum_n (dR^n/dtheta)^T lam_n.
// Vectors lam, rhs, res are FP64 [B][2][ncell] in natural cell order.
// ---------------------------------------------------------------------------

// rhs = dQ/du^r (only c enters the QoI), lam = 0. qoi 0: Q_S = int c rho
// (integrand derivative rho0 + 2 drho c), qoi 2: toe = int c (Lx - x).
static __global__ void k_adj_seed(unsigned long long* ctr, Phys P, Geom G, int B, int qoi,
                           const double* __restrict__ c, double* __restrict__ rhs,
                           double* __restrict__ lam) {
  HENRY_COUNT_LAUNCH(ctr);
  const int n = G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * n) return;
  const int b = (int)(idx / n), cell = (int)(idx - (int64_t)b * n);
  const int i = cell % G.nx;
  const double V = G.hx * G.hy;
  const double cv = c[idx];
  const double g = qoi == 0 ? V * (P.rho0 + 2.0 * P.drho * cv) : V * (P.Lx - (i + 0.5) * G.hx);
  const int64_t o = (int64_t)b * 2 * n;
  rhs[o + cell] = 0.0;
  rhs[o + n + cell] = g;
  lam[o + cell] = 0.0;
  lam[o + n + cell] = 0.0;
}

// Transposed operator of one multigrid level, row-scaled like the forward
// one. With M = A^T: M_PP = D_P^T and M_PQ = (A_QP)^T = (D_Q At_QP)^T, so the
// stored blocks are Dinv'_P = (Dinv_P)^T, D'_P = D_P^T and
//   Mt_PQ = (D_P^T)^{-1} (D_Q At_QP)^T = (D_Q At_QP Dinv_P)^T,
// At_QP being the block of neighbour Q in the direction of P (P's west
// block comes from the east block of its west neighbour, etc.).
template <typename T>
__global__ void k_transpose(unsigned long long* ctr, Geom G, int B, const int* __restrict__ active,
                            const T* __restrict__ J, T* __restrict__ JT) {
  HENRY_COUNT_LAUNCH(ctr);
  const int n = G.ncell(), half = G.half(), nx = G.nx;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * n) return;
  const int b = (int)(idx / n);
  if (!active[b]) return;
  const int cell = (int)(idx - (int64_t)b * n);
  const int j = cell / nx, i = cell - j * nx;
  const T* Jb = J + (int64_t)b * kJP * n;
  T* Ob = JT + (int64_t)b * kJP * n;
  const int cs = cs_pos(i, j, nx, half);
  auto blk = [&](int m0, int at, T* v) {
    for (int e = 0; e < 4; ++e) v[e] = Jb[(int64_t)(m0 + e) * n + at];
  };
  auto put = [&](int m0, const T* v) {   // store v transposed: (pp, pc, cp, cc) -> (pp, cp, pc, cc)
    Ob[(int64_t)(m0 + 0) * n + cs] = v[0];
    Ob[(int64_t)(m0 + 1) * n + cs] = v[2];
    Ob[(int64_t)(m0 + 2) * n + cs] = v[1];
    Ob[(int64_t)(m0 + 3) * n + cs] = v[3];
  };
  auto mul = [](const T* x, const T* y, T* z) {   // z = x y, 2x2 row-major
    z[0] = x[0] * y[0] + x[1] * y[2];
    z[1] = x[0] * y[1] + x[1] * y[3];
    z[2] = x[2] * y[0] + x[3] * y[2];
    z[3] = x[2] * y[1] + x[3] * y[3];
  };
  T dinv[4], d[4];
  blk(0, cs, dinv);
  blk(20, cs, d);
  put(0, dinv);
  put(20, d);
  // (dst plane of P, neighbour, plane of the neighbour pointing back to P)
  const int nbr[4] = {i > 0 ? cs_pos(i - 1, j, nx, half) : -1,
                      i < nx - 1 ? cs_pos(i + 1, j, nx, half) : -1,
                      j > 0 ? cs_pos(i, j - 1, nx, half) : -1,
                      j < G.ny - 1 ? cs_pos(i, j + 1, nx, half) : -1};
  const int back[4] = {8, 4, 16, 12};
  for (int q = 0; q < 4; ++q) {
    T g[4] = {0, 0, 0, 0};
    if (nbr[q] >= 0) {
      T dq[4], aq[4], t[4];
      blk(20, nbr[q], dq);
      blk(back[q], nbr[q], aq);
      mul(dq, aq, t);
      mul(t, dinv, g);
    }
    put(4 + 4 * q, g);
  }
}

// res = rhs - J^T lam with the FP64 Jacobian J64 in natural layout
// ([B][20][ncell]); b = Dinv' res in the multigrid type (colour-split; Dinv'
// from the transposed multigrid operator Jmg), x = 0;
// one partial sum of res^2 per block. grid = (chunks of 256 cells, B).
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_adj_residual(unsigned long long* ctr, Geom G, int B, const int* __restrict__ active,
               const double* __restrict__ J64, const double* __restrict__ rhs,
               const double* __restrict__ lam, double* __restrict__ res, const T* __restrict__ Jmg,
               T* __restrict__ bvec, T* __restrict__ xvec, double* __restrict__ partial) {
  HENRY_COUNT_LAUNCH(ctr);
  __shared__ double sh[kBlock / 32];
  const int b = blockIdx.y;
  if (!active[b]) return;
  const int n = G.ncell(), nx = G.nx;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (cell < n) {
    const int j = cell / nx, i = cell - j * nx;
    const double* Jb = J64 + (int64_t)b * 20 * n;
    const double* lp = lam + (int64_t)b * 2 * n;
    const double* lc = lp + n;
    double ap = 0.0, ac = 0.0;
    // contribution of row block (Q, P)^T lam_Q
    auto add = [&](int q, int m0) {
      const double a = Jb[(int64_t)(m0 + 0) * n + q], bb = Jb[(int64_t)(m0 + 1) * n + q];
      const double cc = Jb[(int64_t)(m0 + 2) * n + q], d = Jb[(int64_t)(m0 + 3) * n + q];
      ap += a * lp[q] + cc * lc[q];
      ac += bb * lp[q] + d * lc[q];
    };
    add(cell, 0);
    if (i > 0) add(cell - 1, 8);
    if (i < nx - 1) add(cell + 1, 4);
    if (j > 0) add(cell - nx, 16);
    if (j < G.ny - 1) add(cell + nx, 12);
    const int64_t o = (int64_t)b * 2 * n;
    const double rp = rhs[o + cell] - ap, rc = rhs[o + n + cell] - ac;
    res[o + cell] = rp;
    res[o + n + cell] = rc;
    const int cs = cs_pos(i, j, nx, G.half());
    // right-hand side of the row-scaled transposed multigrid system
    const T* d = Jmg + (int64_t)b * kJP * n + cs;
    const T mp = (T)rp, mc = (T)rc;
    bvec[o + cs] = d[0] * mp + d[n] * mc;
    bvec[o + n + cs] = d[2 * n] * mp + d[3 * n] * mc;
    xvec[o + cs] = (T)0;
    xvec[o + n + cs] = (T)0;
    v = rp * rp + rc * rc;
  }
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) partial[(int64_t)b * gridDim.x + blockIdx.x] = s;
}

// lam += x (colour-split multigrid correction -> natural FP64).
template <typename T>
__global__ void k_adj_update(unsigned long long* ctr, Geom G, int B, const int* __restrict__ active,
                             const T* __restrict__ xvec, double* __restrict__ lam) {
  HENRY_COUNT_LAUNCH(ctr);
  const int n = G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * n) return;
  const int b = (int)(idx / n);
  if (!active[b]) return;
  const int cell = (int)(idx - (int64_t)b * n);
  const int j = cell / G.nx, i = cell - j * G.nx;
  const int cs = cs_pos(i, j, G.nx, G.half());
  const int64_t o = (int64_t)b * 2 * n;
  lam[o + cell] += (double)xvec[o + cs];
  lam[o + n + cell] += (double)xvec[o + n + cs];
}

// Sensitivities of step n: gK[P] -= lam^T dR/dlogK_P, gphi[P] -= lam^T
// dR/dphi_P, gq[j] -= lam^T dR/dq_in(j). A face's advective flux is
// proportional to its transmissibility t = A K_f/(mu d), K_f the harmonic
// mean, so dF/dlogK_L = F_adv K_U/(K_L + K_U); the diffusive salt flux is
// proportional to phi_f, dphi_f/dphi_L = 2 phi_U^2/(phi_L + phi_U)^2. The
// right side's flux is proportional to K_P, its and the left side's
// diffusion to phi_P. Each cell evaluates its four faces itself (no
// atomics); p is the reduced pressure.
static __global__ void k_adj_sens(unsigned long long* ctr, Phys P, Geom G, double tau, double qfac, int B,
                           const double* __restrict__ p, const double* __restrict__ c,
                           const double* __restrict__ c_old, const double* __restrict__ phi,
                           const double* __restrict__ K, const double* __restrict__ tx,
                           const double* __restrict__ dx, const double* __restrict__ ty,
                           const double* __restrict__ dy, const double* __restrict__ lam,
                           double* __restrict__ gK, double* __restrict__ gphi,
                           double* __restrict__ gq) {
  HENRY_COUNT_LAUNCH(ctr);
  const int n = G.ncell(), nx = G.nx, ny = G.ny;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * n) return;
  const int b = (int)(idx / n), cell = (int)(idx - (int64_t)b * n);
  const int j = cell / nx, i = cell - j * nx;
  const int64_t o = (int64_t)b * n;
  const double* lp = lam + (int64_t)b * 2 * n;
  const double* lc = lp + n;
  const double V = G.hx * G.hy, A = G.hy;
  const double cP = c[o + cell], pP = p[o + cell], phP = phi[o + cell], KP = K[o + cell];
  const double rho = P.rho0 + P.drho * cP;
  const double cO = c_old[o + cell];
  const double rho_o = P.rho0 + P.drho * cO;
  double sK = 0.0, sphi = 0.0;
  // accumulation terms
  sphi += lp[cell] * V * (rho - rho_o) / tau + lc[cell] * V * (rho * cP - rho_o * cO) / tau;
  // interior faces: (L, U) canonical, this cell is L (east/north) or U (west/south)
  auto face = [&](int other, bool self_is_L, double t, double gd, double AD_d) {
    const int q = other;
    const double cQ = c[o + q], pQ = p[o + q], phQ = phi[o + q], KQ = K[o + q];
    const double cL = self_is_L ? cP : cQ, cU = self_is_L ? cQ : cP;
    const double pL = self_is_L ? pP : pQ, pU = self_is_L ? pQ : pP;
    const double rL = P.rho0 + P.drho * cL, rU = P.rho0 + P.drho * cU;
    const double flux = -t * ((pU - pL) + (0.5 * P.drho) * (cL + cU) * gd);
    const bool up = flux >= 0.0;
    const double rup = up ? rL : rU, rcup = up ? rL * cL : rU * cU;
    const double share = KQ / (KP + KQ);
    const double dlp = self_is_L ? lp[cell] - lp[q] : lp[q] - lp[cell];
    const double dlc = self_is_L ? lc[cell] - lc[q] : lc[q] - lc[cell];
    sK += (dlp * flux * rup + dlc * flux * rcup) * share;
    const double rbar = 0.5 * (rL + rU);
    const double dphif = 2.0 * phQ * phQ / ((phP + phQ) * (phP + phQ));
    sphi += dlc * (-AD_d * dphif * rbar * (cU - cL));
  };
  const double gdy = P.g * G.hy;
  if (i > 0) face(cell - 1, false, tx[o + cell - 1], 0.0, G.hy * P.D / G.hx);
  if (i < nx - 1) face(cell + 1, true, tx[o + cell], 0.0, G.hy * P.D / G.hx);
  if (j > 0) face(cell - nx, false, ty[o + cell - nx], gdy, G.hx * P.D / G.hy);
  if (j < ny - 1) face(cell + nx, true, ty[o + cell], gdy, G.hx * P.D / G.hy);
  const double dcoF = 2.0 * A * P.D / G.hx;   // boundary diffusion per unit phi
  if (i == 0) {
    const double rb = 0.5 * (rho + P.rho0);
    sphi += lc[cell] * dcoF * rb * cP;
    gq[(int64_t)b * ny + j] -= lp[cell] * (-A * P.rho0) * qfac;   // inflow factor of this step
  }
  if (i == nx - 1) {
    const double rho1 = P.rho0 + P.drho;
    const double tR = 2.0 * A * KP / (P.mu * G.hx);
    const double pb = P.drho * P.g * (P.Ly - (j + 0.5) * G.hy);
    const double q = -tR * (pb - pP);
    const bool up = q >= 0.0;
    const double rup = up ? rho : rho1, rcup = up ? rho * cP : rho1;
    sK += lp[cell] * q * rup + lc[cell] * q * rcup;
    const double rb = 0.5 * (rho + rho1);
    sphi += lc[cell] * (-dcoF * rb * (1.0 - cP));
  }
  gK[o + cell] -= sK;
  gphi[o + cell] -= sphi;
}

// rhs for step n-1: -(dR^n/du^{n-1})^T lam^n; R^n sees u^{n-1} through
// c_old only: dR_p/dc_old = -V phi drho / tau, dR_c/dc_old = -V phi
// (rho(c_old) + drho c_old) / tau.
static __global__ void k_adj_prev_rhs(unsigned long long* ctr, Phys P, Geom G, double tau, int B,
                               const double* __restrict__ phi, const double* __restrict__ c_old,
                               const double* __restrict__ lam, double* __restrict__ rhs) {
  HENRY_COUNT_LAUNCH(ctr);
  const int n = G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * n) return;
  const int b = (int)(idx / n), cell = (int)(idx - (int64_t)b * n);
  const int64_t o = (int64_t)b * 2 * n;
  const double vt = G.hx * G.hy * phi[idx] / tau;
  const double co = c_old[idx];
  rhs[o + cell] = 0.0;
  rhs[o + n + cell] = vt * (P.drho * lam[o + cell] + (P.rho0 + 2.0 * P.drho * co) * lam[o + n + cell]);
}

// dQ/dxi from the per-cell and per-row sensitivities (fields of k_fields);
// one block per sample.
static __global__ void __launch_bounds__(kBlock)
k_adj_contract(unsigned long long* ctr, Phys P, Geom G, int B, int n_xi, int model,
               const double* __restrict__ xi, const double* __restrict__ gK,
               const double* __restrict__ gphi, const double* __restrict__ gq,
               double* __restrict__ dq_dxi) {
  HENRY_COUNT_LAUNCH(ctr);
  __shared__ double sh[kBlock / 32];
  const int b = blockIdx.x;
  const int n = G.ncell();
  const double pi = 3.14159265358979323846;
  double s[6] = {0, 0, 0, 0, 0, 0};
  if (model == 1) {
    // Eq. poro_2levels: phi = phi0 C0 C1 C2 with C0 = 1.2 (1 + 0.2 xi1) in the
    // lower layer, C1 = 1 + 0.15 (xi2 a + xi1 cw), C2 = 1 + 0.2 (xi1 d + xi2 e);
    // log K = log kappa + 3 log phi - log(1 - phi^2) + theta, so
    // dlogK/dxi = (3/phi + 2 phi/(1 - phi^2)) dphi/dxi; q_in base q0 (1 + 0.5 xi3)
    const double z0 = xi[(int64_t)b * n_xi], z1 = xi[(int64_t)b * n_xi + 1];
    for (int cell = threadIdx.x; cell < n; cell += blockDim.x) {
      const int j = cell / G.nx, i = cell - j * G.nx;
      const double x = (i + 0.5) * G.hx, yp = (j + 0.5) * G.hy - P.Ly;
      const bool low = yp < -0.8;
      const double c0 = low ? 1.2 * (1.0 + 0.2 * z0) : 1.0, dc0 = low ? 1.2 * 0.2 : 0.0;
      const double a = cos(pi * x / 2) - sin(2 * pi * yp), cw = cos(2 * pi * x);
      const double d = sin(64 * pi * x), e = sin(32 * pi * yp);
      const double c1 = 1.0 + 0.15 * (z1 * a + z0 * cw), c2 = 1.0 + 0.2 * (z0 * d + z1 * e);
      const double ph = P.phi0 * c0 * c1 * c2;
      const double dph0 = P.phi0 * (dc0 * c1 * c2 + c0 * 0.15 * cw * c2 + c0 * c1 * 0.2 * d);
      const double dph1 = P.phi0 * (c0 * 0.15 * a * c2 + c0 * c1 * 0.2 * e);
      const double dlk = 3.0 / ph + 2.0 * ph / (1.0 - ph * ph);
      const double gp = gphi[(int64_t)b * n + cell], gk = gK[(int64_t)b * n + cell];
      s[0] += (gp + gk * dlk) * dph0;
      s[1] += (gp + gk * dlk) * dph1;
    }
    for (int j = threadIdx.x; j < G.ny; j += blockDim.x) s[2] += gq[(int64_t)b * G.ny + j] * P.q0 * 0.5;
    for (int k = 0; k < n_xi; ++k) {
      const double t = block_sum(s[k], sh);
      if (threadIdx.x == 0) dq_dxi[(int64_t)b * n_xi + k] = t;
    }
    return;
  }
  for (int cell = threadIdx.x; cell < n; cell += blockDim.x) {
    const int j = cell / G.nx, i = cell - j * G.nx;
    const double x = (i + 0.5) * G.hx, y = (j + 0.5) * G.hy;
    const double gp = gphi[(int64_t)b * n + cell], gk = gK[(int64_t)b * n + cell];
    s[0] += gp * P.phi0 * 0.1 * cos(0.5 * pi * x) * sin(pi * y);
    s[1] += gk * 0.5 * sin(0.5 * pi * x) * cos(pi * y);
    if (n_xi >= 6) {
      s[3] += gp * P.phi0 * 0.05 * cos(pi * x) * sin(2.0 * pi * y);
      s[4] += gk * 0.05 * sin(pi * x) * cos(2.0 * pi * y);
    }
  }
  for (int j = threadIdx.x; j < G.ny; j += blockDim.x) {
    const double gv = gq[(int64_t)b * G.ny + j];
    s[2] += gv * P.q0 * 0.1;
    if (n_xi >= 6) s[5] += gv * P.q0 * 0.05 * cos(pi * (j + 0.5) * G.hy);
  }
  for (int k = 0; k < n_xi; ++k) {
    const double t = block_sum(s[k], sh);
    if (threadIdx.x == 0) dq_dxi[(int64_t)b * n_xi + k] = t;
  }
}

}  // namespace henry
