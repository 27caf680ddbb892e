// Vertex-centred variant of the solve (discretisation = 1; arxiv 2403.17018,
// section 2.3: vertex-centred finite volumes with partial upwinding of the
// convective terms, first order in h + tau in practice, Eq. 1st_ord_conv).
//
// Readings (the paper gives the scheme by reference only):
//  * unknowns at the nodes (i hx, j hy), i = 0..nx-1, j = 0..ny of the level
//    grid (nx x ny cells); the column x = Lx is Dirichlet (p = rho1 g (Ly -
//    y), c = 1) and the column x = 0 has c = 0 (a Dirichlet row scaled by
//    V phi0 rho0 / tau) and the fresh-water mass inflow (section 2.1);
//  * control volume of a node: its box clipped to the domain; the random
//    field enters at integration points: phi at the centres of the box's
//    quarter cells (storage), K and phi at the midpoints of the two half
//    segments of each box face (transmissibility T and diffusive conductance
//    Dc of the face);
//  * two-point fluxes, Q = -T (p_U - p_L + rho_bar g d e_y), and partial
//    upwinding of the advected rho and rho c with the exponentially fitted
//    weight w = (1 + alpha(Pe) sgn Q) / 2, alpha(Pe) = coth(Pe/2) - 2/Pe,
//    Pe = |Q| / Dc (Allen-Southwell / Il'in).
// The node grid is a Geom of nx x (ny + 1) "cells" (its colour-split layout
// needs nx even), so the batched BiCGStab, smoother, check and update
// kernels of the cell-centred solver serve it unchanged. The linear solver
// of each defect-correction iteration is BiCGStab right-preconditioned by
// red-black point-block Gauss-Seidel sweeps (no multigrid hierarchy for
// this variant); the FP64 residual decides convergence as in the
// cell-centred solve. Pressure unknown: p' = p - rho0 g (Ly - y).
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "kernels.cuh"
#include "vc.h"

namespace henry {

namespace {

inline int grid1(int64_t n) { return (int)((n + kBlock - 1) / kBlock); }
size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

#define VCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
      return e_ == cudaErrorMemoryAllocation ? HENRY_E_NOMEM : HENRY_E_CUDA;      \
    }                                                                              \
  } while (0)

}  // namespace

// alpha(Pe) = coth(Pe/2) - 2/Pe (Pe >= 0) and its derivative. Taylor series
// where the direct forms lose digits to cancellation: alpha below Pe = 1e-2
// (Pe/6 - Pe^3/360 + Pe^5/15120 - Pe^7/604800), alpha' below Pe = 0.1
// (1/6 - Pe^2/120 + Pe^4/3024 - 7 Pe^6/604800 + 9 Pe^8/23950080).
__device__ __forceinline__ void fitted_alpha(double Pe, double& a, double& da) {
  const double P2 = Pe * Pe;
  if (Pe < 1e-2)
    a = Pe * (1.0 / 6 - P2 * (1.0 / 360 - P2 * (1.0 / 15120 - P2 / 604800)));
  else
    a = 1.0 / tanh(0.5 * Pe) - 2.0 / Pe;
  if (Pe < 0.1) {
    da = 1.0 / 6 - P2 * (1.0 / 120 - P2 * (1.0 / 3024 - P2 * (7.0 / 604800 - P2 * (9.0 / 23950080))));
  } else {
    const double cth = 1.0 / tanh(0.5 * Pe);
    da = 2.0 / P2 - 0.5 * (cth * cth - 1.0);
  }
}

struct VcFace {
  double Fm, Fs;
  double mLp, mLc, mUp, mUc, sLp, sLc, sUp, sUc;   // d(Fm, Fs)/d(p, c) of L and U
};

// Flux from L to U (reduced pressures; gd = g d for a vertical pair, else 0).
template <bool WANT_J>
__device__ __forceinline__ void vc_face(const Phys& P, double T, double Dc, double pL, double cL,
                                        double pU, double cU, double gd, VcFace& f) {
  const double rL = P.rho0 + P.drho * cL;
  const double rU = P.rho0 + P.drho * cU;
  const double rbar = 0.5 * (rL + rU);
  const double Q = -T * ((pU - pL) + (0.5 * P.drho) * (cL + cU) * gd);
  const double s = Q >= 0.0 ? 1.0 : -1.0;
  double alpha = 1.0, dalpha = 0.0;
  if (Dc > 0.0) fitted_alpha(Q * s / Dc, alpha, dalpha);
  const double w = 0.5 * (1.0 + alpha * s);
  const double aL = rL * cL, aU = rU * cU;
  const double rst = w * rL + (1.0 - w) * rU;
  const double ast = w * aL + (1.0 - w) * aU;
  f.Fm = Q * rst;
  f.Fs = Q * ast - Dc * rbar * (cU - cL);
  if (WANT_J) {
    const double dw = Dc > 0.0 ? 0.5 * dalpha / Dc : 0.0;   // dw/dQ
    const double dQc = -T * gd * 0.5 * P.drho;              // dQ/dc_L = dQ/dc_U
    const double gm = rst + Q * (rL - rU) * dw;             // dFm/dQ
    const double gs = ast + Q * (aL - aU) * dw;             // dFs/dQ
    const double dif = -Dc * 0.5 * P.drho * (cU - cL);
    f.mLp = gm * T;
    f.mUp = -gm * T;
    f.mLc = gm * dQc + Q * w * P.drho;
    f.mUc = gm * dQc + Q * (1.0 - w) * P.drho;
    f.sLp = gs * T;
    f.sUp = -gs * T;
    f.sLc = gs * dQc + Q * w * (rL + P.drho * cL) + dif + Dc * rbar;
    f.sUc = gs * dQc + Q * (1.0 - w) * (rU + P.drho * cU) + dif - Dc * rbar;
  }
}

// Coefficients of every unknown node (G: node grid nx x (ny + 1), hx, hy
// the cell sizes): box storage integral vphi and area vol, T and Dc of the
// east face (the last column's to the Dirichlet column) and of the north
// face, the inflow through the left box face, and the storage integral of
// the Dirichlet column (for the QoIs).
__global__ void k_vc_coeffs(unsigned long long* ctr, Phys P, Geom G, int B, int n_xi, int model,
                            const double* __restrict__ xi, double* __restrict__ vphi,
                            double* __restrict__ vol, double* __restrict__ tx,
                            double* __restrict__ dx, double* __restrict__ ty,
                            double* __restrict__ dy, double* __restrict__ qin,
                            double* __restrict__ vphi_r, int* __restrict__ status) {
  HENRY_COUNT_LAUNCH(ctr);
  const int n = G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * n) return;
  const int b = (int)(idx / n), node = (int)(idx - (int64_t)b * n);
  const int nx = G.nx, nrow = G.ny, j = node / nx, i = node - j * nx;
  const double hx = G.hx, hy = G.hy;
  const double* z = xi + (int64_t)b * n_xi;
  const double x = i * hx, y = j * hy;
  // half segments of the box: (centre, length), zero length where clipped
  const double xc[2] = {x - hx / 4, x + hx / 4}, xl[2] = {i > 0 ? hx / 2 : 0.0, hx / 2};
  const double yc[2] = {y - hy / 4, y + hy / 4};
  const double yl[2] = {j > 0 ? hy / 2 : 0.0, j < nrow - 1 ? hy / 2 : 0.0};
  double ph, K, s = 0.0, v = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int c = 0; c < 2; ++c) {
      field_at(P, model, n_xi, z, xc[a], yc[c], false, 0.0, ph, K);
      s = s + ph * (yl[c] * xl[a]);
      v = v + yl[c] * xl[a];
    }
  vphi[idx] = s;
  vol[idx] = v;
  double t = 0.0, d = 0.0;
  for (int c = 0; c < 2; ++c) {
    field_at(P, model, n_xi, z, x + hx / 2, yc[c], false, 0.0, ph, K);
    t = t + K * yl[c] / (P.mu * hx);
    d = d + ph * yl[c] * P.D / hx;
  }
  tx[idx] = t;
  dx[idx] = d;
  t = d = 0.0;
  if (j < nrow - 1) {
    for (int a = 0; a < 2; ++a) {
      field_at(P, model, n_xi, z, xc[a], y + hy / 2, false, 0.0, ph, K);
      t = t + K * xl[a] / (P.mu * hy);
      d = d + ph * xl[a] * P.D / hy;
    }
  }
  ty[idx] = t;
  dy[idx] = d;
  if (i == 0)
    qin[(int64_t)b * nrow + j] = inflow_at(P, model, n_xi, z, yc[0]) * yl[0] +
                                 inflow_at(P, model, n_xi, z, yc[1]) * yl[1];
  if (i == nx - 1) {   // the Dirichlet column's box: its left half only
    const double xr = nx * hx;
    double sr = 0.0;
    for (int c = 0; c < 2; ++c) {
      field_at(P, model, n_xi, z, xr - hx / 4, yc[c], false, 0.0, ph, K);
      sr = sr + ph * (yl[c] * (hx / 2));
    }
    vphi_r[(int64_t)b * nrow + j] = sr;
  }
  if (node == 0 && status) {
    bool ok = true;
    for (int m = 0; m < n_xi; ++m) ok = ok && isfinite(z[m]);
    status[b] = ok ? 0 : kStatusBadInput;
  }
}

// Residual of one implicit step at every node and, optionally, its exact
// Jacobian. NATURAL: R [B][2][n] and J [B][20][n] in natural node order
// (blocks P, W, E, S, N; (pp, pc, cp, cc)); else the multigrid layout of
// the cell-centred solver: row-scaled operator (store_operator), b = -D^-1
// R, x = 0, and one partial sum of R_p^2 + R_c^2 per block. grid (chunks of
// kBlock nodes, B).
template <bool NATURAL, bool WANT_J>
__global__ void __launch_bounds__(kBlock)
k_vc_resjac(unsigned long long* ctr, Phys P, Geom G, double tau, int B,
            const double* __restrict__ vphi, const double* __restrict__ vol,
            const double* __restrict__ tx, const double* __restrict__ dx,
            const double* __restrict__ ty, const double* __restrict__ dy,
            const double* __restrict__ qin, const double* __restrict__ p,
            const double* __restrict__ c, const double* __restrict__ c_old,
            const int* __restrict__ active, double* __restrict__ J, double* __restrict__ bvec,
            double* __restrict__ xvec, double* __restrict__ partial) {
  HENRY_COUNT_LAUNCH(ctr);
  __shared__ double sh[kBlock / 32];
  const int b = blockIdx.y;
  if (!NATURAL && !active[b]) return;
  const int nx = G.nx, nrow = G.ny, n = G.ncell();
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (node < n) {
    const int j = node / nx, i = node - j * nx;
    const int64_t o = (int64_t)b * n + node;
    const double pP = p[o], cP = c[o], cO = c_old[o];
    const double rho = P.rho0 + P.drho * cP, rho_o = P.rho0 + P.drho * cO;
    const double vp = vphi[o];
    double Rp = vp * (rho - rho_o) / tau;
    double Rc = vp * (rho * cP - rho_o * cO) / tau;
    double Jc[20];
#pragma unroll
    for (int m = 0; m < 20; ++m) Jc[m] = 0.0;
    Jc[1] = vp * P.drho / tau;
    Jc[3] = vp * (rho + P.drho * cP) / tau;
    VcFace f;
    const double gdy = P.g * G.hy;
    // east face (to the Dirichlet column at i = nx - 1)
    if (i < nx - 1) {
      vc_face<WANT_J>(P, tx[o], dx[o], pP, cP, p[o + 1], c[o + 1], 0.0, f);
      if (WANT_J) { Jc[8] = f.mUp; Jc[9] = f.mUc; Jc[10] = f.sUp; Jc[11] = f.sUc; }
    } else {
      const double pb = P.drho * P.g * (P.Ly - j * G.hy);
      vc_face<WANT_J>(P, tx[o], dx[o], pP, cP, pb, 1.0, 0.0, f);
    }
    Rp = Rp + f.Fm;
    Rc = Rc + f.Fs;
    if (WANT_J) { Jc[0] += f.mLp; Jc[1] += f.mLc; Jc[2] += f.sLp; Jc[3] += f.sLc; }
    if (i > 0) {   // west face: this node is U
      vc_face<WANT_J>(P, tx[o - 1], dx[o - 1], p[o - 1], c[o - 1], pP, cP, 0.0, f);
      Rp -= f.Fm;
      Rc -= f.Fs;
      if (WANT_J) {
        Jc[0] -= f.mUp; Jc[1] -= f.mUc; Jc[2] -= f.sUp; Jc[3] -= f.sUc;
        Jc[4] = -f.mLp; Jc[5] = -f.mLc; Jc[6] = -f.sLp; Jc[7] = -f.sLc;
      }
    }
    if (j < nrow - 1) {   // north face: this node is L
      vc_face<WANT_J>(P, ty[o], dy[o], pP, cP, p[o + nx], c[o + nx], gdy, f);
      Rp += f.Fm;
      Rc += f.Fs;
      if (WANT_J) {
        Jc[0] += f.mLp; Jc[1] += f.mLc; Jc[2] += f.sLp; Jc[3] += f.sLc;
        Jc[16] = f.mUp; Jc[17] = f.mUc; Jc[18] = f.sUp; Jc[19] = f.sUc;
      }
    }
    if (j > 0) {   // south face: this node is U
      vc_face<WANT_J>(P, ty[o - nx], dy[o - nx], p[o - nx], c[o - nx], pP, cP, gdy, f);
      Rp -= f.Fm;
      Rc -= f.Fs;
      if (WANT_J) {
        Jc[0] -= f.mUp; Jc[1] -= f.mUc; Jc[2] -= f.sUp; Jc[3] -= f.sUc;
        Jc[12] = -f.mLp; Jc[13] = -f.mLc; Jc[14] = -f.sLp; Jc[15] = -f.sLc;
      }
    }
    if (i == 0) {   // fresh-water inflow; c = 0 as a Dirichlet row
      Rp += -P.rho0 * qin[(int64_t)b * nrow + j];
      const double S = vol[o] * P.phi0 * P.rho0 / tau;
      Rc = S * cP;
      Jc[2] = 0.0;
      Jc[3] = S;
#pragma unroll
      for (int q = 1; q < 5; ++q) { Jc[4 * q + 2] = 0.0; Jc[4 * q + 3] = 0.0; }
    }
    if (NATURAL) {
      double* Rn = bvec + (int64_t)b * 2 * n;
      Rn[node] = Rp;
      Rn[n + node] = Rc;
      if (WANT_J && J) {
        double* Jn = J + (int64_t)b * 20 * n + node;
#pragma unroll
        for (int m = 0; m < 20; ++m) Jn[(int64_t)m * n] = Jc[m];
      }
    } else {
      const int cs = cs_pos(i, j, nx, G.half());
      double* Jb = J + (int64_t)b * kJP * n + cs;
      double d[4];
      if (WANT_J) {
        store_operator<double>(Jb, n, Jc, d);
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) d[m] = Jb[(int64_t)m * n];
      }
      const int64_t ob = (int64_t)b * 2 * n;
      bvec[ob + cs] = d[0] * (-Rp) + d[1] * (-Rc);
      bvec[ob + n + cs] = d[2] * (-Rp) + d[3] * (-Rc);
      xvec[ob + cs] = 0.0;
      xvec[ob + n + cs] = 0.0;
    }
    v = Rp * Rp + Rc * Rc;
  }
  if (!NATURAL) {
    const double s = block_sum(v, sh);
    if (threadIdx.x == 0) partial[(int64_t)b * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_vc_copy_int(unsigned long long* ctr, int n, const int* __restrict__ src,
                              int* __restrict__ dst, int do_or) {
  HENRY_COUNT_LAUNCH(ctr);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = do_or ? (dst[i] | src[i]) : src[i];
}

// Full pressure -> reduced pressure p' = p - rho0 g (Ly - y) at the nodes.
__global__ void k_vc_reduce_pressure(Phys P, Geom G, int B, const double* __restrict__ p,
                                     double* __restrict__ pr) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * G.ncell()) return;
  const int j = (int)(idx % G.ncell()) / G.nx;
  pr[idx] = p[idx] - P.rho0 * P.g * (P.Ly - j * G.hy);
}

// Initial state: c = 0, reduced pressure of seawater hydrostatics.
__global__ void k_vc_init(unsigned long long* ctr, Phys P, Geom G, int B, double* __restrict__ p,
                          double* __restrict__ c, int* __restrict__ iters, int* __restrict__ step) {
  HENRY_COUNT_LAUNCH(ctr);
  const int n = G.ncell();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * n) return;
  const int node = (int)(idx % n);
  const int j = node / G.nx;
  p[idx] = P.drho * P.g * (P.Ly - j * G.hy);
  c[idx] = 0.0;
  if (node == 0) iters[idx / n] = 0;
  if (idx == 0) *step = 0;
}

// The 22 QoIs with c a nodal field (the Dirichlet column c = 1 included):
// integrals by the box rule, point values by bilinear interpolation of the
// nodes; c_out / p_out (full pressure) at the unknown nodes. One block per
// sample.
__global__ void __launch_bounds__(kBlock)
k_vc_qoi(unsigned long long* ctr, Phys P, Geom G, int B, const double* __restrict__ p,
         const double* __restrict__ c, const double* __restrict__ vphi,
         const double* __restrict__ vphi_r, double* __restrict__ q, double* __restrict__ c_out,
         double* __restrict__ p_out) {
  HENRY_COUNT_LAUNCH(ctr);
  __shared__ double sh[kBlock / 32];
  const int b = blockIdx.x;
  const int nx = G.nx, nrow = G.ny, n = G.ncell();
  const double hx = G.hx, hy = G.hy;
  const int64_t o = (int64_t)b * n;
  double s0 = 0, s1 = 0, s2 = 0, fw = 0, box[15];
#pragma unroll
  for (int m = 0; m < 15; ++m) box[m] = 0.0;
  const double bx[5] = {0.90, 1.15, 1.40, 1.65, 1.90};
  const double by[3] = {0.05, 0.25, 0.50};
  const double thr = 0.012178, half = 0.1;
  for (int k = threadIdx.x; k < nrow * (nx + 1); k += blockDim.x) {
    const int j = k / (nx + 1), i = k - j * (nx + 1);
    const double cv = i < nx ? c[o + j * nx + i] : 1.0;
    const double x = i * hx, y = j * hy;
    const double xl = fmax(x - hx / 2, 0.0), xr = fmin(x + hx / 2, P.Lx);
    const double yb = fmax(y - hy / 2, 0.0), yt = fmin(y + hy / 2, P.Ly);
    const double V = (yt - yb) * (xr - xl);
    const double vph = i < nx ? vphi[o + j * nx + i] : vphi_r[(int64_t)b * nrow + j];
    const double rho = P.rho0 + P.drho * cv;
    s0 += V * cv * rho;
    s1 += vph * rho * cv;
    s2 += V * cv * (P.Lx - x);
    fw += cv <= thr ? V : 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double oy = fmax(fmin(yt, by[r] + half) - fmax(yb, by[r] - half), 0.0);
      if (oy == 0.0) continue;
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        const double ox = fmax(fmin(xr, bx[m] + half) - fmax(xl, bx[m] - half), 0.0);
        box[5 * r + m] += cv * rho * oy * ox;
      }
    }
    if (i < nx) {
      if (c_out) c_out[o + j * nx + i] = cv;
      if (p_out) p_out[o + j * nx + i] = p[o + j * nx + i] + P.rho0 * P.g * (P.Ly - y);
    }
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  fw = block_sum(fw, sh);
#pragma unroll
  for (int m = 0; m < 15; ++m) box[m] = block_sum(box[m], sh);
  if (threadIdx.x == 0) {
    double* qb = q + (int64_t)b * kNQ;
    qb[0] = s0;
    qb[1] = s1;
    qb[2] = s2;
    const double px[3] = {1.40, 1.65, 1.90}, py[3] = {0.05, 0.25, 0.50};
    const double* cb = c + o;
    for (int k = 0; k < 3; ++k) {
      int i0 = (int)floor(px[k] / hx), j0 = (int)floor(py[k] / hy);
      i0 = i0 < 0 ? 0 : (i0 > nx - 1 ? nx - 1 : i0);
      j0 = j0 < 0 ? 0 : (j0 > nrow - 2 ? nrow - 2 : j0);
      const double fx = px[k] / hx - i0, fy = py[k] / hy - j0;
      auto at = [&](int ii, int jj) { return ii < nx ? cb[jj * nx + ii] : 1.0; };
      qb[3 + k] = (1 - fx) * (1 - fy) * at(i0, j0) + fx * (1 - fy) * at(i0 + 1, j0) +
                  (1 - fx) * fy * at(i0, j0 + 1) + fx * fy * at(i0 + 1, j0 + 1);
    }
    qb[6] = fw;
#pragma unroll
    for (int m = 0; m < 15; ++m) qb[7 + m] = box[m];
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
VcSolver::VcSolver(const henry_config& cfg, int nx, int ny, int nt) : cfg_(cfg), nt_(nt) {
  phys_ = Phys{cfg.rho0, cfg.rho1 - cfg.rho0, cfg.mu, cfg.g, cfg.D, cfg.K0, cfg.phi0, cfg.q0,
               cfg.Lx, cfg.Ly};
  tau_ = cfg.T / nt;
  G_ = Geom{nx, ny + 1, cfg.Lx / nx, cfg.Ly / ny};
  kry_ = cfg.krylov_iters >= 2 ? cfg.krylov_iters : 8;
  sweeps_ = cfg.nu1 + cfg.nu2 > 0 ? cfg.nu1 + cfg.nu2 : 1;
}

VcSolver::~VcSolver() {
  if (arena_) cudaFree(arena_);
  if (host_) cudaFreeHost(host_);
}

unsigned long long VcSolver::launches() const {
  unsigned long long v = 0;
  if (counter_) cudaMemcpy(&v, counter_, sizeof(v), cudaMemcpyDeviceToHost);
  return v;
}

int VcSolver::ensure(int B) {
  if (B <= cap_) return HENRY_OK;
  unsigned long long count = 0;
  if (counter_) VCK(cudaMemcpy(&count, counter_, sizeof(count), cudaMemcpyDeviceToHost));
  VCK(cudaDeviceSynchronize());
  if (arena_) cudaFree(arena_);
  arena_ = nullptr;
  if (!host_) VCK(cudaHostAlloc((void**)&host_, 2 * sizeof(int), cudaHostAllocDefault));
  const size_t n = (size_t)G_.ncell() * B, rows = (size_t)G_.ny * B;
  nchunk_ = (G_.ncell() + kBlock - 1) / kBlock;
  kry_nchunk_ = (int)((2 * (size_t)G_.ncell() + kBlock * 4 - 1) / (kBlock * 4));
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  const size_t o_co = take(7 * n * 8);            // vphi vol tx dx ty dy + spare
  const size_t o_row = take(3 * rows * 8);        // qin qin0 vphi_r
  const size_t o_st = take(4 * n * 8);            // p c c_old p_prev
  const size_t o_J = take(kJP * n * 8);
  const size_t o_bx = take(4 * n * 8);            // b x
  const size_t o_kv = take(12 * n * 8);           // r rh p v t xk
  const size_t o_ks = take((size_t)B * kKryS * 8);
  const size_t o_kp = take(2 * (size_t)B * kry_nchunk_ * 8);
  const size_t o_pa = take((size_t)B * nchunk_ * 8);
  const size_t o_s8 = take(2 * (size_t)B * 8);    // res0 res_last
  const size_t o_i4 = take(5 * (size_t)B * 4);    // active it_step status iters (+1)
  const size_t o_misc = take(64);                 // n_active[2] acc[4] step counter
  VCK(cudaMalloc(&arena_, off));
  VCK(cudaMemset(arena_, 0, off));
  char* a = (char*)arena_;
  double* co = (double*)(a + o_co);
  vphi_ = co; vol_ = co + n; tx_ = co + 2 * n; dx_ = co + 3 * n; ty_ = co + 4 * n; dy_ = co + 5 * n;
  double* rw = (double*)(a + o_row);
  qin_ = rw; qin0_ = rw + rows; vphi_r_ = rw + 2 * rows;
  double* st = (double*)(a + o_st);
  p_ = st; c_ = st + n; c_old_ = st + 2 * n; p_prev_ = st + 3 * n;
  J_ = (double*)(a + o_J);
  b_ = (double*)(a + o_bx);
  x_ = b_ + 2 * n;
  for (int k = 0; k < 6; ++k) kv_[k] = (double*)(a + o_kv) + 2 * k * n;
  kS_ = (double*)(a + o_ks);
  kpart_ = (double*)(a + o_kp);
  partial_ = (double*)(a + o_pa);
  res0_ = (double*)(a + o_s8);
  res_last_ = res0_ + B;
  int* i4 = (int*)(a + o_i4);
  active_ = i4; it_step_ = i4 + B; status_w_ = i4 + 2 * B; iters_w_ = i4 + 3 * B;
  n_active_ = (int*)(a + o_misc);
  acc_ = (unsigned int*)(a + o_misc + 16);
  step_ = (int*)(a + o_misc + 40);
  counter_ = (unsigned long long*)(a + o_misc + 48);
  VCK(cudaMemcpy(counter_, &count, sizeof(count), cudaMemcpyHostToDevice));
  cap_ = B;
  return HENRY_OK;
}

// One BiCGStab solve of the row-scaled system on b (x = correction),
// right-preconditioned by `sweeps_` red-black Gauss-Seidel sweeps from zero.
void VcSolver::enqueue_linear(int B, cudaStream_t s) {
  const int n2 = 2 * G_.ncell();
  const int gv = grid1((int64_t)B * n2);
  double *r = kv_[0], *rh = kv_[1], *pv = kv_[2], *v = kv_[3], *t = kv_[4], *xk = kv_[5];
  const dim3 gd(kry_nchunk_, B);
  const int gs = grid1(B);
  const int gh = grid1((int64_t)B * G_.half());
  auto upd = [&](int op) {
    k_kry_update<double><<<gv, kBlock, 0, s>>>(counter_, n2, B, op, active_, kS_, r, rh, pv, v, t,
                                               xk, b_, x_);
  };
  auto precond = [&]() {
    for (int k = 0; k < sweeps_; ++k)
      for (int col = 0; col < 2; ++col)
        k_smooth<double><<<gh, kBlock, 0, s>>>(counter_, G_, B, col, active_, J_, b_, x_);
  };
  upd(0);
  for (int it = 0; it < kry_; ++it) {
    k_kry_dot<double><<<gd, kBlock, 0, s>>>(counter_, n2, B, active_, rh, r, nullptr, nullptr, kpart_);
    k_kry_scalars<<<gs, kBlock, 0, s>>>(counter_, B, kry_nchunk_, 0, active_, kpart_, kS_);
    upd(1);
    precond();
    k_kry_matvec<double><<<grid1((int64_t)B * G_.ncell()), kBlock, 0, s>>>(counter_, G_, B, active_,
                                                                        J_, x_, v);
    k_kry_dot<double><<<gd, kBlock, 0, s>>>(counter_, n2, B, active_, rh, v, nullptr, nullptr, kpart_);
    k_kry_scalars<<<gs, kBlock, 0, s>>>(counter_, B, kry_nchunk_, 1, active_, kpart_, kS_);
    upd(2);
    precond();
    k_kry_matvec<double><<<grid1((int64_t)B * G_.ncell()), kBlock, 0, s>>>(counter_, G_, B, active_,
                                                                        J_, x_, t);
    k_kry_dot<double><<<gd, kBlock, 0, s>>>(counter_, n2, B, active_, t, r, t, t, kpart_);
    k_kry_scalars<<<gs, kBlock, 0, s>>>(counter_, B, kry_nchunk_, 2, active_, kpart_, kS_);
    upd(3);
  }
  upd(4);
}

int VcSolver::run(const double* xi, int B, double* q, double* c_out, double* p_out, int* status,
                  int* iters, int status_or, cudaStream_t s) {
  if (B == 0) return HENRY_OK;
  int rc = ensure(B);
  if (rc) return rc;
  const int n = G_.ncell();
  const int gn = grid1((int64_t)B * n);
  const bool paper = cfg_.field_model == 1;
  k_vc_coeffs<<<gn, kBlock, 0, s>>>(counter_, phys_, G_, B, cfg_.n_xi, cfg_.field_model, xi, vphi_,
                                    vol_, tx_, dx_, ty_, dy_, paper ? qin0_ : qin_, vphi_r_,
                                    status_w_);
  k_vc_init<<<gn, kBlock, 0, s>>>(counter_, phys_, G_, B, p_, c_, iters_w_, step_);
  const double scale = tau_ / (G_.hx * G_.hy * cfg_.phi0 * cfg_.rho0);
  const dim3 gr(nchunk_, B);
  for (int stp = 0; stp < nt_; ++stp) {
    k_begin_step<<<gn, kBlock, 0, s>>>(counter_, G_, B, p_, c_, p_prev_, c_old_, status_w_,
                                       active_, it_step_, step_, cfg_.guess_extrapolation,
                                       paper ? qin0_ : nullptr, qin_, tau_);
    for (;;) {
      k_vc_resjac<false, true><<<gr, kBlock, 0, s>>>(counter_, phys_, G_, tau_, B, vphi_, vol_,
                                                     tx_, dx_, ty_, dy_, qin_, p_, c_, c_old_,
                                                     active_, J_, b_, x_, partial_);
      k_check<false><<<(B + 7) / 8, kBlock, 0, s>>>(
          counter_, B, nchunk_, n, partial_, scale, cfg_.newton_rtol, cfg_.newton_atol,
          cfg_.newton_maxit, active_, it_step_, res0_, res_last_, status_w_, iters_w_, n_active_,
          acc_, cfg_.newton_stag_tol, 0, nullptr, 0);
      VCK(cudaMemcpyAsync(host_, n_active_, sizeof(int), cudaMemcpyDeviceToHost, s));
      VCK(cudaStreamSynchronize(s));
      if (host_[0] == 0) break;
      enqueue_linear(B, s);
      k_update<double><<<gn, kBlock, 0, s>>>(counter_, G_, B, active_, x_, p_, c_);
    }
    k_end_step<<<1, 32, 0, s>>>(counter_, step_);
  }
  k_vc_qoi<<<B, kBlock, 0, s>>>(counter_, phys_, G_, B, p_, c_, vphi_, vphi_r_, q, c_out, p_out);
  k_vc_copy_int<<<grid1(B), kBlock, 0, s>>>(counter_, B, status_w_, status, status_or);
  if (iters) k_vc_copy_int<<<grid1(B), kBlock, 0, s>>>(counter_, B, iters_w_, iters, 0);
  VCK(cudaGetLastError());
  return HENRY_OK;
}

cudaError_t launch_vc_residual_jacobian(const Phys& P, int nx, int ny, int model, int n_xi,
                                        double tau, int B, const double* xi, const double* p,
                                        const double* c, const double* c_old, double* R,
                                        double* J, double* scratch, cudaStream_t s) {
  const Geom G{nx, ny + 1, P.Lx / nx, P.Ly / ny};
  const int64_t n = (int64_t)B * G.ncell(), rows = (int64_t)B * G.ny;
  double* co = scratch;   // vphi vol tx dx ty dy [n] each, reduced p [n], qin vphi_r [rows]
  double *vphi = co, *vol = co + n, *tx = co + 2 * n, *dx = co + 3 * n, *ty = co + 4 * n,
         *dy = co + 5 * n, *pr = co + 6 * n, *qin = co + 7 * n, *vr = co + 7 * n + rows;
  const int gn = (int)((n + kBlock - 1) / kBlock);
  k_vc_coeffs<<<gn, kBlock, 0, s>>>(nullptr, P, G, B, n_xi, model, xi, vphi, vol, tx, dx, ty, dy, qin,
                                    vr, nullptr);
  k_vc_reduce_pressure<<<gn, kBlock, 0, s>>>(P, G, B, p, pr);
  const dim3 gr((G.ncell() + kBlock - 1) / kBlock, B);
  if (J)
    k_vc_resjac<true, true><<<gr, kBlock, 0, s>>>(nullptr, P, G, tau, B, vphi, vol, tx, dx, ty, dy,
                                                  qin, pr, c, c_old, nullptr, J, R, nullptr, nullptr);
  else
    k_vc_resjac<true, false><<<gr, kBlock, 0, s>>>(nullptr, P, G, tau, B, vphi, vol, tx, dx, ty, dy,
                                                   qin, pr, c, c_old, nullptr, nullptr, R, nullptr,
                                                   nullptr);
  return cudaGetLastError();
}

}  // namespace henry
