// Device-side discretisation of the Henry problem (arxiv 2403.17018,
// section 2.1, Eqs. 1-5; section 2.3 implicit Euler).
//
// Cell-centred finite volumes on [0,Lx] x [0,Ly] (y upward). For the face
// between a lower cell L (west or south) and an upper cell U (east or north)
// with unit vector e from L to U, area A and centre distance d:
//   q     = -(K_f/mu) [ (p_U - p_L)/d + rho_bar g e_y ]         (Eq. 3)
//   F_m   = A q rho_up                                          (Eq. 1 flux)
//   F_s   = A [ q (rho c)_up - rho_bar phi_f D (c_U - c_L)/d ]  (Eq. 2 flux, Eq. 5)
// K_f, phi_f harmonic means, rho_bar arithmetic mean of rho(c) (Eq. 4),
// upwind from L when q >= 0, else from U. Both cells evaluate a face with the
// same canonical orientation and the same operations, so the two residual
// contributions cancel exactly in floating point.
// Boundaries: left x=0 prescribed mass inflow rho0 q_in(y), no advected salt,
// diffusive Dirichlet c=0 at hx/2; right x=Lx Dirichlet p = rho1 g (Ly - y)
// at hx/2, advected values upwinded with c=1 on inflow, diffusive Dirichlet
// c=1 at hx/2; top and bottom no flux.
// Accumulation per cell: V phi (rho - rho_old)/tau and V phi (rho c -
// rho_old c_old)/tau.
//
// Pressure unknown: the kernels carry the reduced pressure
//   p' = p - rho0 g (Ly - y)
// (the fresh-water hydrostatic part removed), so the gravity term of a
// vertical face becomes (rho_bar - rho0) g d = 0.5 (rho1 - rho0)(c_L + c_U) g d
// and the Dirichlet value on the right side (rho1 - rho0) g (Ly - y). This
// is the same discrete equation as with p, but without the cancellation of
// two ~rho0 g d terms in every vertical face flux, which lowers the rounding
// floor of the FP64 residual by about (rho0 / (rho1 - rho0)) = 40x.
//
// Face constants are precomputed once per solve (the fields do not change in
// time): tx = A_x K_f / (mu hx), dx = A_x phi_f D / hx for the east face of a
// cell, ty, dy likewise for its north face. This keeps divisions out of the
// per-iteration FP64 work.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace henry {

struct Phys {
  double rho0, drho, mu, g, D, K0, phi0, q0, Lx, Ly;
  double rho1() const { return rho0 + drho; }
};

struct Geom {
  int nx, ny;        // cells
  double hx, hy;     // cell sizes
  __host__ __device__ int ncell() const { return nx * ny; }
  __host__ __device__ int half() const { return (nx * ny) >> 1; }
};

// Previous states beyond u^(n-1) for the extrapolated Newton guess of the
// implicit steps (see k_begin_step): p[k], c[k] hold u^(n-2-k).
constexpr int kMaxGuessHist = 5;   // guess orders up to 6
struct GuessHist {
  double* p[kMaxGuessHist];
  double* c[kMaxGuessHist];
  int depth;                       // arrays in use
};

// Tiling of the temporally blocked multigrid legs (see k_tb_down, k_tb_up).
constexpr int kTbBlock = 1024;
constexpr int kTbTileX = 64, kTbTileY = 32;   // interior cells of a tile, at most

constexpr size_t kMaxSmemOptin = 232448;        // 227 KB per block

struct TbTile {
  int TX, TY;    // interior cells per tile (even)
  int ntx, nty;  // tiles per sample
  int H;         // halo rows (the halo columns are H rounded up to even)
  int EX, EY;    // largest extended tile, for the shared-memory size
  int staged;    // 1: one tile per sample whose operator planes, right-hand
                 // side and unknowns all fit in shared memory
  int cl;        // > 1: staged in strips by a cluster of cl blocks per sample
  size_t smem;   // dynamic shared memory of the launch (per block)
};

// Tiles of at most tx x ty cells (both even) with a halo of 2 nu + extra;
// nplanes operator planes (from plane 4) are staged when the whole sample
// is one tile and fits.
inline TbTile make_tb_tile(const Geom& G, int nu, int extra, int tx, int ty, int nplanes,
                           size_t tsize) {
  TbTile t;
  t.TX = tx < G.nx ? tx : G.nx;
  t.TY = ty < G.ny ? ty : G.ny;
  t.ntx = (G.nx + t.TX - 1) / t.TX;
  t.nty = (G.ny + t.TY - 1) / t.TY;
  t.H = 2 * nu + extra;
  const int hx = (t.H + 1) & ~1;
  t.EX = t.TX + 2 * hx < G.nx ? t.TX + 2 * hx : G.nx;
  t.EY = t.TY + 2 * t.H < G.ny ? t.TY + 2 * t.H : G.ny;
  const size_t staged = 16 + (size_t)(nplanes + 4) * G.ncell() * tsize;
  t.staged = t.ntx == 1 && t.nty == 1 && staged <= kMaxSmemOptin;
  t.cl = 0;
  t.smem = t.staged ? staged : (size_t)2 * t.EX * t.EY * tsize;
  // otherwise strips of an even number of rows, one block each, in a
  // cluster of at most 8 blocks (the portable cluster size)
  for (int cl = 2; !t.staged && cl <= 8; cl *= 2) {
    const size_t strip = 16 + (size_t)(nplanes + 4) * (G.ncell() / cl) * tsize;
    if (G.ny % (2 * cl) == 0 && (G.nx >> 1) % 2 == 0 && strip <= kMaxSmemOptin) {
      t.cl = cl;
      t.smem = strip;
      break;
    }
  }
  return t;
}

// Colour-split position of cell (i, j) inside one plane: red cells
// ((i + j) even) first, then black, each in row-major order of (j, i/2).
// Requires nx even.
__device__ __forceinline__ int cs_pos(int i, int j, int nx, int half) {
  return (((i + j) & 1) ? half : 0) + j * (nx >> 1) + (i >> 1);
}

// Per-face flux and its derivatives with respect to (p, c) of L and U.
template <typename JT>
struct FaceD {
  JT mLp, mLc, mUp, mUc;   // d F_m / d (p_L, c_L, p_U, c_U)
  JT sLp, sLc, sUp, sUc;   // d F_s / d (p_L, c_L, p_U, c_U)
};

// Interior face. t = A K_f/(mu d), dco = A phi_f D / d, gd = g e_y d.
// q is the area-weighted face flux A q.n: computed from p unless Q_GIVEN, in
// which case the caller supplies it (coarse multigrid levels linearise about
// the restricted fine-level flux field) and the pressures are not used.
// VERT: a vertical (south-north) face, the only kind with a gravity term;
// horizontal faces skip it (and its derivative) instead of multiplying by a
// zero gd.
template <typename JT, bool WANT_J, bool Q_GIVEN, bool VERT>
__device__ __forceinline__ void face_flux(const Phys& P, double pL, double cL, double pU, double cU,
                                          double t, double dco, double gd, double& q,
                                          double& Fm, double& Fs, FaceD<JT>& J) {
  const double rL = P.rho0 + P.drho * cL;
  const double rU = P.rho0 + P.drho * cU;
  const double rbar = 0.5 * (rL + rU);
  if (!Q_GIVEN) q = VERT ? -t * ((pU - pL) + (0.5 * P.drho) * (cL + cU) * gd) : -t * (pU - pL);
  const bool up = q >= 0.0;
  const double rup = up ? rL : rU;
  const double rcup = up ? rL * cL : rU * cU;
  const double dc = cU - cL;
  Fm = q * rup;
  Fs = q * rcup - dco * rbar * dc;
  if (WANT_J) {
    // Jacobian entries in the multigrid type from five converted values (on
    // GB300 a conversion costs an FP64-pipe slot, like an FP64 operation)
    const JT t_ = (JT)t, q_ = (JT)q, dco_ = (JT)dco, cL_ = (JT)cL, cU_ = (JT)cU;
    const JT dr = (JT)P.drho, r0 = (JT)P.rho0;
    const JT rL_ = r0 + dr * cL_, rU_ = r0 + dr * cU_;
    const JT rup_ = up ? rL_ : rU_;
    const JT rcup_ = up ? rL_ * cL_ : rU_ * cU_;
    const JT diffc = -dco_ * (JT)0.5 * dr * (cU_ - cL_);   // d(-dco rbar dc)/dc from rbar
    const JT drb = dco_ * (JT)0.5 * (rL_ + rU_);
    J.mLp = t_ * rup_;
    J.mUp = -t_ * rup_;
    J.mLc = up ? q_ * dr : (JT)0;
    J.mUc = up ? (JT)0 : q_ * dr;
    J.sLp = t_ * rcup_;
    J.sUp = -t_ * rcup_;
    J.sLc = (up ? q_ * (rL_ + dr * cL_) : (JT)0) + diffc + drb;
    J.sUc = (up ? (JT)0 : q_ * (rU_ + dr * cU_)) + diffc - drb;
    if (VERT) {
      const JT s_ = -t_ * (JT)gd * (JT)0.5 * dr;       // dq/dc_L = dq/dc_U
      J.mLc += s_ * rup_;
      J.mUc += s_ * rup_;
      J.sLc += s_ * rcup_;
      J.sUc += s_ * rcup_;
    }
  }
}

// Right side (x = Lx, outward +x): flux from P to the seawater boundary and
// its derivatives with respect to (p_P, c_P). tR = 2 A K_P / (mu hx),
// dco = 2 A phi_P D / hx, pb = reduced Dirichlet pressure.
template <typename JT, bool WANT_J, bool Q_GIVEN>
__device__ __forceinline__ void right_face(const Phys& P, double p, double c, double tR, double dco,
                                           double pb, double& q, double& Fm, double& Fs, JT* jd) {
  const double rho = P.rho0 + P.drho * c;
  const double rho1 = P.rho0 + P.drho;
  if (!Q_GIVEN) q = -tR * (pb - p);
  const bool up = q >= 0.0;
  const double rup = up ? rho : rho1;
  const double rcup = up ? rho * c : rho1;
  const double rb = 0.5 * (rho + rho1);
  Fm = q * rup;
  Fs = q * rcup - dco * rb * (1.0 - c);
  if (WANT_J) {
    jd[0] = (JT)(tR * rup);
    jd[1] = (JT)(up ? q * P.drho : 0.0);
    jd[2] = (JT)(tR * rcup);
    jd[3] = (JT)((up ? q * (rho + P.drho * c) : 0.0) - dco * 0.5 * P.drho * (1.0 - c) + dco * rb);
  }
}

// Inputs of one cell's residual/Jacobian evaluation, gathered by the caller.
struct CellIn {
  double p, c, c_old, phi, K;       // own values (K used on the right side only)
  double pW, cW, pE, cE, pS, cS, pN, cN;
  double tW, dW, tE, dE, tS, dS, tN, dN;   // face constants (valid where the face exists)
  double qin;                        // left inflow velocity of this row (i == 0)
  double qW, qE, qS, qN;             // face fluxes A q.n (qE: right side when i == nx-1);
                                     // outputs, or inputs when Q_GIVEN
  bool hasW, hasE, hasS, hasN;       // interior faces
  double y;                          // cell-centre y (right boundary pressure)
};

// Residual (FP64) and, optionally, the 20 Jacobian entries of one cell;
// vtau = cell volume / time step:
// J[0..3] = dR_P/du_P, J[4..7] W, J[8..11] E, J[12..15] S, J[16..19] N;
// each block (pp, pc, cp, cc), row = equation, column = variable.
template <typename JT, bool WANT_J, bool Q_GIVEN = false>
__device__ __forceinline__ void cell_residual(const Phys& P, const Geom& G, double vtau,
                                              CellIn& in, double& Rp, double& Rc, JT* J) {
  const double vt = vtau * in.phi;
  const double rho = P.rho0 + P.drho * in.c;
  const double rho_o = P.rho0 + P.drho * in.c_old;
  Rp = vt * (rho - rho_o);
  Rc = vt * (rho * in.c - rho_o * in.c_old);
  if (WANT_J) {
#pragma unroll
    for (int m = 0; m < 20; ++m) J[m] = (JT)0;
    J[1] = (JT)(vt * P.drho);
    J[3] = (JT)(vt * (rho + P.drho * in.c));
  }
  FaceD<JT> d;
  double Fm, Fs;
  const double gdy = P.g * G.hy;
  // west face: L = W, U = P; contributes -F to P
  if (in.hasW) {
    face_flux<JT, WANT_J, Q_GIVEN, false>(P, in.pW, in.cW, in.p, in.c, in.tW, in.dW, 0.0, in.qW, Fm, Fs, d);
    Rp -= Fm;
    Rc -= Fs;
    if (WANT_J) {
      J[0] -= d.mUp; J[1] -= d.mUc; J[2] -= d.sUp; J[3] -= d.sUc;
      J[4] = -d.mLp; J[5] = -d.mLc; J[6] = -d.sLp; J[7] = -d.sLc;
    }
  } else {
    // left side: fixed freshwater mass inflow, diffusion to c = 0 at hx/2
    const double A = G.hy;
    const double dco = 2.0 * A * in.phi * P.D / G.hx;
    const double rb = 0.5 * (rho + P.rho0);
    Rp += -A * P.rho0 * in.qin;
    Rc += dco * rb * in.c;
    if (WANT_J) J[3] += (JT)(dco * (0.5 * P.drho * in.c + rb));
  }
  // east face: L = P, U = E; contributes +F to P
  if (in.hasE) {
    face_flux<JT, WANT_J, Q_GIVEN, false>(P, in.p, in.c, in.pE, in.cE, in.tE, in.dE, 0.0, in.qE, Fm, Fs, d);
    Rp += Fm;
    Rc += Fs;
    if (WANT_J) {
      J[0] += d.mLp; J[1] += d.mLc; J[2] += d.sLp; J[3] += d.sLc;
      J[8] = d.mUp; J[9] = d.mUc; J[10] = d.sUp; J[11] = d.sUc;
    }
  } else {
    // right side: hydrostatic seawater, Dirichlet at hx/2
    const double A = G.hy;
    const double rho1 = P.rho0 + P.drho;
    const double tR = 2.0 * A * in.K / (P.mu * G.hx);
    const double dco = 2.0 * A * in.phi * P.D / G.hx;
    const double pb = P.drho * P.g * (P.Ly - in.y);   // reduced pressure
    if (!Q_GIVEN) in.qE = -tR * (pb - in.p);
    const double q = in.qE;
    const bool up = q >= 0.0;
    const double rup = up ? rho : rho1;
    const double rcup = up ? rho * in.c : rho1;
    const double rb = 0.5 * (rho + rho1);
    Rp += q * rup;
    Rc += q * rcup - dco * rb * (1.0 - in.c);
    if (WANT_J) {
      J[0] += (JT)(tR * rup);
      J[1] += (JT)(up ? q * P.drho : 0.0);
      J[2] += (JT)(tR * rcup);
      J[3] += (JT)((up ? q * (rho + P.drho * in.c) : 0.0)
                   - dco * 0.5 * P.drho * (1.0 - in.c) + dco * rb);
    }
  }
  // south face: L = S, U = P (e = +y); contributes -F
  if (in.hasS) {
    face_flux<JT, WANT_J, Q_GIVEN, true>(P, in.pS, in.cS, in.p, in.c, in.tS, in.dS, gdy, in.qS, Fm, Fs, d);
    Rp -= Fm;
    Rc -= Fs;
    if (WANT_J) {
      J[0] -= d.mUp; J[1] -= d.mUc; J[2] -= d.sUp; J[3] -= d.sUc;
      J[12] = -d.mLp; J[13] = -d.mLc; J[14] = -d.sLp; J[15] = -d.sLc;
    }
  }
  // north face: L = P, U = N; contributes +F
  if (in.hasN) {
    face_flux<JT, WANT_J, Q_GIVEN, true>(P, in.p, in.c, in.pN, in.cN, in.tN, in.dN, gdy, in.qN, Fm, Fs, d);
    Rp += Fm;
    Rc += Fs;
    if (WANT_J) {
      J[0] += d.mLp; J[1] += d.mLc; J[2] += d.sLp; J[3] += d.sLc;
      J[16] = d.mUp; J[17] = d.mUc; J[18] = d.sUp; J[19] = d.sUc;
    }
  }
}

// Gather the stencil of cell (i, j) from natural-layout arrays of one sample.
// tx/dx hold east-face constants, ty/dy north-face constants.
__device__ __forceinline__ void gather_cell(const Geom& G, int i, int j, const double* __restrict__ p,
                                            const double* __restrict__ c, const double* __restrict__ phi,
                                            const double* __restrict__ K, const double* __restrict__ tx,
                                            const double* __restrict__ dx, const double* __restrict__ ty,
                                            const double* __restrict__ dy, CellIn& in) {
  const int nx = G.nx;
  const int id = j * nx + i;
  in.p = p[id];
  in.c = c[id];
  in.phi = phi[id];
  in.hasW = i > 0;
  in.hasE = i < nx - 1;
  in.hasS = j > 0;
  in.hasN = j < G.ny - 1;
  in.K = in.hasE ? 0.0 : K[id];
  in.y = (j + 0.5) * G.hy;
  if (in.hasW) { in.pW = p[id - 1]; in.cW = c[id - 1]; in.tW = tx[id - 1]; in.dW = dx[id - 1]; }
  if (in.hasE) { in.pE = p[id + 1]; in.cE = c[id + 1]; in.tE = tx[id]; in.dE = dx[id]; }
  if (in.hasS) { in.pS = p[id - nx]; in.cS = c[id - nx]; in.tS = ty[id - nx]; in.dS = dy[id - nx]; }
  if (in.hasN) { in.pN = p[id + nx]; in.cN = c[id + nx]; in.tN = ty[id]; in.dN = dy[id]; }
}

// Random fields at the point (x, y) (frame y in [0, Ly]) for one sample's
// random vector z (see henry.h, henry_fields): porosity and permeability,
// with the log-K perturbation lk when has_lk. model 1: the paper's
// two-layer porosity (Eq. poro_2levels, in its frame y_p = y - Ly) and
// Kozeny-Carman K with kappa = K0 (1 - phi0^2) / phi0^3 (Eq.
// e_perm_Kozeny_Carman); model 0: the smooth fields of 3 or 6 variables.
__device__ __forceinline__ void field_at(const Phys& P, int model, int n_xi, const double* z,
                                         double x, double y, bool has_lk, double lk, double& phi,
                                         double& K) {
  const double pi = 3.14159265358979323846;
  if (model == 1) {
    const double yp = y - P.Ly;
    const double c0 = yp < -0.8 ? 1.2 * (1.0 + 0.2 * z[0]) : 1.0;
    const double c1 = 1.0 + 0.15 * (z[1] * cos(pi * x / 2) - z[1] * sin(2 * pi * yp) +
                                    z[0] * cos(2 * pi * x));
    const double c2 = 1.0 + 0.2 * (z[0] * sin(64 * pi * x) + z[1] * sin(32 * pi * yp));
    phi = P.phi0 * c0 * c1 * c2;
    const double kappa = P.K0 * (1.0 - P.phi0 * P.phi0) / (P.phi0 * P.phi0 * P.phi0);
    K = kappa * (phi * phi * phi) / (1.0 - phi * phi);
    if (has_lk) K *= exp(lk);
    return;
  }
  double a = 0.1 * z[0] * cos(0.5 * pi * x) * sin(pi * y);
  double e = 0.5 * z[1] * sin(0.5 * pi * x) * cos(pi * y);
  if (n_xi >= 6) {
    a += 0.05 * z[3] * cos(pi * x) * sin(2.0 * pi * y);
    e += 0.05 * z[4] * sin(pi * x) * cos(2.0 * pi * y);
  }
  if (has_lk) e += lk;
  phi = P.phi0 * (1.0 + a);
  K = P.K0 * exp(e);
}

// Left-side inflow velocity at height y (model 1: the base of Eq.
// e_recharge_of_param, its time factor applied per step).
__device__ __forceinline__ double inflow_at(const Phys& P, int model, int n_xi, const double* z,
                                            double y) {
  if (model == 1) return P.q0 * (1.0 + 0.5 * z[2]);
  double qf = 1.0 + 0.1 * z[2];
  if (n_xi >= 6) qf += 0.05 * z[5] * cos(3.14159265358979323846 * y);
  return P.q0 * qf;
}

// Face constants of cell (i, j): east face (if any) and north face (if any).
// The last column's east slots hold the right side's coefficients, 2 A K_P
// / (mu hx) and 2 A phi_P D / hx (the Dirichlet side at hx/2), for kernels
// that treat the right side as one more face (k_resid); the others compute
// them from K and phi and read tx, dx only where an east neighbour exists.
__device__ __forceinline__ void face_constants(const Phys& P, const Geom& G, int i, int j,
                                               const double* __restrict__ phi,
                                               const double* __restrict__ K, double& tx, double& dx,
                                               double& ty, double& dy) {
  const int id = j * G.nx + i;
  tx = dx = ty = dy = 0.0;
  if (i < G.nx - 1) {
    const double k1 = K[id], k2 = K[id + 1], f1 = phi[id], f2 = phi[id + 1];
    const double Kf = 2.0 * k1 * k2 / (k1 + k2);
    const double ff = 2.0 * f1 * f2 / (f1 + f2);
    tx = G.hy * Kf / (P.mu * G.hx);
    dx = G.hy * ff * P.D / G.hx;
  } else {
    tx = (2.0 * G.hy / (P.mu * G.hx)) * K[id];
    dx = (2.0 * G.hy * P.D / G.hx) * phi[id];
  }
  if (j < G.ny - 1) {
    const double k1 = K[id], k2 = K[id + G.nx], f1 = phi[id], f2 = phi[id + G.nx];
    const double Kf = 2.0 * k1 * k2 / (k1 + k2);
    const double ff = 2.0 * f1 * f2 / (f1 + f2);
    ty = G.hx * Kf / (P.mu * G.hy);
    dy = G.hx * ff * P.D / G.hy;
  }
}

}  // namespace henry
