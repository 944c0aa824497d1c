// Device-side per-node arithmetic of the time step (sm_103a).
//
// The collision is the efficient execution sequence (1)-(6) of the paper's
// supplement Sec. IV, which equals the matrix form of Eq. 13 (supplement Eq. 1)
// up to rounding.  Conserved moments are not relaxed: rho stays, and the
// momentum gains F (their rows of S, R, T, X and Q_m act on zero).
#pragma once

#include <cuda_fp16.h>

#include "lbm_internal.h"

namespace lbm {

// Storage <-> compute conversions.
__device__ __forceinline__ float ld_st(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ld_st(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_st(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void st_st(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_st(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_st(__half* p, float v) { *p = __float2half_rn(v); }

template <typename real>
__device__ __forceinline__ real rcp(real x) {
  return real(1) / x;
}

// p_EOS / c^2 and d(p_EOS/c^2)/drho.  vdW: rho R T/(1 - b rho) - a rho^2;
// Carnahan-Starling (Eq. 20) with t = b rho / 4.  Both times K_EOS / c^2.
template <typename real>
__device__ __forceinline__ void eos(const Coef<real>& c, real rho, real& pe, real& dpe) {
  if (c.eos == LB_EOS_VDW) {
    const real io = rcp(real(1) - c.bq * rho);
    const real rt_io = c.RT * io;
    pe = c.lam * (rho * rt_io - c.a * rho * rho);
    dpe = c.lam * (rt_io * io - real(2) * c.a * rho);
  } else {
    const real t = c.bq * rho;
    const real io = rcp(real(1) - t);
    const real io3 = io * io * io;
    const real t2 = t * t;
    const real z = (real(1) + t + t2 - t2 * t) * io3;
    const real dz = (real(1) + real(4) * t + real(4) * t2 - real(4) * t2 * t + t2 * t2) * io3 * io;
    pe = c.lam * (rho * c.RT * z - c.a * rho * rho);
    dpe = c.lam * (c.RT * dz - real(2) * c.a * rho);
  }
}

// One node.  d: post-streaming populations stored as deviations f_i - w_i rho_ref;
// (Sx, Sy) = sum_i omega_i rho(x + e_i) e_i (Eq. 12, = grad rho of supplement
// Eq. 61); o: post-collision deviations.
template <typename real>
__device__ __forceinline__ void collide(const Coef<real>& c, const real (&d)[9], real Sx, real Sy,
                                        real (&o)[9]) {
  // Moment transform (supplement Eq. 4) with shared sums; M w = (1, -2, 1, 0, ...).
  const real a13 = d[1] + d[3], a24 = d[2] + d[4], a57 = d[5] + d[7], a68 = d[6] + d[8];
  const real s13 = d[1] - d[3], s24 = d[2] - d[4], s57 = d[5] - d[7], s68 = d[6] - d[8];
  const real axis = a13 + a24, diag = a57 + a68;
  const real rho_dev = d[0] + axis + diag;
  const real rho = rho_dev + c.rho_ref;
  const real m1 = real(-4) * d[0] - axis + real(2) * diag - real(2) * c.rho_ref;
  const real m2 = real(4) * d[0] - real(2) * axis + diag + c.rho_ref;
  const real jx = s13 + s57 - s68;
  const real jy = s24 + s57 + s68;
  const real m4 = real(-2) * s13 + s57 - s68;
  const real m6 = real(-2) * s24 + s57 + s68;
  const real m7 = a13 - a24;
  const real m8 = a57 - a68;

  // Interaction force (Eq. 12) and velocity (Eq. 5), c = 1.
  const real Fx = c.G2 * rho * Sx, Fy = c.G2 * rho * Sy;
  const real inv_rho = rcp(rho);
  const real ux = (jx + real(0.5) * Fx) * inv_rho;
  const real uy = (jy + real(0.5) * Fy) * inv_rho;

  // Self-tuning EOS: p_LBE = p_EOS + G^2 rho^2/2 (Eq. 18) = c_s^2 (rho + eta);
  // grad p_LBE = (p_EOS' + G^2 rho) grad rho (supplement Eq. 61).
  real pe, dpe;
  eos(c, rho, pe, dpe);
  const real eta = real(3) * (pe + real(0.5) * c.G2 * rho * rho) - rho;
  const real g = dpe + c.G2 * rho;

  const real x2 = ux * ux, y2 = uy * uy, xy = ux * uy, u2 = x2 + y2;
  // Equilibrium (Eq. 3, alpha_1 = -1, beta_1 = 1, alpha_2 = 1), non-conserved rows.
  const real meq1 = real(-2) * rho + real(2) * eta + real(3) * rho * u2;
  const real meq2 = rho + c.beta2 * eta - real(3) * rho * u2 + real(9) * rho * x2 * y2;
  const real meq4 = rho * ux * (real(3) * y2 - real(1));
  const real meq6 = rho * uy * (real(3) * x2 - real(1));
  const real meq7 = rho * (x2 - y2);
  const real meq8 = rho * xy;
  // Forcing (Eq. 4), brackets summed over the force's positions.
  const real Fu = Fx * ux + Fy * uy;
  const real Fm1 = real(6) * Fu;
  const real Fm2 = real(-6) * Fu + real(18) * xy * (Fx * uy + Fy * ux);
  const real Fm4 = -Fx + real(3) * (Fx * y2 + real(2) * Fy * xy);
  const real Fm6 = -Fy + real(3) * (real(2) * Fx * xy + Fy * x2);
  const real Fm7 = real(2) * (Fx * ux - Fy * uy);
  const real Fm8 = Fx * uy + Fy * ux;

  // (1): mbar = 2 m_eq - m ; G = m - m_eq + F_m / 2.
  real mb1 = real(2) * meq1 - m1, mb2 = real(2) * meq2 - m2, mb4 = real(2) * meq4 - m4;
  real mb6 = real(2) * meq6 - m6, mb7 = real(2) * meq7 - m7, mb8 = real(2) * meq8 - m8;
  const real G1 = m1 - meq1 + real(0.5) * Fm1, G2 = m2 - meq2 + real(0.5) * Fm2;
  const real G4 = m4 - meq4 + real(0.5) * Fm4, G6 = m6 - meq6 + real(0.5) * Fm6;
  const real G7 = m7 - meq7 + real(0.5) * Fm7, G8 = m8 - meq8 + real(0.5) * Fm8;
  // (2) off-diagonal part of S, then (3) I - diag(S)/2.
  const real A1 = c.om_e * (G1 + c.hk_seps * G2 + c.hh_sq * (ux * G4 + uy * G6));
  const real A2 = c.om_eps * G2;
  const real A4 = c.om_q * G4, A6 = c.om_q * G6;
  const real A7 = c.om_p * (G7 + c.b_sq * (ux * G4 - uy * G6));
  const real A8 = c.om_p * (G8 + c.hb_sq * (uy * G4 + ux * G6));
  // (4) cubic-velocity correction: R (I - S/2) G + T . grad rho + X . grad p_LBE.
  const real ax = x2 * ux * Sx, ay = y2 * uy * Sy;
  const real cr1 = c.T1a * (ax + ay) + (g * c.X1 - c.T1b) * xy * (uy * Sx + ux * Sy);
  const real cr7 = c.T7 * (ax - ay) + (c.T7b + g * c.X7) * xy * (uy * Sx - ux * Sy);
  const real cr8 = (c.T8 + g * c.X8) * ((y2 + real(2) * x2) * uy * Sx + (x2 + real(2) * y2) * ux * Sy);
  mb1 -= c.R11 * u2 * A1 + c.R17 * (x2 - y2) * A7 + c.R18 * xy * A8 + cr1;
  mb7 -= c.R71 * (x2 - y2) * A1 + c.R77 * u2 * A7 + cr7;
  mb8 -= c.R81 * xy * A1 + c.R88 * u2 * A8 + cr8;
  // (5)
  mb1 += real(2) * A1;
  mb2 += real(2) * A2;
  mb4 += real(2) * A4;
  mb6 += real(2) * A6;
  mb7 += real(2) * A7;
  mb8 += real(2) * A8;
  // (6) S Q_m with |F~|^2 = G^2 |S|^2 (Eq. 14).
  const real sxx = Sx * Sx, syy = Sy * Sy;
  mb1 += c.Q1 * c.G2 * (sxx + syy);
  mb2 += c.Q2 * c.G2 * (sxx + syy);
  mb7 += c.Q78 * c.G2 * (sxx - syy);
  mb8 += c.Q78 * c.G2 * Sx * Sy;

  // Inverse transform M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4),
  // applied to mbar - rho_ref M w (deviation storage); conserved: rho, j + F.
  const real n0 = rho_dev * real(1.0 / 9.0);
  const real n1 = (mb1 + real(2) * c.rho_ref) * real(1.0 / 36.0);
  const real n2 = (mb2 - c.rho_ref) * real(1.0 / 36.0);
  const real n3 = (jx + Fx) * real(1.0 / 6.0);
  const real n4 = mb4 * real(1.0 / 12.0);
  const real n5 = (jy + Fy) * real(1.0 / 6.0);
  const real n6 = mb6 * real(1.0 / 12.0);
  const real n7 = mb7 * real(0.25);
  const real n8 = mb8 * real(0.25);
  const real base_a = n0 - n1 - real(2) * n2, base_d = n0 + real(2) * n1 + n2;
  const real px = n3 - real(2) * n4, py = n5 - real(2) * n6;
  const real qx = n3 + n4, qy = n5 + n6;
  o[0] = n0 - real(4) * n1 + real(4) * n2;
  o[1] = base_a + px + n7;
  o[2] = base_a + py - n7;
  o[3] = base_a - px + n7;
  o[4] = base_a - py - n7;
  o[5] = base_d + qx + qy + n8;
  o[6] = base_d - qx + qy - n8;
  o[7] = base_d - qx - qy + n8;
  o[8] = base_d + qx - qy - n8;
}

// Force stencil of Eq. 12 from the densities of the 8 neighbours
// (r_<row><col>: row m/c/p = y-1/y/y+1, col l/r = x-1/x+1).
template <typename real>
__device__ __forceinline__ void stencil(real r_ml, real r_mc, real r_mr, real r_cl, real r_cr, real r_pl,
                                        real r_pc, real r_pr, real& Sx, real& Sy) {
  const real third = real(1.0 / 3.0), twelfth = real(1.0 / 12.0);
  Sx = third * (r_cr - r_cl) + twelfth * ((r_pr - r_pl) + (r_mr - r_ml));
  Sy = third * (r_pc - r_mc) + twelfth * ((r_pr + r_pl) - (r_mr + r_ml));
}

}  // namespace lbm
