// Device-side per-node arithmetic of the time step (sm_103a).
//
// The collision is the efficient execution sequence (1)-(6) of the paper's
// supplement Sec. IV, which equals the matrix form of Eq. 13 (supplement Eq. 1)
// up to rounding.  Conserved moments are not relaxed: rho stays, and the
// momentum gains F (their rows of S, R, T, X and Q_m act on zero).
//
// The arithmetic is written once for a value type V: double, float, or f2 = a
// pair of FP32 lanes (two lattice nodes) executed with Blackwell's packed
// FFMA2 / FADD2 / FMUL2 instructions, which halves the instruction count of the
// FP32 collision.  Every constant comes from the Coef<V> block.
#pragma once

#include <cuda_fp16.h>

#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------------------
// Value types.
struct f2 {
  float2 v;
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 fmav(f2 a, f2 b, f2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return {__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
// FP32 reciprocal: the hardware approximation (rcp.approx.ftz, within 1 ulp) when
// LBM_FAST_RCP is set, else the correctly rounded __frcp_rn.  The densities and
// 1 - b rho it inverts are normal numbers far from the flush-to-zero range.
#ifndef LBM_FAST_RCP
#define LBM_FAST_RCP 1
#endif
__device__ __forceinline__ float rcp32(float x) {
#if LBM_FAST_RCP
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return __frcp_rn(x);
#endif
}
__device__ __forceinline__ f2 rcp(f2 x) { return {make_float2(rcp32(x.v.x), rcp32(x.v.y))}; }

__device__ __forceinline__ float fmav(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmav(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rcp(float x) { return rcp32(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// Lanes of a value (1 for scalars, 2 for f2).
template <typename V>
struct Lanes;
template <>
struct Lanes<double> {
  static constexpr int n = 1;
  __device__ static double get(double v, int) { return v; }
  __device__ static void set(double& v, int, double x) { v = x; }
};
template <>
struct Lanes<float> {
  static constexpr int n = 1;
  __device__ static float get(float v, int) { return v; }
  __device__ static void set(float& v, int, float x) { v = x; }
};
template <>
struct Lanes<f2> {
  static constexpr int n = 2;
  __device__ static float get(f2 v, int k) { return k ? v.v.y : v.v.x; }
  __device__ static void set(f2& v, int k, float x) {
    if (k)
      v.v.y = x;
    else
      v.v.x = x;
  }
};

// Scalar type of each lane.
template <typename V>
struct LaneType {
  using type = V;
};
template <>
struct LaneType<f2> {
  using type = float;
};

// Storage <-> compute conversions.
__device__ __forceinline__ float ld_st(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ld_st(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_st(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void st_st(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_st(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_st(__half* p, float v) { *p = __float2half_rn(v); }

// 32-bit integer mixer (xor-shift-multiply rounds; constants of the published
// "lowbias32" hash).
__host__ __device__ __forceinline__ unsigned mix32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Rounding of FP16 stores: stochastic with a per-step seed, or nearest.  A launch
// that a graph replays reads the step count from device memory (*step + k, k its
// place in the graph); a direct launch carries the seed itself.
struct Rounding {
  unsigned seed;
  int stochastic;
  const unsigned* step;
  int k;
};

// Seed of the FP16 stores of time step n.
__host__ __device__ __forceinline__ unsigned step_seed(unsigned n) { return mix32(n * 2654435761u + 12345u); }

__device__ __forceinline__ Rounding resolve(Rounding r) {
  if (r.step) r.seed = step_seed(*r.step + unsigned(r.k));
  return r;
}

// FP32 -> FP16 pair with stochastic rounding (Blackwell's cvt.rs.f16x2.f32): each
// value is rounded toward zero after 13 random bits are added below the half's
// last mantissa bit (bits 12..0 of rbits for the low half, 28..16 for the high
// one), so a value between two halves goes up with probability equal to its
// distance from the lower one and the rounding error has zero mean.  The two
// halves are converted independently.  Returns (high << 16) | low.
__device__ __forceinline__ unsigned cvt_rs_f16x2(float lo, float hi, unsigned rbits) {
  unsigned r;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(r) : "f"(hi), "f"(lo), "r"(rbits));
  return r;
}

// Random words of the FP16 stores.  The nodes (2j, y) and (2j + 1, y) of a row
// form pair j; its words are a linear congruential sequence s_1, s_2, ... (mod
// 2^32) started at a hash of (pair index, step seed), population i taking s_{i+1}.
// Node 2j rounds with bits 12..0 of the word, node 2j + 1 with bits 28..16,
// whichever kernel stores it.  With a uniformly distributed start every s_i is
// uniform, so the two disjoint bit fields are independent and uniform and each
// rounding is unbiased; the short periods of an LCG's low bits only correlate the
// dithers of one node's nine populations, which does not bias any of them.
__device__ __forceinline__ unsigned sr_start(int x, int y, int nx, unsigned seed) {
  return mix32(unsigned(y * ((nx + 1) >> 1) + (x >> 1)) * 0x9e3779b9u + seed);
}
__device__ __forceinline__ unsigned sr_next(unsigned& s) {
  s = s * 1664525u + 1013904223u;
  return s;
}

// Stores the nine populations of node (x, y) of a lattice nx wide at p + i * plane.
template <typename store_t>
__device__ __forceinline__ void store9(store_t* p, int plane, const float (&o)[9], int x, int y, int nx, Rounding r) {
  if constexpr (sizeof(store_t) == 2) {
    if (r.stochastic) {
      unsigned s = sr_start(x, y, nx, r.seed);
      const bool odd = x & 1;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const unsigned w = sr_next(s);
        const unsigned h = cvt_rs_f16x2(odd ? 0.f : o[i], odd ? o[i] : 0.f, w);
        p[i * plane] = __ushort_as_half((unsigned short)(odd ? h >> 16 : h & 0xffffu));
      }
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) st_st(p + i * plane, o[i]);
}
template <typename store_t>
__device__ __forceinline__ void store9(store_t* p, int plane, const double (&o)[9], int, int, int, Rounding) {
#pragma unroll
  for (int i = 0; i < 9; ++i) st_st(p + i * plane, o[i]);
}

// FP16: the nine populations of nodes (x, y) and (x + 1, y), x even, as one half
// pair each at p + i * plane (p and plane even: 4-byte aligned pairs); the same
// halves as two store9 calls.
__device__ __forceinline__ void store9_pair(__half* p, int plane, const float (&o0)[9], const float (&o1)[9], int x,
                                            int y, int nx, Rounding r) {
  if (r.stochastic) {
    unsigned s = sr_start(x, y, nx, r.seed);
#pragma unroll
    for (int i = 0; i < 9; ++i)
      *reinterpret_cast<unsigned*>(p + i * plane) = cvt_rs_f16x2(o0[i], o1[i], sr_next(s));
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) *reinterpret_cast<__half2*>(p + i * plane) = __floats2half2_rn(o0[i], o1[i]);
  }
}

// ---------------------------------------------------------------------------
// Collision constants for value type V (host: make_vcoef).
template <typename V>
struct VCoef {
  int eos;
  V G2, rho_ref, neg_bq, bq, RT, lam_RT, neg_lam_a, neg_2lam_a, lam, a;
  V beta2, hk_seps, hh_sq, b_sq, hb_sq, om_e, om_eps, om_q, om_p;
  V R11, R17, R18, R71, R77, R81, R88, T1a, negT1b, X1, T7, T7b, X7, T8, X8, Q1G2, Q2G2, Q78G2;
  // literals and products of parameters with literals
  V one, mone, two, three, four, six, m6, nine, eighteen, half, m2, m4, m2rr, g15, ninth, i36, sixth, i12,
      quarter, h15, m3, mhalf;
  // 2 (1 - s_eps/2), 2 (1 - s_q/2): rows 2, 4, 6 of steps (3) and (5) in one factor
  V two_om_eps, two_om_q;
  // used by the adjoint only: -a, 8, 20 and the S Q_m factors without G^2
  V neg_a, eight, twenty, Q1, Q2, Q78;
  // stencil weights omega = 1/3 (axes), 1/12 (diagonals) of Eq. 12
  V third, twelfth;
};

// The coefficients that depend on the lattice's temperature, pressure scale,
// interaction strength and storage shift (everything else depends only on
// varpi, the relaxation rates and the EOS constants a, b).
template <typename V>
struct LatCoef {
  V G2, rho_ref, m2rr, lam_RT, neg_lam_a, neg_2lam_a, g15, Q1G2, Q2G2, Q78G2;
};

template <typename V>
__device__ __forceinline__ LatCoef<V> lattice_part(const VCoef<V>& c) {
  return LatCoef<V>{c.G2, c.rho_ref, c.m2rr, c.lam_RT, c.neg_lam_a, c.neg_2lam_a, c.g15, c.Q1G2, c.Q2G2, c.Q78G2};
}

// p_EOS / c^2 and d(p_EOS/c^2)/drho.  vdW: rho R T/(1 - b rho) - a rho^2;
// Carnahan-Starling (Eq. 20) with t = b rho / 4.  Both times K_EOS / c^2.
template <typename V>
__device__ __forceinline__ void eos(const VCoef<V>& c, const LatCoef<V>& l, V rho, V& pe, V& dpe) {
  if (c.eos == LB_EOS_VDW) {
    const V io = rcp(fmav(c.neg_bq, rho, c.one));
    const V q = l.lam_RT * io;                       // lam R T / (1 - b rho)
    pe = rho * fmav(l.neg_lam_a, rho, q);            // lam (rho R T/(1 - b rho) - a rho^2)
    dpe = fmav(q, io, l.neg_2lam_a * rho);           // lam (R T/(1 - b rho)^2 - 2 a rho)
  } else {
    const V t = c.bq * rho;
    const V io = rcp(c.one - t);
    const V io3 = io * io * io;
    const V t2 = t * t;
    const V z = fmav(t2, c.one - t, c.one + t) * io3;                              // (1+t+t^2-t^3)/(1-t)^3
    const V poly = fmav(t2, fmav(t, t - c.four, c.four), fmav(c.four, t, c.one));  // 1+4t+4t^2-4t^3+t^4
    const V dz = poly * io3 * io;
    pe = rho * fmav(l.neg_lam_a, rho, l.lam_RT * z);
    dpe = fmav(l.lam_RT, dz, l.neg_2lam_a * rho);
  }
}

template <typename V>
__device__ __forceinline__ void eos(const VCoef<V>& c, V rho, V& pe, V& dpe) {
  eos(c, lattice_part(c), rho, pe, dpe);
}

// One node (or a pair of nodes for V = f2).  d: post-streaming populations
// stored as deviations f_i - w_i rho_ref; (Sx, Sy) = sum_i omega_i rho(x + e_i) e_i
// (Eq. 12, = grad rho of supplement Eq. 61); o: post-collision deviations.
// The sequence is the paper's; its terms are grouped to share products (the
// halves of F_m enter G directly, ux Sy and uy Sx serve the forcing and the
// corrections, rho u is taken from Eq. 5 before the division by rho).
template <typename V>
__device__ __forceinline__ void collide(const VCoef<V>& c, const LatCoef<V>& l, const V (&d)[9], V Sx, V Sy,
                                        V (&o)[9]) {
  // Moment transform (supplement Eq. 4) with shared sums.  M w = (1, -2, 1, 0, ...):
  // the energy moments are carried as e + 2 rho_ref and eps - rho_ref (the moments
  // of the stored deviations) and their equilibria shifted alike, so that the
  // shift cancels in m - m_eq and in the inverse transform of mbar - rho_ref M w.
  const V a13 = d[1] + d[3], a24 = d[2] + d[4], a57 = d[5] + d[7], a68 = d[6] + d[8];
  const V s13 = d[1] - d[3], s24 = d[2] - d[4], s57 = d[5] - d[7], s68 = d[6] - d[8];
  const V axis = a13 + a24, diag = a57 + a68;
  const V rho_dev = d[0] + (axis + diag);
  const V rho = rho_dev + l.rho_ref;
  const V m1 = fmav(c.m4, d[0], (diag + diag) - axis);   // e + 2 rho_ref: -4 d0 - axis + 2 diag
  const V m2 = fmav(c.four, d[0], fmav(c.m2, axis, diag));  // eps - rho_ref: 4 d0 - 2 axis + diag
  const V dm = s57 - s68, dp = s57 + s68;
  const V jx = s13 + dm, jy = s24 + dp;
  const V m4 = fmav(c.m2, s13, dm);
  const V m6 = fmav(c.m2, s24, dp);
  const V m7 = a13 - a24;
  const V m8 = a57 - a68;

  // Interaction force (Eq. 12) and velocity (Eq. 5), c = 1.
  const V G2rho = l.G2 * rho;
  const V Fx = G2rho * Sx, Fy = G2rho * Sy;
  const V Jx = fmav(c.half, Fx, jx), Jy = fmav(c.half, Fy, jy);  // rho u
  const V inv_rho = rcp(rho);
  const V ux = Jx * inv_rho, uy = Jy * inv_rho;

  // Self-tuning EOS: p_LBE = p_EOS + G^2 rho^2/2 (Eq. 18) = c_s^2 (rho + eta);
  // grad p_LBE = (p_EOS' + G^2 rho) grad rho (supplement Eq. 61).
  V pe, dpe;
  eos(c, l, rho, pe, dpe);
  const V eta = fmav(c.three, pe, rho * fmav(l.g15, rho, c.mone));  // 3 pe + 1.5 G2 rho^2 - rho
  const V g = G2rho + dpe;

  const V x2 = ux * ux, y2 = uy * uy, xy = ux * uy, u2 = x2 + y2, x2my2 = x2 - y2;
  const V r3u2 = c.three * rho * u2;
  // Equilibrium (Eq. 3, alpha_1 = -1, beta_1 = 1, alpha_2 = 1), non-conserved rows
  // (rows 1 and 2 shifted by 2 rho_ref and -rho_ref, as m1 and m2).
  const V meq8 = rho * xy;
  const V meq1 = fmav(c.two, eta - rho_dev, r3u2);
  const V meq2 = fmav(c.nine * meq8, xy, fmav(c.beta2, eta, rho_dev) - r3u2);  // 9 rho ux^2 uy^2 + ...
  const V meq4 = Jx * fmav(c.three, y2, c.mone);  // rho ux (3 uy^2 - 1)
  const V meq6 = Jy * fmav(c.three, x2, c.mone);  // rho uy (3 ux^2 - 1)
  const V meq7 = rho * x2my2;
  // Forcing (Eq. 4), brackets summed over the force's positions, taken at half
  // weight: F_m/2 = (0, 3 Fu, -3 Fu + 9 xy Fc, ., -Fx/2 + 3/2 (Fx y2 + 2 Fy xy), .,
  // -Fy/2 + 3/2 (Fy x2 + 2 Fx xy), Fx ux - Fy uy, Fc/2), Fu = F.u, Fc = Fx uy + Fy ux.
  const V uySx = uy * Sx, uxSy = ux * Sy;
  const V uSp = uySx + uxSy, uSm = uySx - uxSy;
  const V FyUy = Fy * uy;
  const V Fu = fmav(Fx, ux, FyUy);
  const V Fc = G2rho * uSp;
  const V xy2 = xy + xy;

  // (1): D = m - m_eq, G = D + F_m / 2, and mbar starts as 2 m_eq - m = m_eq - D.
  const V D1 = m1 - meq1, D2 = m2 - meq2, D4 = m4 - meq4, D6 = m6 - meq6, D7 = m7 - meq7, D8 = m8 - meq8;
  const V G1 = fmav(c.three, Fu, D1);
  const V G2 = fmav(c.nine * xy, Fc, fmav(c.m3, Fu, D2));
  const V G4 = fmav(c.h15, fmav(Fx, y2, Fy * xy2), fmav(c.mhalf, Fx, D4));
  const V G6 = fmav(c.h15, fmav(Fy, x2, Fx * xy2), fmav(c.mhalf, Fy, D6));
  const V G7 = fmav(Fx, ux, D7 - FyUy);
  const V G8 = fmav(c.half, Fc, D8);
  // (2) off-diagonal part of S, then (3) I - diag(S)/2 (rows 2, 4, 6 enter step (5)
  // as 2 A with the factor 2 (1 - s/2) taken into one constant).
  const V uG = fmav(ux, G4, uy * G6), vG = ux * G4 - uy * G6, wG = fmav(uy, G4, ux * G6);
  const V A1 = c.om_e * fmav(c.hh_sq, uG, fmav(c.hk_seps, G2, G1));
  const V A7 = c.om_p * fmav(c.b_sq, vG, G7);
  const V A8 = c.om_p * fmav(c.hb_sq, wG, G8);
  // (4) cubic-velocity correction: R (I - S/2) G + T . grad rho + X . grad p_LBE
  // (supplement Eqs. 34, 37, 40), with grad p_LBE = g S.
  const V ax = x2 * ux * Sx, ay = y2 * uy * Sy;
  const V cr1 = fmav(c.T1a, ax + ay, fmav(g, c.X1, c.negT1b) * (xy * uSp));
  const V cr7 = fmav(c.T7, ax - ay, fmav(g, c.X7, c.T7b) * (xy * uSm));
  // (2 x2 + y2) uy Sx + (2 y2 + x2) ux Sy = u2 (uy Sx + ux Sy) + x2 uy Sx + y2 ux Sy.
  const V cr8 = fmav(g, c.X8, c.T8) * fmav(u2, uSp, fmav(x2, uySx, y2 * uxSy));
  const V corr1 = fmav(c.R11 * u2, A1, fmav(c.R17 * x2my2, A7, fmav(c.R18 * xy, A8, cr1)));
  const V corr7 = fmav(c.R71 * x2my2, A1, fmav(c.R77 * u2, A7, cr7));
  const V corr8 = fmav(c.R81 * xy, A1, fmav(c.R88 * u2, A8, cr8));
  // (5): mbar = m_eq - D + 2 A - corrections; (6): + S Q_m with |F~|^2 = G^2 |S|^2.
  const V sxx = Sx * Sx, syy = Sy * Sy, ss = sxx + syy;
  const V mb1 = fmav(l.Q1G2, ss, fmav(c.two, A1, meq1 - D1) - corr1);
  const V mb2 = fmav(l.Q2G2, ss, fmav(c.two_om_eps, G2, meq2 - D2));
  const V mb4 = fmav(c.two_om_q, G4, meq4 - D4);
  const V mb6 = fmav(c.two_om_q, G6, meq6 - D6);
  const V mb7 = fmav(l.Q78G2, sxx - syy, fmav(c.two, A7, meq7 - D7) - corr7);
  const V mb8 = fmav(l.Q78G2 * Sx, Sy, fmav(c.two, A8, meq8 - D8) - corr8);

  // Inverse transform M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4),
  // applied to mbar - rho_ref M w (deviation storage; rows 1 and 2 are already
  // shifted); conserved: rho, j + F.
  const V n0 = rho_dev * c.ninth;
  const V n1 = mb1 * c.i36;
  const V n2 = mb2 * c.i36;
  const V n3 = (jx + Fx) * c.sixth;
  const V n4 = mb4 * c.i12;
  const V n5 = (jy + Fy) * c.sixth;
  const V n6 = mb6 * c.i12;
  const V n7 = mb7 * c.quarter;
  const V n8 = mb8 * c.quarter;
  const V base_a = fmav(c.m2, n2, n0 - n1), base_d = fmav(c.two, n1, n0 + n2);
  const V px = fmav(c.m2, n4, n3), py = fmav(c.m2, n6, n5);
  const V qx = n3 + n4, qy = n5 + n6;
  const V ba7 = base_a + n7, bm7 = base_a - n7, bd8 = base_d + n8, bm8 = base_d - n8;
  o[0] = fmav(c.four, n2 - n1, n0);
  o[1] = ba7 + px;
  o[2] = bm7 + py;
  o[3] = ba7 - px;
  o[4] = bm7 - py;
  o[5] = bd8 + (qx + qy);
  o[6] = bm8 + (qy - qx);
  o[7] = bd8 - (qx + qy);
  o[8] = bm8 + (qx - qy);
}

template <typename V>
__device__ __forceinline__ void collide(const VCoef<V>& c, const V (&d)[9], V Sx, V Sy, V (&o)[9]) {
  collide(c, lattice_part(c), d, Sx, Sy, o);
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
