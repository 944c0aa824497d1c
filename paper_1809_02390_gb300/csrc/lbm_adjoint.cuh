// Hand-written reverse mode (vector-Jacobian product) of the per-node collision.
//
// Forward: o = C(d, S; theta) is the collision of lbm_device.cuh (execution
// sequence (1)-(6) of the paper's supplement Sec. IV, i.e. Eq. 13), with d the
// post-streaming populations of the node, S = sum_i omega_i rho(x + e_i) e_i the
// force stencil (Eq. 12), theta = (R T, G^2/c^2, K_EOS/c^2).  Given the cotangent
// ob of o, collide_vjp returns the cotangents of d, of S and of theta.  The
// forward values are recomputed here (in the same order as collide) and then
// every assignment is transposed in reverse order.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

template <typename real>
struct AdjOut {
  real d[9];         // cotangent of the pulled populations of the node
  real Sx, Sy;       // cotangent of the force stencil sum
  real RT, G2, lam;  // cotangents of the parameters
};

template <typename real>
__device__ __forceinline__ void collide_vjp(const VCoef<real>& c, const real (&d)[9], real Sx, real Sy,
                                            const real (&ob)[9], AdjOut<real>& r) {
  // ---------------- forward recomputation (same formulas as collide) ----------------
  const real a13 = d[1] + d[3], a24 = d[2] + d[4], a57 = d[5] + d[7], a68 = d[6] + d[8];
  const real s13 = d[1] - d[3], s24 = d[2] - d[4], s57 = d[5] - d[7], s68 = d[6] - d[8];
  const real axis = a13 + a24, diag = a57 + a68;
  const real rho = d[0] + axis + diag + c.rho_ref;
  const real m1 = real(-4) * d[0] - axis + real(2) * diag - real(2) * c.rho_ref;
  const real m2 = real(4) * d[0] - real(2) * axis + diag + c.rho_ref;
  const real jx = s13 + s57 - s68, jy = s24 + s57 + s68;
  const real m4 = real(-2) * s13 + s57 - s68, m6 = real(-2) * s24 + s57 + s68;
  const real m7 = a13 - a24, m8 = a57 - a68;
  const real G2 = c.G2, lam = c.lam, RT = c.RT, a = c.a, bq = c.bq;
  const real G2rho = G2 * rho;
  const real Fx = G2rho * Sx, Fy = G2rho * Sy;
  const real ir = real(1) / rho;
  const real hx = jx + real(0.5) * Fx, hy = jy + real(0.5) * Fy;
  const real ux = hx * ir, uy = hy * ir;
  // EOS and its parameter dependence.
  real pe, dpe;
  real io = 0, q = 0, t = 0, z = 0, dz = 0, zt = 0, dzt = 0;
  if (c.eos == LB_EOS_VDW) {
    io = real(1) / (real(1) - bq * rho);
    q = lam * RT * io;
    pe = rho * (q - lam * a * rho);
    dpe = q * io - real(2) * lam * a * rho;
  } else {
    t = bq * rho;
    const real om = real(1) - t;
    io = real(1) / om;
    const real io3 = io * io * io, io4 = io3 * io;
    z = (real(1) + t + t * t - t * t * t) * io3;
    dz = (real(1) + real(4) * t + real(4) * t * t - real(4) * t * t * t + t * t * t * t) * io4;
    zt = (real(4) + real(4) * t - real(2) * t * t) * io4;  // dz/dt
    dzt = (real(8) + real(20) * t - real(4) * t * t) * io4 * io;  // d(dz)/dt
    pe = rho * (lam * RT * z - lam * a * rho);
    dpe = lam * RT * dz - real(2) * lam * a * rho;
  }
  const real eta = real(3) * pe + real(1.5) * G2 * rho * rho - rho;
  const real g = G2rho + dpe;
  const real x2 = ux * ux, y2 = uy * uy, xy = ux * uy, u2 = x2 + y2;
  const real r3u2 = real(3) * rho * u2;
  const real meq1 = real(2) * (eta - rho) + r3u2;
  const real meq2 = real(9) * rho * x2 * y2 + c.beta2 * eta + rho - r3u2;
  const real meq4 = rho * ux * (real(3) * y2 - real(1)), meq6 = rho * uy * (real(3) * x2 - real(1));
  const real meq7 = rho * (x2 - y2), meq8 = rho * xy;
  const real Fu = Fx * ux + Fy * uy, Fc = Fx * uy + Fy * ux;
  const real Fm1 = real(6) * Fu;
  const real Fm2 = real(18) * xy * Fc - real(6) * Fu;
  const real Fm4 = real(3) * (Fx * y2 + real(2) * Fy * xy) - Fx;
  const real Fm6 = real(3) * (Fy * x2 + real(2) * Fx * xy) - Fy;
  const real Fm7 = real(2) * (Fx * ux - Fy * uy), Fm8 = Fc;
  const real G1 = m1 - meq1 + real(0.5) * Fm1, Gm2 = m2 - meq2 + real(0.5) * Fm2;
  const real G4 = m4 - meq4 + real(0.5) * Fm4, G6 = m6 - meq6 + real(0.5) * Fm6;
  const real G7 = m7 - meq7 + real(0.5) * Fm7, G8 = m8 - meq8 + real(0.5) * Fm8;
  const real uG = ux * G4 + uy * G6, vG = ux * G4 - uy * G6, wG = uy * G4 + ux * G6;
  const real A1 = c.om_e * (G1 + c.hk_seps * Gm2 + c.hh_sq * uG);
  const real A7 = c.om_p * (G7 + c.b_sq * vG), A8 = c.om_p * (G8 + c.hb_sq * wG);
  const real ax = x2 * ux * Sx, ay = y2 * uy * Sy;
  const real P1 = xy * (uy * Sx + ux * Sy), P7 = xy * (uy * Sx - ux * Sy);
  const real K1 = g * c.X1 + c.negT1b, K7 = c.T7b + g * c.X7, K8 = c.T8 + g * c.X8;
  const real B8 = (real(2) * x2 + y2) * uy * Sx + (real(2) * y2 + x2) * ux * Sy;
  const real x2my2 = x2 - y2;
  const real sxx = Sx * Sx, syy = Sy * Sy, ss = sxx + syy;
  // Parameter-free parts of the S Q_m coefficients (they are proportional to G2).
  const real q1 = c.Q1G2 / G2, q2 = c.Q2G2 / G2, q78 = c.Q78G2 / G2;

  // ---------------- reverse pass ----------------
  // o = M^T n  =>  nb = M ob.
  const real b13 = ob[1] + ob[3], b24 = ob[2] + ob[4], b57 = ob[5] + ob[7], b68 = ob[6] + ob[8];
  const real c13 = ob[1] - ob[3], c24 = ob[2] - ob[4], c57 = ob[5] - ob[7], c68 = ob[6] - ob[8];
  const real baxis = b13 + b24, bdiag = b57 + b68;
  const real nb0 = ob[0] + baxis + bdiag;
  const real nb1 = real(-4) * ob[0] - baxis + real(2) * bdiag;
  const real nb2 = real(4) * ob[0] - real(2) * baxis + bdiag;
  const real nb3 = c13 + c57 - c68, nb5 = c24 + c57 + c68;
  const real nb4 = real(-2) * c13 + c57 - c68, nb6 = real(-2) * c24 + c57 + c68;
  const real nb7 = b13 - b24, nb8 = b57 - b68;
  // n0 = rho_dev/9, n1 = (mb1 + 2 rr)/36, n2 = (mb2 - rr)/36, n3 = (jx + Fx)/6, ...
  real rho_b = nb0 * real(1.0 / 9.0);  // cotangent of rho (rho_dev and rho differ by a constant)
  const real mb1b = nb1 * real(1.0 / 36.0), mb2b = nb2 * real(1.0 / 36.0);
  const real mb4b = nb4 * real(1.0 / 12.0), mb6b = nb6 * real(1.0 / 12.0);
  const real mb7b = nb7 * real(0.25), mb8b = nb8 * real(0.25);
  real jxb = nb3 * real(1.0 / 6.0), jyb = nb5 * real(1.0 / 6.0);
  real Fxb = jxb, Fyb = jyb;
  real G2b = 0, lamb = 0, RTb = 0, Sxb = 0, Syb = 0;
  // mbar_k = (S Q_m)_k + 2 A_k + m_eq,k - D_k - corr_k, D_k = m_k - m_eq,k.
  real ssb = c.Q1G2 * mb1b + c.Q2G2 * mb2b;
  G2b += q1 * ss * mb1b + q2 * ss * mb2b + q78 * ((sxx - syy) * mb7b + Sx * Sy * mb8b);
  real sxxb = ssb + c.Q78G2 * mb7b, syyb = ssb - c.Q78G2 * mb7b;
  Sxb += c.Q78G2 * Sy * mb8b;
  Syb += c.Q78G2 * Sx * mb8b;
  real A1b = real(2) * mb1b, A2b = real(2) * mb2b, A4b = real(2) * mb4b, A6b = real(2) * mb6b;
  real A7b = real(2) * mb7b, A8b = real(2) * mb8b;
  real meq1b = mb1b, meq2b = mb2b, meq4b = mb4b, meq6b = mb6b, meq7b = mb7b, meq8b = mb8b;
  real D1b = -mb1b, D2b = -mb2b, D4b = -mb4b, D6b = -mb6b, D7b = -mb7b, D8b = -mb8b;
  const real corr1b = -mb1b, corr7b = -mb7b, corr8b = -mb8b;
  Sxb += real(2) * Sx * sxxb;
  Syb += real(2) * Sy * syyb;
  // corr8 = R81 xy A1 + R88 u2 A8 + cr8 ; corr7 ; corr1.
  real xyb = c.R81 * A1 * corr8b + c.R18 * A8 * corr1b;
  real u2b = c.R88 * A8 * corr8b + c.R77 * A7 * corr7b + c.R11 * A1 * corr1b;
  real x2my2b = c.R71 * A1 * corr7b + c.R17 * A7 * corr1b;
  A1b += c.R81 * xy * corr8b + c.R71 * x2my2 * corr7b + c.R11 * u2 * corr1b;
  A8b += c.R88 * u2 * corr8b + c.R18 * xy * corr1b;
  A7b += c.R77 * u2 * corr7b + c.R17 * x2my2 * corr1b;
  const real cr8b = corr8b, cr7b = corr7b, cr1b = corr1b;
  real x2b = x2my2b, y2b = -x2my2b;
  real uxb = 0, uyb = 0, gb = 0;
  // cr8 = K8 B8.
  gb += c.X8 * B8 * cr8b;
  const real B8b = K8 * cr8b;
  x2b += (real(2) * uy * Sx + ux * Sy) * B8b;
  y2b += (uy * Sx + real(2) * ux * Sy) * B8b;
  uyb += (real(2) * x2 + y2) * Sx * B8b;
  uxb += (real(2) * y2 + x2) * Sy * B8b;
  Sxb += (real(2) * x2 + y2) * uy * B8b;
  Syb += (real(2) * y2 + x2) * ux * B8b;
  // cr7 = T7 (ax - ay) + K7 P7 ; cr1 = T1a (ax + ay) + K1 P1.
  real axb = c.T7 * cr7b + c.T1a * cr1b, ayb = -c.T7 * cr7b + c.T1a * cr1b;
  gb += c.X7 * P7 * cr7b + c.X1 * P1 * cr1b;
  const real P7b = K7 * cr7b, P1b = K1 * cr1b;
  xyb += (uy * Sx - ux * Sy) * P7b + (uy * Sx + ux * Sy) * P1b;
  const real q7 = xy * P7b, q1b = xy * P1b;
  uyb += Sx * (q7 + q1b);
  uxb += Sy * (q1b - q7);
  Sxb += uy * (q7 + q1b);
  Syb += ux * (q1b - q7);
  // ax = x2 ux Sx ; ay = y2 uy Sy.
  x2b += ux * Sx * axb;
  uxb += x2 * Sx * axb;
  Sxb += x2 * ux * axb;
  y2b += uy * Sy * ayb;
  uyb += y2 * Sy * ayb;
  Syb += y2 * uy * ayb;
  // A8 = om_p (G8 + hb wG) ; A7 = om_p (G7 + b vG) ; A6, A4, A2 ; A1 = om_e (G1 + hk G2 + hh uG).
  real G8b = c.om_p * A8b;
  const real wGb = c.om_p * c.hb_sq * A8b;
  real G7b = c.om_p * A7b;
  const real vGb = c.om_p * c.b_sq * A7b;
  real G6b = c.om_q * A6b, G4b = c.om_q * A4b, Gm2b = c.om_eps * A2b;
  const real t1 = c.om_e * A1b;
  real G1b = t1;
  Gm2b += c.hk_seps * t1;
  const real uGb = c.hh_sq * t1;
  // uG, vG, wG.
  uxb += G4 * (uGb + vGb) + G6 * wGb;
  uyb += G6 * (uGb - vGb) + G4 * wGb;
  G4b += ux * (uGb + vGb) + uy * wGb;
  G6b += uy * (uGb - vGb) + ux * wGb;
  // G_k = D_k + F_m,k / 2 ; D_k = m_k - m_eq,k.
  D1b += G1b;
  D2b += Gm2b;
  D4b += G4b;
  D6b += G6b;
  D7b += G7b;
  D8b += G8b;
  const real Fm1b = real(0.5) * G1b, Fm2b = real(0.5) * Gm2b, Fm4b = real(0.5) * G4b;
  const real Fm6b = real(0.5) * G6b, Fm7b = real(0.5) * G7b, Fm8b = real(0.5) * G8b;
  const real m1b = D1b, m2b = D2b, m4b = D4b, m6b = D6b, m7b = D7b, m8b = D8b;
  meq1b -= D1b;
  meq2b -= D2b;
  meq4b -= D4b;
  meq6b -= D6b;
  meq7b -= D7b;
  meq8b -= D8b;
  // Forcing.
  real Fcb = Fm8b + real(18) * xy * Fm2b;
  real Fub = real(6) * Fm1b - real(6) * Fm2b;
  xyb += real(18) * Fc * Fm2b + real(6) * Fy * Fm4b + real(6) * Fx * Fm6b;
  Fxb += real(2) * ux * Fm7b + (real(3) * y2 - real(1)) * Fm4b + real(6) * xy * Fm6b;
  Fyb += real(-2) * uy * Fm7b + (real(3) * x2 - real(1)) * Fm6b + real(6) * xy * Fm4b;
  uxb += real(2) * Fx * Fm7b;
  uyb += real(-2) * Fy * Fm7b;
  y2b += real(3) * Fx * Fm4b;
  x2b += real(3) * Fy * Fm6b;
  // Fc = Fx uy + Fy ux ; Fu = Fx ux + Fy uy.
  Fxb += uy * Fcb + ux * Fub;
  Fyb += ux * Fcb + uy * Fub;
  uxb += Fy * Fcb + Fx * Fub;
  uyb += Fx * Fcb + Fy * Fub;
  // Equilibrium.
  rho_b += xy * meq8b + x2my2 * meq7b + uy * (real(3) * x2 - real(1)) * meq6b +
           ux * (real(3) * y2 - real(1)) * meq4b + (real(9) * x2 * y2 + real(1)) * meq2b - real(2) * meq1b;
  xyb += rho * meq8b;
  x2b += rho * meq7b + real(3) * rho * uy * meq6b + real(9) * rho * y2 * meq2b;
  y2b += -rho * meq7b + real(3) * rho * ux * meq4b + real(9) * rho * x2 * meq2b;
  uyb += rho * (real(3) * x2 - real(1)) * meq6b;
  uxb += rho * (real(3) * y2 - real(1)) * meq4b;
  real etab = c.beta2 * meq2b + real(2) * meq1b;
  const real r3u2b = meq1b - meq2b;
  rho_b += real(3) * u2 * r3u2b;
  u2b += real(3) * rho * r3u2b;
  x2b += u2b;
  y2b += u2b;
  uxb += uy * xyb + real(2) * ux * x2b;
  uyb += ux * xyb + real(2) * uy * y2b;
  // g = G2 rho + dpe ; eta = 3 pe + 1.5 G2 rho^2 - rho.
  real G2rhob = gb;
  const real dpeb = gb;
  const real peb = real(3) * etab;
  G2b += real(1.5) * rho * rho * etab;
  rho_b += (real(3) * G2 * rho - real(1)) * etab;
  // EOS.
  if (c.eos == LB_EOS_VDW) {
    // pe = rho (q - lam a rho) ; dpe = q io - 2 lam a rho ; q = lam RT io ; io = 1/(1 - b rho).
    rho_b += (q - real(2) * lam * a * rho) * peb - real(2) * lam * a * dpeb;
    const real qb = rho * peb + io * dpeb;
    lamb += -a * rho * rho * peb - real(2) * a * rho * dpeb + RT * io * qb;
    RTb += lam * io * qb;
    const real iob = q * dpeb + lam * RT * qb;
    rho_b += bq * io * io * iob;  // d io / d rho = b io^2
  } else {
    // pe = rho (lam RT z - lam a rho) ; dpe = lam RT dz - 2 lam a rho ; z(t), dz(t), t = bq rho.
    rho_b += (lam * RT * z - real(2) * lam * a * rho) * peb - real(2) * lam * a * dpeb;
    const real zb = lam * RT * rho * peb, dzb = lam * RT * dpeb;
    lamb += (RT * z - a * rho) * rho * peb + (RT * dz - real(2) * a * rho) * dpeb;
    RTb += lam * z * rho * peb + lam * dz * dpeb;
    rho_b += bq * (zt * zb + dzt * dzb);
  }
  // Fx = G2rho Sx ; ux = (jx + Fx/2)/rho.
  Fxb += real(0.5) * ir * uxb;
  Fyb += real(0.5) * ir * uyb;
  jxb += ir * uxb;
  jyb += ir * uyb;
  rho_b += -(hx * uxb + hy * uyb) * ir * ir;
  G2rhob += Sx * Fxb + Sy * Fyb;
  Sxb += G2rho * Fxb;
  Syb += G2rho * Fyb;
  G2b += rho * G2rhob;
  rho_b += G2 * G2rhob;
  // Moments: (rho, m1, m2, jx, m4, jy, m6, m7, m8) = M d  =>  db = M^T (their cotangents).
  const real n0 = rho_b, n1 = m1b, n2 = m2b, n3 = jxb, n4 = m4b, n5 = jyb, n6 = m6b, n7 = m7b, n8 = m8b;
  const real base_a = n0 - n1 - real(2) * n2, base_d = n0 + real(2) * n1 + n2;
  const real px = n3 - real(2) * n4, py = n5 - real(2) * n6, qx = n3 + n4, qy = n5 + n6;
  r.d[0] = n0 - real(4) * n1 + real(4) * n2;
  r.d[1] = base_a + px + n7;
  r.d[2] = base_a + py - n7;
  r.d[3] = base_a - px + n7;
  r.d[4] = base_a - py - n7;
  r.d[5] = base_d + qx + qy + n8;
  r.d[6] = base_d - qx + qy - n8;
  r.d[7] = base_d - qx - qy + n8;
  r.d[8] = base_d + qx - qy - n8;
  r.Sx = Sxb;
  r.Sy = Syb;
  r.RT = RTb;
  r.G2 = G2b;
  r.lam = lamb;
}

}  // namespace lbm
