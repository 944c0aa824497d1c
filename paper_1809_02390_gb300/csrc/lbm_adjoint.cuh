// Hand-written reverse mode (vector-Jacobian product) of the per-node collision.
//
// Forward: o = C(d, S; theta) is the collision of lbm_device.cuh (execution
// sequence (1)-(6) of the paper's supplement Sec. IV, i.e. Eq. 13), with d the
// post-streaming populations of the node, S = sum_i omega_i rho(x + e_i) e_i the
// force stencil (Eq. 12), theta = (R T, G^2/c^2, K_EOS/c^2).  Given the cotangent
// ob of o, collide_vjp returns the cotangents of d, of S and of theta.  The
// forward values are recomputed here (the formulas of collide, grouped in the
// paper's form: F_m in full, the storage shift in m1 and m2) and then every
// assignment is transposed in reverse order.
//
// Written once for a value type V (double, float, or f2 = two FP32 nodes per
// packed FFMA2 / FADD2 / FMUL2 instruction, as in collide); every constant comes
// from the VCoef<V> block.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

template <typename V>
struct AdjOut {
  V d[9];         // cotangent of the pulled populations of the node
  V Sx, Sy;       // cotangent of the force stencil sum
  V RT, G2, lam;  // cotangents of the parameters
};

template <typename V>
__device__ __forceinline__ void collide_vjp(const VCoef<V>& c, const V (&d)[9], V Sx, V Sy, const V (&ob)[9],
                                            AdjOut<V>& r) {
  // ---------------- forward recomputation (the formulas of collide) ----------------
  const V a13 = d[1] + d[3], a24 = d[2] + d[4], a57 = d[5] + d[7], a68 = d[6] + d[8];
  const V s13 = d[1] - d[3], s24 = d[2] - d[4], s57 = d[5] - d[7], s68 = d[6] - d[8];
  const V axis = a13 + a24, diag = a57 + a68;
  const V rho = d[0] + (axis + diag) + c.rho_ref;
  const V m1 = fmav(c.m4, d[0], fmav(c.two, diag, c.m2rr) - axis);
  const V m2 = fmav(c.four, d[0], fmav(c.m2, axis, diag + c.rho_ref));
  const V dm = s57 - s68, dp = s57 + s68;
  const V jx = s13 + dm, jy = s24 + dp;
  const V m4 = fmav(c.m2, s13, dm), m6 = fmav(c.m2, s24, dp);
  const V m7 = a13 - a24, m8 = a57 - a68;
  const V G2rho = c.G2 * rho;
  const V Fx = G2rho * Sx, Fy = G2rho * Sy;
  const V ir = rcp(rho);
  const V hx = fmav(c.half, Fx, jx), hy = fmav(c.half, Fy, jy);
  const V ux = hx * ir, uy = hy * ir;
  // EOS and its parameter dependence.
  V pe, dpe, io, q, z, dz, zt, dzt;
  if (c.eos == LB_EOS_VDW) {
    io = rcp(fmav(c.neg_bq, rho, c.one));
    q = c.lam_RT * io;
    pe = rho * fmav(c.neg_lam_a, rho, q);
    dpe = fmav(q, io, c.neg_2lam_a * rho);
    z = dz = zt = dzt = q;  // unused
  } else {
    const V t = c.bq * rho;
    io = rcp(c.one - t);
    const V io3 = io * io * io, io4 = io3 * io;
    const V t2 = t * t;
    z = fmav(t2, c.one - t, c.one + t) * io3;
    dz = fmav(t2, fmav(t, t - c.four, c.four), fmav(c.four, t, c.one)) * io4;
    zt = fmav(t, fmav(c.m2, t, c.four), c.four) * io4;              // dz/dt
    dzt = fmav(t, fmav(c.m4, t, c.twenty), c.eight) * (io4 * io);  // d(dz)/dt
    pe = rho * fmav(c.neg_lam_a, rho, c.lam_RT * z);
    dpe = fmav(c.lam_RT, dz, c.neg_2lam_a * rho);
    q = pe;  // unused
  }
  const V eta = fmav(c.three, pe, rho * fmav(c.g15, rho, c.mone));
  const V g = G2rho + dpe;
  const V x2 = ux * ux, y2 = uy * uy, xy = ux * uy, u2 = x2 + y2;
  const V r3u2 = c.three * rho * u2;
  const V meq1 = fmav(c.two, eta - rho, r3u2);
  const V meq2 = fmav(c.nine * rho * x2, y2, fmav(c.beta2, eta, rho) - r3u2);
  const V tx3 = fmav(c.three, y2, c.mone), ty3 = fmav(c.three, x2, c.mone);  // 3 uy^2 - 1, 3 ux^2 - 1
  const V meq4 = rho * ux * tx3, meq6 = rho * uy * ty3;
  const V x2my2 = x2 - y2;
  const V meq7 = rho * x2my2, meq8 = rho * xy;
  const V Fu = fmav(Fx, ux, Fy * uy), Fc = fmav(Fx, uy, Fy * ux);
  const V Fm1 = c.six * Fu;
  const V Fm2 = fmav(c.eighteen * xy, Fc, c.m6 * Fu);
  const V Fm4 = fmav(c.three, fmav(Fx, y2, (c.two * Fy) * xy), c.mone * Fx);
  const V Fm6 = fmav(c.three, fmav(Fy, x2, (c.two * Fx) * xy), c.mone * Fy);
  const V Fm7 = c.two * (Fx * ux - Fy * uy), Fm8 = Fc;
  const V G1 = fmav(c.half, Fm1, m1 - meq1), Gm2 = fmav(c.half, Fm2, m2 - meq2);
  const V G4 = fmav(c.half, Fm4, m4 - meq4), G6 = fmav(c.half, Fm6, m6 - meq6);
  const V G7 = fmav(c.half, Fm7, m7 - meq7), G8 = fmav(c.half, Fm8, m8 - meq8);
  const V uG = fmav(ux, G4, uy * G6), vG = ux * G4 - uy * G6, wG = fmav(uy, G4, ux * G6);
  const V A1 = c.om_e * fmav(c.hh_sq, uG, fmav(c.hk_seps, Gm2, G1));
  const V A7 = c.om_p * fmav(c.b_sq, vG, G7), A8 = c.om_p * fmav(c.hb_sq, wG, G8);
  const V ax = x2 * ux * Sx, ay = y2 * uy * Sy;
  const V uSp = fmav(uy, Sx, ux * Sy), uSm = uy * Sx - ux * Sy;  // uy Sx +- ux Sy
  const V P1 = xy * uSp, P7 = xy * uSm;
  const V K1 = fmav(g, c.X1, c.negT1b), K7 = fmav(g, c.X7, c.T7b), K8 = fmav(g, c.X8, c.T8);
  const V cx8 = fmav(c.two, x2, y2), cy8 = fmav(c.two, y2, x2);  // 2 x2 + y2, 2 y2 + x2
  const V B8 = fmav(cx8 * uy, Sx, cy8 * ux * Sy);
  const V sxx = Sx * Sx, syy = Sy * Sy, ss = sxx + syy;

  // ---------------- reverse pass ----------------
  // o = M^T n  =>  nb = M ob.
  const V b13 = ob[1] + ob[3], b24 = ob[2] + ob[4], b57 = ob[5] + ob[7], b68 = ob[6] + ob[8];
  const V c13 = ob[1] - ob[3], c24 = ob[2] - ob[4], c57 = ob[5] - ob[7], c68 = ob[6] - ob[8];
  const V baxis = b13 + b24, bdiag = b57 + b68;
  const V cdm = c57 - c68, cdp = c57 + c68;
  // n0 = rho_dev/9, n1 = (mb1 + 2 rr)/36, n2 = (mb2 - rr)/36, n3 = (jx + Fx)/6, ...
  V rho_b = (ob[0] + (baxis + bdiag)) * c.ninth;  // rho_dev and rho differ by a constant
  const V mb1b = fmav(c.m4, ob[0], c.two * bdiag - baxis) * c.i36;
  const V mb2b = fmav(c.four, ob[0], fmav(c.m2, baxis, bdiag)) * c.i36;
  const V mb4b = fmav(c.m2, c13, cdm) * c.i12, mb6b = fmav(c.m2, c24, cdp) * c.i12;
  const V mb7b = (b13 - b24) * c.quarter, mb8b = (b57 - b68) * c.quarter;
  V jxb = (c13 + cdm) * c.sixth, jyb = (c24 + cdp) * c.sixth;
  V Fxb = jxb, Fyb = jyb;
  // mbar_k = (S Q_m)_k + 2 A_k + m_eq,k - D_k - corr_k, D_k = m_k - m_eq,k.
  const V ssb = fmav(c.Q1G2, mb1b, c.Q2G2 * mb2b);
  V G2b = fmav(ss, fmav(c.Q1, mb1b, c.Q2 * mb2b), c.Q78 * fmav(sxx - syy, mb7b, (Sx * Sy) * mb8b));
  const V e8 = c.Q78G2 * mb8b;
  V Sxb = fmav(c.two * Sx, fmav(c.Q78G2, mb7b, ssb), Sy * e8);
  V Syb = fmav(c.two * Sy, ssb - c.Q78G2 * mb7b, Sx * e8);
  // Cotangents of the corrections: corr_kb = -mb_kb.
  const V k1 = c.mone * mb1b, k7 = c.mone * mb7b, k8 = c.mone * mb8b;
  // corr8 = R81 xy A1 + R88 u2 A8 + cr8 ; corr7 = R71 x2my2 A1 + R77 u2 A7 + cr7 ;
  // corr1 = R11 u2 A1 + R17 x2my2 A7 + R18 xy A8 + cr1.
  V xyb = fmav(c.R81 * A1, k8, c.R18 * A8 * k1);
  V u2b = fmav(c.R88 * A8, k8, fmav(c.R77 * A7, k7, c.R11 * A1 * k1));
  const V x2my2b = fmav(c.R71 * A1, k7, c.R17 * A7 * k1);
  const V A1b = fmav(c.two, mb1b, fmav(c.R81 * xy, k8, fmav(c.R71 * x2my2, k7, c.R11 * u2 * k1)));
  const V A8b = fmav(c.two, mb8b, fmav(c.R88 * u2, k8, c.R18 * xy * k1));
  const V A7b = fmav(c.two, mb7b, fmav(c.R77 * u2, k7, c.R17 * x2my2 * k1));
  // cr8 = K8 B8 ; cr7 = T7 (ax - ay) + K7 P7 ; cr1 = T1a (ax + ay) + K1 P1.
  V gb = fmav(c.X8 * B8, k8, fmav(c.X7 * P7, k7, c.X1 * P1 * k1));
  const V B8b = K8 * k8;
  const V P7b = K7 * k7, P1b = K1 * k1;
  const V axb = fmav(c.T7, k7, c.T1a * k1), ayb = fmav(c.T1a, k1, c.mone * c.T7 * k7);
  const V q7 = xy * P7b, q1 = xy * P1b;
  const V qp = q7 + q1, qm = q1 - q7;
  xyb = fmav(uSm, P7b, fmav(uSp, P1b, xyb));
  V x2b = fmav(fmav(c.two * uy, Sx, ux * Sy), B8b, fmav(ux * Sx, axb, x2my2b));
  V y2b = fmav(fmav(uy, Sx, (c.two * ux) * Sy), B8b, fmav(uy * Sy, ayb, c.mone * x2my2b));
  V uxb = fmav(cy8 * Sy, B8b, fmav(Sy, qm, x2 * Sx * axb));
  V uyb = fmav(cx8 * Sx, B8b, fmav(Sx, qp, y2 * Sy * ayb));
  Sxb = fmav(cx8 * uy, B8b, fmav(uy, qp, fmav(x2 * ux, axb, Sxb)));
  Syb = fmav(cy8 * ux, B8b, fmav(ux, qm, fmav(y2 * uy, ayb, Syb)));
  // A8 = om_p (G8 + hb wG) ; A7 = om_p (G7 + b vG) ; A6 = om_q G6 ; A4 = om_q G4 ;
  // A2 = om_eps G2 ; A1 = om_e (G1 + hk G2 + hh uG) ; mb_k gets 2 A_k.
  const V G8b = c.om_p * A8b, wGb = c.om_p * c.hb_sq * A8b;
  const V G7b = c.om_p * A7b, vGb = c.om_p * c.b_sq * A7b;
  const V t1 = c.om_e * A1b;
  const V G1b = t1;
  const V Gm2b = fmav(c.hk_seps, t1, c.om_eps * (c.two * mb2b));
  const V uGb = c.hh_sq * t1;
  const V uvp = uGb + vGb, uvm = uGb - vGb;
  uxb = fmav(G4, uvp, fmav(G6, wGb, uxb));
  uyb = fmav(G6, uvm, fmav(G4, wGb, uyb));
  const V G4b = fmav(ux, uvp, fmav(uy, wGb, c.om_q * (c.two * mb4b)));
  const V G6b = fmav(uy, uvm, fmav(ux, wGb, c.om_q * (c.two * mb6b)));
  // G_k = D_k + F_m,k / 2 ; D_k = m_k - m_eq,k, and mb_k holds -D_k.
  const V m1b = G1b - mb1b, m2b = Gm2b - mb2b, m4b = G4b - mb4b;
  const V m6b = G6b - mb6b, m7b = G7b - mb7b, m8b = G8b - mb8b;
  const V meq1b = mb1b - m1b, meq2b = mb2b - m2b, meq4b = mb4b - m4b;
  const V meq6b = mb6b - m6b, meq7b = mb7b - m7b, meq8b = mb8b - m8b;
  const V Fm1b = c.half * G1b, Fm2b = c.half * Gm2b, Fm4b = c.half * G4b;
  const V Fm6b = c.half * G6b, Fm7b = c.half * G7b, Fm8b = c.half * G8b;
  // Forcing.
  const V Fcb = fmav(c.eighteen * xy, Fm2b, Fm8b);
  const V Fub = c.six * (Fm1b - Fm2b);
  xyb = fmav(c.eighteen * Fc, Fm2b, fmav(c.six * Fy, Fm4b, fmav(c.six * Fx, Fm6b, xyb)));
  Fxb = fmav(c.two * ux, Fm7b, fmav(tx3, Fm4b, fmav(c.six * xy, Fm6b, Fxb)));
  Fyb = fmav(c.m2 * uy, Fm7b, fmav(ty3, Fm6b, fmav(c.six * xy, Fm4b, Fyb)));
  uxb = fmav(c.two * Fx, Fm7b, uxb);
  uyb = fmav(c.m2 * Fy, Fm7b, uyb);
  y2b = fmav(c.three * Fx, Fm4b, y2b);
  x2b = fmav(c.three * Fy, Fm6b, x2b);
  // Fc = Fx uy + Fy ux ; Fu = Fx ux + Fy uy.
  Fxb = fmav(uy, Fcb, fmav(ux, Fub, Fxb));
  Fyb = fmav(ux, Fcb, fmav(uy, Fub, Fyb));
  uxb = fmav(Fy, Fcb, fmav(Fx, Fub, uxb));
  uyb = fmav(Fx, Fcb, fmav(Fy, Fub, uyb));
  // Equilibrium.
  rho_b = fmav(xy, meq8b, fmav(x2my2, meq7b, fmav(uy * ty3, meq6b, fmav(ux * tx3, meq4b,
          fmav(fmav(c.nine * x2, y2, c.one), meq2b, fmav(c.m2, meq1b, rho_b))))));
  xyb = fmav(rho, meq8b, xyb);
  const V r3 = c.three * rho, r9 = c.nine * rho;
  x2b = fmav(rho, meq7b, fmav(r3 * uy, meq6b, fmav(r9 * y2, meq2b, x2b)));
  y2b = fmav(r3 * ux, meq4b, fmav(r9 * x2, meq2b, y2b - rho * meq7b));
  uyb = fmav(rho * ty3, meq6b, uyb);
  uxb = fmav(rho * tx3, meq4b, uxb);
  const V etab = fmav(c.beta2, meq2b, c.two * meq1b);
  const V r3u2b = meq1b - meq2b;
  rho_b = fmav(c.three * u2, r3u2b, rho_b);
  u2b = fmav(r3, r3u2b, u2b);
  x2b = x2b + u2b;
  y2b = y2b + u2b;
  uxb = fmav(uy, xyb, fmav(c.two * ux, x2b, uxb));
  uyb = fmav(ux, xyb, fmav(c.two * uy, y2b, uyb));
  // g = G2 rho + dpe ; eta = 3 pe + 1.5 G2 rho^2 - rho.
  V G2rhob = gb;
  const V dpeb = gb, peb = c.three * etab;
  G2b = fmav(c.h15 * rho * rho, etab, G2b);
  rho_b = fmav(fmav(c.two * c.g15, rho, c.mone), etab, rho_b);  // (3 G2 rho - 1) etab
  // EOS.
  V lamb, RTb;
  if (c.eos == LB_EOS_VDW) {
    // pe = rho (q - lam a rho) ; dpe = q io - 2 lam a rho ; q = lam RT io ; io = 1/(1 - b rho).
    rho_b = fmav(fmav(c.neg_2lam_a, rho, q), peb, fmav(c.neg_2lam_a, dpeb, rho_b));
    const V qb = fmav(rho, peb, io * dpeb);
    lamb = fmav(c.RT * io, qb, (c.neg_a * rho) * fmav(rho, peb, c.two * dpeb));
    RTb = c.lam * io * qb;
    const V iob = fmav(q, dpeb, c.lam_RT * qb);
    rho_b = fmav(c.bq * io * io, iob, rho_b);  // d io / d rho = b io^2
  } else {
    // pe = rho (lam RT z - lam a rho) ; dpe = lam RT dz - 2 lam a rho ; z(t), dz(t), t = bq rho.
    rho_b = fmav(fmav(c.lam_RT, z, c.neg_2lam_a * rho), peb, fmav(c.neg_2lam_a, dpeb, rho_b));
    const V rpeb = rho * peb;
    lamb = fmav(fmav(c.RT, z, c.neg_a * rho), rpeb, fmav(c.RT, dz, (c.two * c.neg_a) * rho) * dpeb);
    RTb = c.lam * fmav(z, rpeb, dz * dpeb);
    rho_b = fmav(c.bq * c.lam_RT, fmav(zt, rpeb, dzt * dpeb), rho_b);
  }
  // Fx = G2rho Sx ; ux = (jx + Fx/2)/rho.
  Fxb = fmav(c.half * ir, uxb, Fxb);
  Fyb = fmav(c.half * ir, uyb, Fyb);
  jxb = fmav(ir, uxb, jxb);
  jyb = fmav(ir, uyb, jyb);
  rho_b = fmav(c.mone * fmav(hx, uxb, hy * uyb), ir * ir, rho_b);
  G2rhob = fmav(Sx, Fxb, fmav(Sy, Fyb, G2rhob));
  Sxb = fmav(G2rho, Fxb, Sxb);
  Syb = fmav(G2rho, Fyb, Syb);
  G2b = fmav(rho, G2rhob, G2b);
  rho_b = fmav(c.G2, G2rhob, rho_b);
  // Moments: (rho, m1, m2, jx, m4, jy, m6, m7, m8) = M d  =>  db = M^T (their cotangents).
  const V n0 = rho_b, n1 = m1b, n2 = m2b, n3 = jxb, n4 = m4b, n5 = jyb, n6 = m6b, n7 = m7b, n8 = m8b;
  const V base_a = fmav(c.m2, n2, n0 - n1), base_d = fmav(c.two, n1, n0 + n2);
  const V px = fmav(c.m2, n4, n3), py = fmav(c.m2, n6, n5);
  const V qx = n3 + n4, qy = n5 + n6;
  const V ba7 = base_a + n7, bm7 = base_a - n7, bd8 = base_d + n8, bm8 = base_d - n8;
  r.d[0] = fmav(c.four, n2 - n1, n0);
  r.d[1] = ba7 + px;
  r.d[2] = bm7 + py;
  r.d[3] = ba7 - px;
  r.d[4] = bm7 - py;
  r.d[5] = bd8 + (qx + qy);
  r.d[6] = bm8 + (qy - qx);
  r.d[7] = bd8 - (qx + qy);
  r.d[8] = bm8 + (qx - qy);
  r.Sx = Sxb;
  r.Sy = Syb;
  r.RT = RTb;
  r.G2 = G2b;
  r.lam = lamb;
}

}  // namespace lbm
