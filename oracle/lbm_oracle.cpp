// Plain FP64 CPU oracle for the per-node time step of the self-tuning-EOS
// multiphase lattice Boltzmann model (Huang, Wu & Adams, arXiv:1809.02390).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
// load this file: only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / reference leg use it.  It shares no code, header, table or
// constant with the CUDA library.
//
// Every quantity is in lattice units with delta_x = 1 and lattice speed c = 1
// (the model is invariant under c -> 1 with p -> p/c^2 and G^2 -> G^2/c^2;
// hatted quantities of the paper are then the plain ones).  The collision is
// evaluated in the plain matrix form of the paper's Eq. 13 (supplement Eq. 1):
//
//   mbar = m + F_m - S (m - m_eq + F_m/2) + S Q_m
//            - R (I - S/2) (m - m_eq + F_m/2) - T . grad(rho) - X . grad(p_LBE)
//
// with the 9x9 matrices S, R and the 9x2 matrices T, X assembled entry by entry,
// followed by fbar = M^-1 mbar and pull streaming (supplement Eq. 2).  No
// blocking, fusion or reordering beyond that definition.  `form` selects the
// paper's three nested collision equations: 2 (plain, Eq. 2), 10 (with the
// cubic-velocity correction, Eq. 10) and 13 (with S Q_m as well, Eq. 13).
//
// Templated on the scalar so that the same code runs in double and in
// std::complex<double> (complex-step derivatives for the adjoint checks).
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

using cplx = std::complex<double>;

// D2Q9 velocities, supplement Eq. 3 (c = 1): rest, four axis, four diagonal.
const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Dimensionless transformation matrix, supplement Eq. 4 (Lallemand & Luo).
// Moment order: rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy.
const double MMAT[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

// Interaction-force weights of Eq. 12: omega(1) = 1/3 on the axes,
// omega(2) = 1/12 on the diagonals; the rest direction does not contribute.
const double WFORCE[9] = {0.0,        1.0 / 3.0,  1.0 / 3.0,  1.0 / 3.0, 1.0 / 3.0,
                          1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0};

// M^-1 by Gauss-Jordan elimination with partial pivoting (a library-style
// primitive; the oracle does not use the orthogonality shortcut).
struct MInverse {
  double inv[9][9];
  MInverse() {
    double a[9][18];
    for (int r = 0; r < 9; ++r)
      for (int c = 0; c < 18; ++c) a[r][c] = c < 9 ? MMAT[r][c] : (c - 9 == r ? 1.0 : 0.0);
    for (int col = 0; col < 9; ++col) {
      int piv = col;
      for (int r = col + 1; r < 9; ++r)
        if (std::abs(a[r][col]) > std::abs(a[piv][col])) piv = r;
      for (int c = 0; c < 18; ++c) std::swap(a[col][c], a[piv][c]);
      const double d = a[col][col];
      for (int c = 0; c < 18; ++c) a[col][c] /= d;
      for (int r = 0; r < 9; ++r) {
        if (r == col) continue;
        const double fac = a[r][col];
        for (int c = 0; c < 18; ++c) a[r][c] -= fac * a[col][c];
      }
    }
    for (int r = 0; r < 9; ++r)
      for (int c = 0; c < 9; ++c) inv[r][c] = a[r][c + 9];
  }
};
const MInverse MINV;

}  // namespace

extern "C" {

// Lattice-unit parameters (c = 1, delta_x = 1).
typedef struct {
  int32_t eos;   // 0: van der Waals, 1: Carnahan-Starling (Eq. 20), 2: ideal gas p = rho/3
  int32_t form;  // 2, 10 or 13: collision of Eq. 2, Eq. 10 or Eq. 13
  double eos_a, eos_b, R_gas, T;  // EOS constants and temperature
  double lam;    // pressure scale K_EOS / c^2 (multiplies the vdW / CS EOS)
  double G2;     // interaction strength G^2 / c^2 of Eq. 12
  double varpi;  // bulk-viscosity coefficient of Eq. 7
  double s0, se, seps, sj, sq, sp;  // diagonal of S (Eq. 6)
} or_params;

}  // extern "C"

namespace {

template <class R>
struct P {
  int eos, form;
  R eos_a, eos_b, R_gas, T, lam, G2;
  double varpi, s0, se, seps, sj, sq, sp;
  // Coefficients of Eq. 7 with alpha_1 = -1, beta_1 = 1 (hence alpha_2 = 1).
  double alpha2, beta2, k, h, b;
};

template <class R>
P<R> make_params(const or_params& q, const double* dtheta_im) {
  P<R> p;
  p.eos = q.eos;
  p.form = q.form;
  p.eos_a = q.eos_a;
  p.eos_b = q.eos_b;
  p.R_gas = q.R_gas;
  p.T = q.T;
  p.lam = q.lam;
  p.G2 = q.G2;
  p.varpi = q.varpi;
  p.s0 = q.s0;
  p.se = q.se;
  p.seps = q.seps;
  p.sj = q.sj;
  p.sq = q.sq;
  p.sp = q.sp;
  const double w = q.varpi;
  // Eq. 7 (supplement Eq. 31) with alpha_1 = -1, beta_1 = 1; alpha_2 =
  // -(2 alpha_1 + varpi + 1)/(1 - varpi) is then 1 for every varpi (main text
  // after Eq. 9), written as such so that varpi = 1 stays finite.
  p.alpha2 = 1.0;
  // varpi = 1 is the classical model: eta must vanish and beta_2 is unused.
  p.beta2 = (w == 1.0) ? 0.0 : -2.0 * 1.0 / (1.0 - w);
  p.k = 1.0 - w;
  p.h = 6.0 * w * (1.0 - w) / (1.0 - 3.0 * w);
  p.b = (1.0 - w) / (1.0 - 3.0 * w);
  (void)dtheta_im;
  return p;
}

template <>
P<cplx> make_params<cplx>(const or_params& q, const double* dtheta_im) {
  P<double> d = make_params<double>(q, nullptr);
  P<cplx> p;
  p.eos = d.eos;
  p.form = d.form;
  p.eos_a = d.eos_a;
  p.eos_b = d.eos_b;
  p.R_gas = d.R_gas;
  // Complex-step perturbations of the differentiable parameters (T, G2, lam).
  p.T = cplx(d.T, dtheta_im ? dtheta_im[0] : 0.0);
  p.G2 = cplx(d.G2, dtheta_im ? dtheta_im[1] : 0.0);
  p.lam = cplx(d.lam, dtheta_im ? dtheta_im[2] : 0.0);
  p.varpi = d.varpi;
  p.s0 = d.s0;
  p.se = d.se;
  p.seps = d.seps;
  p.sj = d.sj;
  p.sq = d.sq;
  p.sp = d.sp;
  p.alpha2 = d.alpha2;
  p.beta2 = d.beta2;
  p.k = d.k;
  p.h = d.h;
  p.b = d.b;
  return p;
}

// p_EOS / c^2 and its density derivative.  vdW: p = rho R T/(1 - b rho) - a rho^2.
// Carnahan-Starling, Eq. 20: p = rho R T (1 + t + t^2 - t^3)/(1 - t)^3 - a rho^2,
// t = b rho / 4.  Both carry the scale K_EOS / c^2.  Ideal gas: p = rho c_s^2.
template <class R>
void eos(const P<R>& p, R rho, R* pe, R* dpe) {
  if (p.eos == 0) {
    const R one_m = 1.0 - p.eos_b * rho;
    *pe = p.lam * (rho * p.R_gas * p.T / one_m - p.eos_a * rho * rho);
    *dpe = p.lam * (p.R_gas * p.T / (one_m * one_m) - 2.0 * p.eos_a * rho);
  } else if (p.eos == 1) {
    const R t = p.eos_b * rho / 4.0;
    const R om = 1.0 - t;
    const R om3 = om * om * om;
    const R z = (1.0 + t + t * t - t * t * t) / om3;
    // d(rho z)/d rho = (1 + 4t + 4t^2 - 4t^3 + t^4) / (1 - t)^4
    const R dz = (1.0 + 4.0 * t + 4.0 * t * t - 4.0 * t * t * t + t * t * t * t) / (om3 * om);
    *pe = p.lam * (rho * p.R_gas * p.T * z - p.eos_a * rho * rho);
    *dpe = p.lam * (p.R_gas * p.T * dz - 2.0 * p.eos_a * rho);
  } else {
    *pe = rho / 3.0;
    *dpe = R(1.0 / 3.0);
  }
}

// Equilibrium moments, Eq. 3, with alpha_1 = -1, beta_1 = 1.
template <class R>
void moments_eq(const P<R>& p, R rho, R eta, R ux, R uy, R meq[9]) {
  const R u2 = ux * ux + uy * uy;
  meq[0] = rho;
  meq[1] = 2.0 * (-1.0) * rho + 2.0 * 1.0 * eta + 3.0 * rho * u2;
  meq[2] = p.alpha2 * rho + p.beta2 * eta - 3.0 * rho * u2 + 9.0 * rho * ux * ux * uy * uy;
  meq[3] = rho * ux;
  meq[4] = -rho * ux + 3.0 * rho * ux * uy * uy;
  meq[5] = rho * uy;
  meq[6] = -rho * uy + 3.0 * rho * uy * ux * ux;
  meq[7] = rho * (ux * ux - uy * uy);
  meq[8] = rho * ux * uy;
}

// Forcing in moment space, Eq. 4.  The bracket [.] is the sum over the
// positions the force takes in the tensor product (supplement, after Eq. 16):
//   [F u u]_xyy   = Fx uy uy + Fy ux uy + Fy uy ux = Fx uy^2 + 2 Fy ux uy
//   [F u u]_xxy   = 2 Fx ux uy + Fy ux^2
//   [F u u u]_xxyy = 2 Fx ux uy^2 + 2 Fy ux^2 uy
template <class R>
void moments_force(R Fx, R Fy, R ux, R uy, R Fm[9]) {
  const R Fu = Fx * ux + Fy * uy;
  const R b_xyy = Fx * uy * uy + 2.0 * Fy * ux * uy;
  const R b_xxy = 2.0 * Fx * ux * uy + Fy * ux * ux;
  const R b_xxyy = 2.0 * Fx * ux * uy * uy + 2.0 * Fy * ux * ux * uy;
  Fm[0] = 0.0;
  Fm[1] = 6.0 * Fu;
  Fm[2] = -6.0 * Fu + 9.0 * b_xxyy;
  Fm[3] = Fx;
  Fm[4] = -Fx + 3.0 * b_xyy;
  Fm[5] = Fy;
  Fm[6] = -Fy + 3.0 * b_xxy;
  Fm[7] = 2.0 * (Fx * ux - Fy * uy);
  Fm[8] = Fx * uy + Fy * ux;
}

// Collision matrix S of Eq. 6 (velocity dependent, non-diagonal).
template <class R>
void matrix_S(const P<R>& p, R ux, R uy, R S[9][9]) {
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) S[r][c] = 0.0;
  const double om_e = p.se / 2.0 - 1.0;
  const double om_p = p.sp / 2.0 - 1.0;
  S[0][0] = p.s0;
  S[1][1] = p.se;
  S[1][2] = p.k * p.seps * om_e;
  S[1][4] = p.h * ux * p.sq * om_e;
  S[1][6] = p.h * uy * p.sq * om_e;
  S[2][2] = p.seps;
  S[3][3] = p.sj;
  S[4][4] = p.sq;
  S[5][5] = p.sj;
  S[6][6] = p.sq;
  S[7][4] = 2.0 * p.b * ux * p.sq * om_p;
  S[7][6] = -2.0 * p.b * uy * p.sq * om_p;
  S[7][7] = p.sp;
  S[8][4] = p.b * uy * p.sq * om_p;
  S[8][6] = p.b * ux * p.sq * om_p;
  S[8][8] = p.sp;
}

// Cubic-velocity correction matrices of Eq. 11; nonzero entries from the
// supplement's Eq. 34 (row 1), Eq. 37 (row 7) and Eq. 40 (row 8).
template <class R>
void matrices_RTX(const P<R>& p, R ux, R uy, R Rm[9][9], R Tm[9][2], R Xm[9][2]) {
  for (int r = 0; r < 9; ++r) {
    for (int c = 0; c < 9; ++c) Rm[r][c] = 0.0;
    Tm[r][0] = Tm[r][1] = 0.0;
    Xm[r][0] = Xm[r][1] = 0.0;
  }
  const double se = p.se, sp = p.sp, k = p.k, h = p.h, b = p.b, w = p.varpi;
  const R x2 = ux * ux, y2 = uy * uy, xy = ux * uy;
  // Eq. 34
  Rm[1][1] = -se / (4.0 * w) * (9.0 * (1.0 - k) - 2.0 * (3.0 * k + h)) * (x2 + y2);
  Rm[1][7] = -3.0 * sp * (2.0 - se) / (4.0 * (2.0 - sp)) * (9.0 * (1.0 - k) + 2.0 * (3.0 * k + h)) *
             (x2 - y2);
  Rm[1][8] = 12.0 * sp * (2.0 - se) / (2.0 - sp) * (3.0 * k + h) * xy;
  Tm[1][0] = 3.0 * (2.0 - se) / 2.0 * ((1.0 - k) * ux * x2 - (2.0 * k + h) * ux * y2);
  Tm[1][1] = 3.0 * (2.0 - se) / 2.0 * ((1.0 - k) * uy * y2 - (2.0 * k + h) * x2 * uy);
  Xm[1][0] = 9.0 * (2.0 - se) / 2.0 * (2.0 * k + h) * ux * y2;
  Xm[1][1] = 9.0 * (2.0 - se) / 2.0 * (2.0 * k + h) * x2 * uy;
  // Eq. 37
  Rm[7][1] = -se * (2.0 - sp) / (4.0 * w * (2.0 - se)) * (3.0 - 4.0 * b) * (x2 - y2);
  Rm[7][7] = -3.0 * sp / 4.0 * (3.0 + 4.0 * b) * (x2 + y2);
  Rm[7][8] = 0.0;
  Tm[7][0] = (2.0 - sp) / 2.0 * (ux * x2 + 2.0 * b * ux * y2);
  Tm[7][1] = (2.0 - sp) / 2.0 * (-uy * y2 - 2.0 * b * x2 * uy);
  Xm[7][0] = -3.0 * (2.0 - sp) * b * (ux * y2);
  Xm[7][1] = -3.0 * (2.0 - sp) * b * (-x2 * uy);
  // Eq. 40
  Rm[8][1] = se * (2.0 - sp) / (w * (2.0 - se)) * b * xy;
  Rm[8][7] = 0.0;
  Rm[8][8] = 6.0 * sp * b * (x2 + y2);
  Tm[8][0] = -(2.0 - sp) / 2.0 * b * (uy * y2 + 2.0 * x2 * uy);
  Tm[8][1] = -(2.0 - sp) / 2.0 * b * (ux * x2 + 2.0 * ux * y2);
  Xm[8][0] = 3.0 * (2.0 - sp) / 2.0 * b * (uy * y2 + 2.0 * x2 * uy);
  Xm[8][1] = 3.0 * (2.0 - sp) / 2.0 * b * (ux * x2 + 2.0 * ux * y2);
}

// Discrete additional term of Eq. 14 with F~ = F/(G rho c) = G S (c = 1).
template <class R>
void moments_Q(const P<R>& p, R Sx, R Sy, R Qm[9]) {
  const R F2 = p.G2 * (Sx * Sx + Sy * Sy);  // |F~|^2
  for (int r = 0; r < 9; ++r) Qm[r] = 0.0;
  Qm[1] = F2 / 2.0;
  Qm[2] = -F2 / 2.0;
  Qm[7] = p.G2 * (Sx * Sx - Sy * Sy) / 12.0;
  Qm[8] = p.G2 * Sx * Sy / 12.0;
}

// One node: post-streaming f and the force stencil sum
// S = sum_i omega_i rho(x + e_i) e_i (Eq. 12, = grad rho of supplement Eq. 61)
// -> post-collision fbar.
template <class R>
void collide_node(const P<R>& p, const R f[9], R Sx, R Sy, R fbar[9]) {
  // Density, force (Eq. 12) and velocity (Eq. 5).
  R rho = 0.0;
  for (int i = 0; i < 9; ++i) rho += f[i];
  const R Fx = p.G2 * rho * Sx;
  const R Fy = p.G2 * rho * Sy;
  R jx = 0.0, jy = 0.0;
  for (int i = 0; i < 9; ++i) {
    jx += double(EX[i]) * f[i];
    jy += double(EY[i]) * f[i];
  }
  jx += Fx / 2.0;
  jy += Fy / 2.0;
  const R ux = jx / rho, uy = jy / rho;

  // Moments.
  R m[9];
  for (int r = 0; r < 9; ++r) {
    m[r] = 0.0;
    for (int c = 0; c < 9; ++c) m[r] += MMAT[r][c] * f[c];
  }

  // Self-tuning EOS: p_LBE = p_EOS + G^2 rho^2 / 2 (Eq. 18), and
  // p_LBE = c_s^2 (rho + eta) (Eq. 9 with alpha_1 = -1, beta_1 = 1, c_s^2 = 1/3).
  R pe, dpe;
  eos(p, rho, &pe, &dpe);
  const R pL = pe + p.G2 * rho * rho / 2.0;
  const R eta = 3.0 * pL - rho;
  // Local gradients from the force stencil (supplement Eq. 61).
  const R grho[2] = {Sx, Sy};
  const R gp[2] = {(dpe + p.G2 * rho) * Sx, (dpe + p.G2 * rho) * Sy};

  R meq[9], Fm[9], Qm[9];
  moments_eq(p, rho, eta, ux, uy, meq);
  moments_force(Fx, Fy, ux, uy, Fm);
  moments_Q(p, Sx, Sy, Qm);

  R S[9][9], Rm[9][9], Tm[9][2], Xm[9][2];
  matrix_S(p, ux, uy, S);
  matrices_RTX(p, ux, uy, Rm, Tm, Xm);

  // G = m - meq + F_m/2 ; A = (I - S/2) G.
  R G[9], A[9];
  for (int r = 0; r < 9; ++r) G[r] = m[r] - meq[r] + Fm[r] / 2.0;
  for (int r = 0; r < 9; ++r) {
    A[r] = G[r];
    for (int c = 0; c < 9; ++c) A[r] -= S[r][c] * G[c] / 2.0;
  }

  R mbar[9];
  for (int r = 0; r < 9; ++r) {
    R acc = m[r] + Fm[r];
    for (int c = 0; c < 9; ++c) acc -= S[r][c] * G[c];
    if (p.form >= 13)
      for (int c = 0; c < 9; ++c) acc += S[r][c] * Qm[c];
    if (p.form >= 10) {
      for (int c = 0; c < 9; ++c) acc -= Rm[r][c] * A[c];
      acc -= Tm[r][0] * grho[0] + Tm[r][1] * grho[1];
      acc -= Xm[r][0] * gp[0] + Xm[r][1] * gp[1];
    }
    mbar[r] = acc;
  }
  for (int r = 0; r < 9; ++r) {
    fbar[r] = 0.0;
    for (int c = 0; c < 9; ++c) fbar[r] += MINV.inv[r][c] * mbar[c];
  }
}

inline int wrap(int a, int n) { return ((a % n) + n) % n; }

// One time step on a periodic nx x ny lattice.  Arrays are SoA [9][ny][nx]
// of post-collision populations; fin -> fout.
template <class R>
void step(const P<R>& p, int nx, int ny, const R* fin, R* fout) {
  const size_t N = size_t(nx) * ny;
  std::vector<R> f(9 * N), rho(N);
  // Streaming, supplement Eq. 2, in pull form: f_i(x) = fbar_i(x - e_i).
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      R s = 0.0;
      for (int i = 0; i < 9; ++i) {
        const int xs = wrap(x - EX[i], nx), ys = wrap(y - EY[i], ny);
        const R v = fin[i * N + size_t(ys) * nx + xs];
        f[i * N + size_t(y) * nx + x] = v;
        s += v;
      }
      rho[size_t(y) * nx + x] = s;
    }
  // Collision at every node with the neighbour densities of the same time level.
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      R Sx = 0.0, Sy = 0.0;
      for (int i = 1; i < 9; ++i) {
        const R rn = rho[size_t(wrap(y + EY[i], ny)) * nx + wrap(x + EX[i], nx)];
        Sx += WFORCE[i] * rn * double(EX[i]);
        Sy += WFORCE[i] * rn * double(EY[i]);
      }
      R fl[9], fo[9];
      for (int i = 0; i < 9; ++i) fl[i] = f[i * N + size_t(y) * nx + x];
      collide_node(p, fl, Sx, Sy, fo);
      for (int i = 0; i < 9; ++i) fout[i * N + size_t(y) * nx + x] = fo[i];
    }
}

template <class R>
void force_stencil(int nx, int ny, const R* rho, int x, int y, R* Sx, R* Sy) {
  *Sx = 0.0;
  *Sy = 0.0;
  for (int i = 1; i < 9; ++i) {
    const R rn = rho[size_t(wrap(y + EY[i], ny)) * nx + wrap(x + EX[i], nx)];
    *Sx += WFORCE[i] * rn * double(EX[i]);
    *Sy += WFORCE[i] * rn * double(EY[i]);
  }
}

}  // namespace

extern "C" {

int or_version(void) { return 1; }

// Transcribed matrices, for the pin tests.
void or_matrix_M(double* out) {
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) out[r * 9 + c] = MMAT[r][c];
}
void or_matrix_Minv(double* out) {
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) out[r * 9 + c] = MINV.inv[r][c];
}
void or_velocities(int* ex, int* ey) {
  for (int i = 0; i < 9; ++i) {
    ex[i] = EX[i];
    ey[i] = EY[i];
  }
}

void or_eos(const or_params* q, double rho, double* pe, double* dpe) {
  P<double> p = make_params<double>(*q, nullptr);
  eos(p, rho, pe, dpe);
}

void or_moments_eq(const or_params* q, double rho, double eta, double ux, double uy, double* meq) {
  P<double> p = make_params<double>(*q, nullptr);
  moments_eq(p, rho, eta, ux, uy, meq);
}

void or_moments_force(double Fx, double Fy, double ux, double uy, double* Fm) {
  moments_force<double>(Fx, Fy, ux, uy, Fm);
}

void or_moments_Q(const or_params* q, double Sx, double Sy, double* Qm) {
  P<double> p = make_params<double>(*q, nullptr);
  moments_Q(p, Sx, Sy, Qm);
}

void or_matrices(const or_params* q, double ux, double uy, double* S, double* Rm, double* Tm,
                 double* Xm) {
  P<double> p = make_params<double>(*q, nullptr);
  double s[9][9], r[9][9], t[9][2], x[9][2];
  matrix_S(p, ux, uy, s);
  matrices_RTX(p, ux, uy, r, t, x);
  for (int i = 0; i < 9; ++i) {
    for (int j = 0; j < 9; ++j) {
      S[i * 9 + j] = s[i][j];
      Rm[i * 9 + j] = r[i][j];
    }
    Tm[i * 2 + 0] = t[i][0];
    Tm[i * 2 + 1] = t[i][1];
    Xm[i * 2 + 0] = x[i][0];
    Xm[i * 2 + 1] = x[i][1];
  }
}

void or_collide_node(const or_params* q, const double* f, double Sx, double Sy, double* fbar) {
  P<double> p = make_params<double>(*q, nullptr);
  collide_node(p, f, Sx, Sy, fbar);
}

// Equilibrium populations for initial fields: f_i = (M^-1 m_eq(rho, u))_i with
// eta from the EOS at rho; ux / uy may be null (fluid at rest).  SoA [9][ny][nx].
void or_init_eq(const or_params* q, int nx, int ny, const double* rho0, const double* ux0,
                const double* uy0, double* f) {
  P<double> p = make_params<double>(*q, nullptr);
  const size_t N = size_t(nx) * ny;
  for (size_t n = 0; n < N; ++n) {
    const double rho = rho0[n];
    double pe, dpe;
    eos(p, rho, &pe, &dpe);
    const double eta = 3.0 * (pe + p.G2 * rho * rho / 2.0) - rho;
    double meq[9];
    moments_eq(p, rho, eta, ux0 ? ux0[n] : 0.0, uy0 ? uy0[n] : 0.0, meq);
    for (int r = 0; r < 9; ++r) {
      double acc = 0.0;
      for (int c = 0; c < 9; ++c) acc += MINV.inv[r][c] * meq[c];
      f[r * N + n] = acc;
    }
  }
}

void or_init_feq(const or_params* q, int nx, int ny, const double* rho0, double* f) {
  or_init_eq(q, nx, ny, rho0, nullptr, nullptr, f);
}

// Force stencil sum S = sum_i omega_i rho(x + e_i) e_i of Eq. 12 on a periodic lattice.
void or_force_stencil(int nx, int ny, const double* rho, double* Sx, double* Sy) {
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x)
      force_stencil(nx, ny, rho, x, y, &Sx[size_t(y) * nx + x], &Sy[size_t(y) * nx + x]);
}

// nsteps time steps; fin is not modified; the result is written to fout.
int or_step(const or_params* q, int nx, int ny, const double* fin, double* fout, int nsteps) {
  if (nx < 1 || ny < 1 || nsteps < 0) return -1;
  P<double> p = make_params<double>(*q, nullptr);
  const size_t n9 = 9 * size_t(nx) * ny;
  std::vector<double> a(fin, fin + n9), b(n9);
  for (int s = 0; s < nsteps; ++s) {
    step(p, nx, ny, a.data(), b.data());
    a.swap(b);
  }
  std::memcpy(fout, a.data(), n9 * sizeof(double));
  return 0;
}

// Complex-step version: the populations and the parameters (T, G2, lam) carry
// imaginary perturbations; Im(out)/h is then the directional derivative.
int or_step_cs(const or_params* q, const double* dtheta_im, int nx, int ny, const double* fin_re,
               const double* fin_im, double* fout_re, double* fout_im, int nsteps) {
  if (nx < 1 || ny < 1 || nsteps < 0) return -1;
  P<cplx> p = make_params<cplx>(*q, dtheta_im);
  const size_t n9 = 9 * size_t(nx) * ny;
  std::vector<cplx> a(n9), b(n9);
  for (size_t i = 0; i < n9; ++i) a[i] = cplx(fin_re[i], fin_im ? fin_im[i] : 0.0);
  for (int s = 0; s < nsteps; ++s) {
    step(p, nx, ny, a.data(), b.data());
    a.swap(b);
  }
  for (size_t i = 0; i < n9; ++i) {
    fout_re[i] = a[i].real();
    fout_im[i] = a[i].imag();
  }
  return 0;
}

// Macroscopic fields at the time level of the last collision stored in f
// (post-collision populations): the collision conserves mass and adds F to the
// momentum, so rho = sum_i fbar_i and rho u = sum_i e_i fbar_i - F/2 (Eq. 5).
void or_macro(const or_params* q, int nx, int ny, const double* f, double* rho, double* ux,
              double* uy) {
  P<double> p = make_params<double>(*q, nullptr);
  const size_t N = size_t(nx) * ny;
  for (size_t n = 0; n < N; ++n) {
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += f[i * N + n];
    rho[n] = s;
  }
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t n = size_t(y) * nx + x;
      double Sx, Sy;
      force_stencil(nx, ny, rho, x, y, &Sx, &Sy);
      double jx = 0.0, jy = 0.0;
      for (int i = 0; i < 9; ++i) {
        jx += EX[i] * f[i * N + n];
        jy += EY[i] * f[i * N + n];
      }
      jx -= p.G2 * rho[n] * Sx / 2.0;
      jy -= p.G2 * rho[n] * Sy / 2.0;
      ux[n] = jx / rho[n];
      uy[n] = jy / rho[n];
    }
}

}  // extern "C"
