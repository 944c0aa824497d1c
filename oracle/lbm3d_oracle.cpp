// Plain FP64 CPU oracle for the three-dimensional (D3Q19) form of the
// self-tuning-EOS multiphase lattice Boltzmann model (arXiv:1809.02390).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
// load this file: only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / reference leg use it.  It shares no code, header, table or
// constant with the CUDA library.
//
// The paper works on D2Q9 and says only that the extension to a 3-D lattice is
// straightforward though tedious (main text, after Eq. 2).  The 3-D model here
// keeps every construction of the paper and takes the coefficients that the
// same analysis gives on the D3Q19 moment set (orthogonal polynomial moments,
// no weights, as in Eq. 2):
//
//   * equilibrium (Eq. 3): the second-order Hermite equilibrium of the lattice
//     plus eta in e (coefficient 19, so that p_LBE = c_s^2 (rho + eta) as in
//     Eq. 9) and beta_2 eta in eps;
//   * forcing (Eq. 4): the second-order Hermite force populations;
//   * S (Eq. 6): e couples to eps through k s_eps omega_e and to q_a through
//     h u_a s_q omega_e; the five traceless second-order rows couple to q through
//     b s_q omega_p times the traceless part of (u qhat + qhat u);
//   * Navier-Stokes level (Eq. 7): cancelling every O(Ma) term of the recovered
//     stress that is not Newtonian gives
//       k beta_2 = -19,  bulk viscosity = (1 - 11 k / 38) (2/3) c_s^2 tau_e,
//     so with varpi again the ratio of the bulk viscosity to the one of the
//     plain model: k = 38 (1 - varpi) / 11, beta_2 = -11 / (2 (1 - varpi)),
//     b = 21 (1 - varpi) / (5 (7 - 18 varpi)), h = 798 varpi (1 - varpi) / (5 (7 - 18 varpi));
//   * discrete additional term (Eq. 14): Q_m = M g with
//       g_i = w_i [3/8 (e_i . F~)^2 + 3/16 |e_i|^2 |F~|^2 - 5/16 |F~|^2],
//     the one form of this kind with no mass and the second-order tensor
//     (2 F~F~ + |F~|^2 I) / 24 of the paper's Q_m (the 2-D Q_m is the same form
//     with -1/4 in place of -5/16);
//   * rate closure (Eq. 16): the steady third-order analysis on D3Q19 leaves
//     error terms proportional to (1 + 5 k / 19) tau_e tau_q - tau_p tau_q and to
//     12 tau_p tau_q - 1; both vanish for tau_p tau_q = (1 + 5k/19) tau_e tau_q = 1/12,
//     and the recovered pressure tensor is then Eq. 17 unchanged.
//   * The cubic-velocity corrections R, T, X (Eq. 10) are not part of the 3-D
//     model: the recovered equations carry the plain lattice's O(Ma^3) error.
//
// The collision is evaluated in plain matrix form:
//   mbar = m + F_m - S (m - m_eq + F_m/2) + S Q_m,   fbar = M^-1 mbar,
// followed by pull streaming on a periodic nx x ny x nz lattice.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

constexpr int Q = 19;

// D3Q19 velocities: rest, six axis directions, twelve edge directions.
const int EX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
const int EY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
const int EZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

// Lattice weights: 1/3 rest, 1/18 axis, 1/36 edge.
double weight(int i) {
  const int n2 = EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i];
  return n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Interaction-force weights of Eq. 12 on D3Q19: omega(1) = 1/6, omega(2) = 1/12
// (three times the lattice weights, as on D2Q9: sum_i omega_i e_i e_i = I).
double omega_force(int i) {
  const int n2 = EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i];
  return n2 == 0 ? 0.0 : (n2 == 1 ? 1.0 / 6.0 : 1.0 / 12.0);
}

// Moment polynomials, in the order
//   rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww,
//   p_xy, p_yz, p_xz, m_x, m_y, m_z.
double moment_poly(int r, int i) {
  const double x = EX[i], y = EY[i], z = EZ[i];
  const double n2 = x * x + y * y + z * z;
  switch (r) {
    case 0: return 1.0;
    case 1: return 19.0 * n2 - 30.0;
    case 2: return (21.0 * n2 * n2 - 53.0 * n2 + 24.0) / 2.0;
    case 3: return x;
    case 4: return (5.0 * n2 - 9.0) * x;
    case 5: return y;
    case 6: return (5.0 * n2 - 9.0) * y;
    case 7: return z;
    case 8: return (5.0 * n2 - 9.0) * z;
    case 9: return 3.0 * x * x - n2;
    case 10: return (3.0 * n2 - 5.0) * (3.0 * x * x - n2);
    case 11: return y * y - z * z;
    case 12: return (3.0 * n2 - 5.0) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
  }
}

enum { R_RHO = 0, R_E, R_EPS, R_JX, R_QX, R_JY, R_QY, R_JZ, R_QZ, R_PXX, R_PIXX, R_PWW, R_PIWW,
       R_PXY, R_PYZ, R_PXZ, R_MX, R_MY, R_MZ };

struct Matrices {
  double M[Q][Q], Minv[Q][Q];
  Matrices() {
    for (int r = 0; r < Q; ++r)
      for (int i = 0; i < Q; ++i) M[r][i] = moment_poly(r, i);
    // M^-1 by Gauss-Jordan elimination with partial pivoting.
    double a[Q][2 * Q];
    for (int r = 0; r < Q; ++r)
      for (int c = 0; c < 2 * Q; ++c) a[r][c] = c < Q ? M[r][c] : (c - Q == r ? 1.0 : 0.0);
    for (int col = 0; col < Q; ++col) {
      int piv = col;
      for (int r = col + 1; r < Q; ++r)
        if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
      for (int c = 0; c < 2 * Q; ++c) std::swap(a[col][c], a[piv][c]);
      const double d = a[col][col];
      for (int c = 0; c < 2 * Q; ++c) a[col][c] /= d;
      for (int r = 0; r < Q; ++r) {
        if (r == col) continue;
        const double fac = a[r][col];
        for (int c = 0; c < 2 * Q; ++c) a[r][c] -= fac * a[col][c];
      }
    }
    for (int r = 0; r < Q; ++r)
      for (int c = 0; c < Q; ++c) Minv[r][c] = a[r][c + Q];
  }
};
const Matrices MAT;

void to_moments(const double f[Q], double m[Q]) {
  for (int r = 0; r < Q; ++r) {
    m[r] = 0.0;
    for (int i = 0; i < Q; ++i) m[r] += MAT.M[r][i] * f[i];
  }
}

}  // namespace

extern "C" {

// Lattice-unit parameters (c = 1, delta_x = 1).  The first fields are those of
// the D2Q9 oracle; s_m and s_pi relax the third-order m and the anisotropic
// fourth-order pi moments that D2Q9 does not have.
typedef struct {
  int32_t eos;   // 0: van der Waals, 1: Carnahan-Starling (Eq. 20), 2: ideal gas p = rho/3
  int32_t form;  // 13: mbar of Eq. 13 without R, T, X; 2: without S Q_m; 6: with S Q_m but
                 // without the velocity-dependent entries of S (h = b = 0), for the
                 // sensitivity checks of the tests
  double eos_a, eos_b, R_gas, T;
  double lam;    // pressure scale K_EOS / c^2
  double G2;     // interaction strength G^2 / c^2 of Eq. 12
  double varpi;  // bulk-viscosity ratio (Eq. 7)
  double s0, se, seps, sj, sq, sp, sm, spi;
} or3_params;

}  // extern "C"

namespace {

struct P3 {
  or3_params q;
  double beta2, k, h, b;
};

P3 make_params(const or3_params& q) {
  P3 p;
  p.q = q;
  const double w = q.varpi;
  p.k = 38.0 * (1.0 - w) / 11.0;
  p.beta2 = (w == 1.0) ? 0.0 : -19.0 / p.k;
  p.b = 21.0 * (1.0 - w) / (5.0 * (7.0 - 18.0 * w));
  p.h = 798.0 * w * (1.0 - w) / (5.0 * (7.0 - 18.0 * w));
  if (q.form == 6) p.h = p.b = 0.0;
  return p;
}

// p_EOS / c^2 (scaled by K_EOS / c^2) as in the D2Q9 oracle: vdW, Carnahan-Starling
// (Eq. 20) or the ideal gas.
void eos(const P3& p, double rho, double* pe) {
  const or3_params& q = p.q;
  if (q.eos == 0) {
    *pe = q.lam * (rho * q.R_gas * q.T / (1.0 - q.eos_b * rho) - q.eos_a * rho * rho);
  } else if (q.eos == 1) {
    const double t = q.eos_b * rho / 4.0;
    const double om = 1.0 - t;
    const double z = (1.0 + t + t * t - t * t * t) / (om * om * om);
    *pe = q.lam * (rho * q.R_gas * q.T * z - q.eos_a * rho * rho);
  } else {
    *pe = rho / 3.0;
  }
}

// eta of the self-tuning EOS: p_LBE = p_EOS + G^2 rho^2 / 2 (Eq. 18) = (rho + eta)/3 (Eq. 9).
double eta_of(const P3& p, double rho) {
  double pe;
  eos(p, rho, &pe);
  return 3.0 * (pe + p.q.G2 * rho * rho / 2.0) - rho;
}

// m_eq = M f^H(rho, u) + eta (0, 19, beta_2, 0, ..., 0), f^H the second-order
// Hermite equilibrium w_i rho [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u].
void moments_eq(const P3& p, double rho, double eta, const double u[3], double meq[Q]) {
  double fh[Q];
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    const double eu = EX[i] * u[0] + EY[i] * u[1] + EZ[i] * u[2];
    fh[i] = weight(i) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
  }
  to_moments(fh, meq);
  meq[R_E] += 19.0 * eta;
  meq[R_EPS] += p.beta2 * eta;
}

// F_m = M F_v with the second-order Hermite force populations
// F_v,i = w_i [3 (e_i - u).F + 9 (e_i.u)(e_i.F)].
void moments_force(const double F[3], const double u[3], double Fm[Q]) {
  double fv[Q];
  const double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  for (int i = 0; i < Q; ++i) {
    const double eF = EX[i] * F[0] + EY[i] * F[1] + EZ[i] * F[2];
    const double eu = EX[i] * u[0] + EY[i] * u[1] + EZ[i] * u[2];
    fv[i] = weight(i) * (3.0 * (eF - uF) + 9.0 * eu * eF);
  }
  to_moments(fv, Fm);
}

// Q_m = M g, g_i = w_i [3/8 (e_i.F~)^2 + 3/16 |e_i|^2 |F~|^2 - 5/16 |F~|^2],
// F~ = F / (G rho) = G s with s the force stencil sum (c = 1).
void moments_Q(const P3& p, const double s[3], double Qm[Q]) {
  double g[Q];
  const double G2 = p.q.G2;
  const double F2 = G2 * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  for (int i = 0; i < Q; ++i) {
    const double es = EX[i] * s[0] + EY[i] * s[1] + EZ[i] * s[2];
    const double n2 = EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i];
    g[i] = weight(i) * (3.0 / 8.0 * G2 * es * es + 3.0 / 16.0 * n2 * F2 - 5.0 / 16.0 * F2);
  }
  to_moments(g, Qm);
}

// Collision matrix S (3-D form of Eq. 6), assembled entry by entry.
void matrix_S(const P3& p, const double u[3], double S[Q][Q]) {
  const or3_params& q = p.q;
  for (int r = 0; r < Q; ++r)
    for (int c = 0; c < Q; ++c) S[r][c] = 0.0;
  const double om_e = q.se / 2.0 - 1.0, om_p = q.sp / 2.0 - 1.0;
  const double diag[Q] = {q.s0, q.se, q.seps, q.sj, q.sq, q.sj, q.sq, q.sj, q.sq, q.sp,
                          q.spi, q.sp, q.spi, q.sp, q.sp, q.sp, q.sm, q.sm, q.sm};
  for (int r = 0; r < Q; ++r) S[r][r] = diag[r];
  // e row: k s_eps omega_e on eps, h u_a s_q omega_e on q_a.
  S[R_E][R_EPS] = p.k * q.seps * om_e;
  S[R_E][R_QX] = p.h * u[0] * q.sq * om_e;
  S[R_E][R_QY] = p.h * u[1] * q.sq * om_e;
  S[R_E][R_QZ] = p.h * u[2] * q.sq * om_e;
  // Traceless second-order rows: b s_q omega_p times the row's component of
  // (u qhat + qhat u): 3p_xx ~ 2T_xx - T_yy - T_zz, p_ww ~ T_yy - T_zz, p_ab ~ T_ab.
  const double c = p.b * q.sq * om_p;
  S[R_PXX][R_QX] = 4.0 * c * u[0];
  S[R_PXX][R_QY] = -2.0 * c * u[1];
  S[R_PXX][R_QZ] = -2.0 * c * u[2];
  S[R_PWW][R_QY] = 2.0 * c * u[1];
  S[R_PWW][R_QZ] = -2.0 * c * u[2];
  S[R_PXY][R_QX] = c * u[1];
  S[R_PXY][R_QY] = c * u[0];
  S[R_PYZ][R_QY] = c * u[2];
  S[R_PYZ][R_QZ] = c * u[1];
  S[R_PXZ][R_QX] = c * u[2];
  S[R_PXZ][R_QZ] = c * u[0];
}

// One node: post-streaming f and the force stencil sum s -> post-collision fbar.
void collide_node(const P3& p, const double f[Q], const double s[3], double fbar[Q]) {
  double rho = 0.0;
  for (int i = 0; i < Q; ++i) rho += f[i];
  const double F[3] = {p.q.G2 * rho * s[0], p.q.G2 * rho * s[1], p.q.G2 * rho * s[2]};
  double j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < Q; ++i) {
    j[0] += EX[i] * f[i];
    j[1] += EY[i] * f[i];
    j[2] += EZ[i] * f[i];
  }
  const double u[3] = {(j[0] + F[0] / 2.0) / rho, (j[1] + F[1] / 2.0) / rho, (j[2] + F[2] / 2.0) / rho};
  const double eta = eta_of(p, rho);

  double m[Q], meq[Q], Fm[Q], Qm[Q], S[Q][Q];
  to_moments(f, m);
  moments_eq(p, rho, eta, u, meq);
  moments_force(F, u, Fm);
  moments_Q(p, s, Qm);
  matrix_S(p, u, S);

  double G[Q];
  for (int r = 0; r < Q; ++r) G[r] = m[r] - meq[r] + Fm[r] / 2.0;
  double mbar[Q];
  for (int r = 0; r < Q; ++r) {
    double acc = m[r] + Fm[r];
    for (int c = 0; c < Q; ++c) acc -= S[r][c] * G[c];
    if (p.q.form != 2)
      for (int c = 0; c < Q; ++c) acc += S[r][c] * Qm[c];
    mbar[r] = acc;
  }
  for (int i = 0; i < Q; ++i) {
    fbar[i] = 0.0;
    for (int r = 0; r < Q; ++r) fbar[i] += MAT.Minv[i][r] * mbar[r];
  }
}

inline int wrap(int a, int n) { return ((a % n) + n) % n; }

struct Grid {
  int nx, ny, nz;
  size_t N() const { return size_t(nx) * ny * nz; }
  size_t at(int x, int y, int z) const { return (size_t(z) * ny + y) * nx + x; }
};

void force_stencil(const Grid& g, const double* rho, int x, int y, int z, double s[3]) {
  s[0] = s[1] = s[2] = 0.0;
  for (int i = 1; i < Q; ++i) {
    const double rn = rho[g.at(wrap(x + EX[i], g.nx), wrap(y + EY[i], g.ny), wrap(z + EZ[i], g.nz))];
    s[0] += omega_force(i) * rn * EX[i];
    s[1] += omega_force(i) * rn * EY[i];
    s[2] += omega_force(i) * rn * EZ[i];
  }
}

// One time step; arrays are SoA [19][nz][ny][nx] of post-collision populations.
void step(const P3& p, const Grid& g, const double* fin, double* fout) {
  const size_t N = g.N();
  std::vector<double> f(Q * N), rho(N);
  // Pull streaming: f_i(x) = fbar_i(x - e_i).
  for (int z = 0; z < g.nz; ++z)
    for (int y = 0; y < g.ny; ++y)
      for (int x = 0; x < g.nx; ++x) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) {
          const double v = fin[i * N + g.at(wrap(x - EX[i], g.nx), wrap(y - EY[i], g.ny), wrap(z - EZ[i], g.nz))];
          f[i * N + g.at(x, y, z)] = v;
          s += v;
        }
        rho[g.at(x, y, z)] = s;
      }
  for (int z = 0; z < g.nz; ++z)
    for (int y = 0; y < g.ny; ++y)
      for (int x = 0; x < g.nx; ++x) {
        double s[3], fl[Q], fo[Q];
        force_stencil(g, rho.data(), x, y, z, s);
        for (int i = 0; i < Q; ++i) fl[i] = f[i * N + g.at(x, y, z)];
        collide_node(p, fl, s, fo);
        for (int i = 0; i < Q; ++i) fout[i * N + g.at(x, y, z)] = fo[i];
      }
}

}  // namespace

extern "C" {

int or3_version(void) { return 1; }

void or3_velocities(int* ex, int* ey, int* ez) {
  for (int i = 0; i < Q; ++i) {
    ex[i] = EX[i];
    ey[i] = EY[i];
    ez[i] = EZ[i];
  }
}
void or3_weights(double* w) {
  for (int i = 0; i < Q; ++i) w[i] = weight(i);
}
void or3_matrix_M(double* out) {
  for (int r = 0; r < Q; ++r)
    for (int c = 0; c < Q; ++c) out[r * Q + c] = MAT.M[r][c];
}
void or3_matrix_Minv(double* out) {
  for (int r = 0; r < Q; ++r)
    for (int c = 0; c < Q; ++c) out[r * Q + c] = MAT.Minv[r][c];
}
// Coefficients (beta_2, k, h, b) of the 3-D Eq. 7.
void or3_coefficients(const or3_params* q, double* out) {
  P3 p = make_params(*q);
  out[0] = p.beta2;
  out[1] = p.k;
  out[2] = p.h;
  out[3] = p.b;
}
void or3_moments_eq(const or3_params* q, double rho, double eta, const double* u, double* meq) {
  moments_eq(make_params(*q), rho, eta, u, meq);
}
void or3_moments_force(const double* F, const double* u, double* Fm) { moments_force(F, u, Fm); }
void or3_moments_Q(const or3_params* q, const double* s, double* Qm) { moments_Q(make_params(*q), s, Qm); }
void or3_matrix_S(const or3_params* q, const double* u, double* out) {
  double S[Q][Q];
  matrix_S(make_params(*q), u, S);
  for (int r = 0; r < Q; ++r)
    for (int c = 0; c < Q; ++c) out[r * Q + c] = S[r][c];
}
void or3_collide_node(const or3_params* q, const double* f, const double* s, double* fbar) {
  collide_node(make_params(*q), f, s, fbar);
}

// Equilibrium populations (M^-1 m_eq(rho, u))_i with eta from the EOS; u may be
// null (rest).  SoA [19][nz][ny][nx].
void or3_init_eq(const or3_params* q, int nx, int ny, int nz, const double* rho0, const double* ux,
                 const double* uy, const double* uz, double* f) {
  P3 p = make_params(*q);
  const size_t N = size_t(nx) * ny * nz;
  for (size_t n = 0; n < N; ++n) {
    const double u[3] = {ux ? ux[n] : 0.0, uy ? uy[n] : 0.0, uz ? uz[n] : 0.0};
    double meq[Q];
    moments_eq(p, rho0[n], eta_of(p, rho0[n]), u, meq);
    for (int i = 0; i < Q; ++i) {
      double acc = 0.0;
      for (int r = 0; r < Q; ++r) acc += MAT.Minv[i][r] * meq[r];
      f[i * N + n] = acc;
    }
  }
}

void or3_force_stencil(int nx, int ny, int nz, const double* rho, double* sx, double* sy, double* sz) {
  const Grid g{nx, ny, nz};
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double s[3];
        force_stencil(g, rho, x, y, z, s);
        sx[g.at(x, y, z)] = s[0];
        sy[g.at(x, y, z)] = s[1];
        sz[g.at(x, y, z)] = s[2];
      }
}

int or3_step(const or3_params* q, int nx, int ny, int nz, const double* fin, double* fout, int nsteps) {
  if (nx < 1 || ny < 1 || nz < 1 || nsteps < 0) return -1;
  const P3 p = make_params(*q);
  const Grid g{nx, ny, nz};
  const size_t n = Q * g.N();
  std::vector<double> a(fin, fin + n), b(n);
  for (int s = 0; s < nsteps; ++s) {
    step(p, g, a.data(), b.data());
    a.swap(b);
  }
  std::memcpy(fout, a.data(), n * sizeof(double));
  return 0;
}

// rho = sum_i fbar_i and rho u = sum_i e_i fbar_i - F/2 at the time level of
// the last collision held in f (as for D2Q9, Eq. 5).
void or3_macro(const or3_params* q, int nx, int ny, int nz, const double* f, double* rho, double* ux,
               double* uy, double* uz) {
  const P3 p = make_params(*q);
  const Grid g{nx, ny, nz};
  const size_t N = g.N();
  for (size_t n = 0; n < N; ++n) {
    double s = 0.0;
    for (int i = 0; i < Q; ++i) s += f[i * N + n];
    rho[n] = s;
  }
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const size_t n = g.at(x, y, z);
        double s[3];
        force_stencil(g, rho, x, y, z, s);
        double j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
          j[0] += EX[i] * f[i * N + n];
          j[1] += EY[i] * f[i * N + n];
          j[2] += EZ[i] * f[i * N + n];
        }
        ux[n] = (j[0] - p.q.G2 * rho[n] * s[0] / 2.0) / rho[n];
        uy[n] = (j[1] - p.q.G2 * rho[n] * s[1] / 2.0) / rho[n];
        uz[n] = (j[2] - p.q.G2 * rho[n] * s[2] / 2.0) / rho[n];
      }
}

}  // extern "C"
