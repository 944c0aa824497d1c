// Host-side FP64 thermodynamics and parameter derivation for the library.
//
// Coexistence densities come from the Maxwell construction of the free energy
// given below Eq. 19 (p_EOS = rho psi' - psi): equal pressure and equal chemical
// potential mu = psi' of the gas and liquid branches, solved by bisection on the
// pressure followed by a 2x2 Newton polish.  psi is used in closed form:
//   van der Waals:       psi = K [rho R T ln(rho/(1 - b rho)) - a rho^2]
//   Carnahan-Starling:   psi = K [rho R T (ln rho + (4t - 3t^2)/(1 - t)^2) - a rho^2],
//                        t = b rho / 4   (EOS of Eq. 20)
// The flat-interface thickness and surface tension follow from the pressure
// tensor of Eq. 17: kappa/2 rho'^2 = w(rho) with w = psi - mu* rho + p*, so
// sigma = int sqrt(2 kappa w) drho and W = int sqrt(kappa/(2 w)) drho between the
// 5% and 95% levels (supplement Sec. V), by composite Gauss-Legendre quadrature.
#include "lbm_internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>

namespace lbm {

namespace {

struct Eos {
  int kind;
  double a, b, R, T, K;

  double p_rep(double rho) const {
    if (kind == LB_EOS_VDW) return rho * R * T / (1.0 - b * rho);
    const double t = b * rho / 4.0, om = 1.0 - t;
    return rho * R * T * (1.0 + t + t * t - t * t * t) / (om * om * om);
  }
  double dp_rep(double rho) const {
    if (kind == LB_EOS_VDW) {
      const double om = 1.0 - b * rho;
      return R * T / (om * om);
    }
    const double t = b * rho / 4.0, om = 1.0 - t;
    return R * T * (1.0 + 4.0 * t + 4.0 * t * t - 4.0 * t * t * t + t * t * t * t) / (om * om * om * om);
  }
  double p(double rho) const { return K * (p_rep(rho) - a * rho * rho); }
  double dp(double rho) const { return K * (dp_rep(rho) - 2.0 * a * rho); }
  double psi(double rho) const {
    if (kind == LB_EOS_VDW) return K * (rho * R * T * std::log(rho / (1.0 - b * rho)) - a * rho * rho);
    const double t = b * rho / 4.0, om = 1.0 - t;
    return K * (rho * R * T * (std::log(rho) + (4.0 * t - 3.0 * t * t) / (om * om)) - a * rho * rho);
  }
  double mu(double rho) const {
    if (kind == LB_EOS_VDW) {
      const double om = 1.0 - b * rho;
      return K * (R * T * (std::log(rho / om) + 1.0 / om) - 2.0 * a * rho);
    }
    const double t = b * rho / 4.0, om = 1.0 - t;
    const double g = (4.0 * t - 3.0 * t * t) / (om * om);
    const double tdg = t * (4.0 - 2.0 * t) / (om * om * om);
    return K * (R * T * (std::log(rho) + 1.0 + g + tdg) - 2.0 * a * rho);
  }
  double rho_max() const { return kind == LB_EOS_VDW ? 1.0 / b : 4.0 / b; }
};

// Root of g on [lo, hi] (g(lo), g(hi) of opposite sign) by bisection to adjacency.
template <class F>
double bisect(F g, double lo, double hi) {
  double glo = g(lo);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    const double gm = g(mid);
    if ((gm < 0) == (glo < 0)) {
      lo = mid;
      glo = gm;
    } else {
      hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

bool spinodals(const Eos& e, double* s1, double* s2) {
  const double rmax = e.rho_max();
  const int n = 20000;
  double prev = e.dp(rmax * 0.5 / n);
  int found = 0;
  for (int i = 1; i < n; ++i) {
    const double r = rmax * (i + 0.5) / n;
    const double d = e.dp(r);
    if (found == 0 && prev > 0 && d <= 0) {
      *s1 = bisect([&](double x) { return e.dp(x); }, rmax * (i - 0.5) / n, r);
      found = 1;
    } else if (found == 1 && prev < 0 && d >= 0) {
      *s2 = bisect([&](double x) { return e.dp(x); }, rmax * (i - 0.5) / n, r);
      return true;
    }
    prev = d;
  }
  return false;
}

// Gauss-Legendre nodes and weights, 8 points on [-1, 1].
const double GLX[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                       0.1834346424956498,  0.5255324099163290,  0.7966664774136267,  0.9602898564975363};
const double GLW[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                       0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

template <class F>
double integrate(F g, double lo, double hi, int panels) {
  double acc = 0.0;
  const double h = (hi - lo) / panels;
  for (int k = 0; k < panels; ++k) {
    const double c = lo + (k + 0.5) * h;
    for (int j = 0; j < 8; ++j) acc += GLW[j] * g(c + 0.5 * h * GLX[j]);
  }
  return acc * 0.5 * h;
}

}  // namespace

double critical_temperature(int kind, double a, double b, double R) {
  if (kind == LB_EOS_VDW) return 8.0 * a / (27.0 * R * b);
  // Eq. 20: a = 0.496388 R^2 Tc^2/pc, b = 0.187295 R Tc/pc  =>  Tc = (a/b)(0.187295/0.496388)/R.
  return (a / b) * (0.187295 / 0.496388) / R;
}

int maxwell(int kind, double a, double b, double R, double T, double K, double* rho_g, double* rho_l,
            double* p_star) {
  const Eos e{kind, a, b, R, T, K};
  double s1 = 0, s2 = 0;
  if (!spinodals(e, &s1, &s2)) return -1;
  const double rmax = e.rho_max();
  auto branches = [&](double ps, double* rg, double* rl) {
    *rg = bisect([&](double r) { return e.p(r) - ps; }, 1e-300, s1);
    *rl = bisect([&](double r) { return e.p(r) - ps; }, s2, rmax * (1.0 - 1e-15));
  };
  const double p_hi = e.p(s1);
  const double p_lo = std::fmax(e.p(s2), 0.0);
  const double span = p_hi - p_lo;
  const double ps = bisect(
      [&](double q) {
        double rg, rl;
        branches(q, &rg, &rl);
        return e.mu(rl) - e.mu(rg);
      },
      p_lo + 1e-13 * span, p_hi - 1e-13 * span);
  double rg, rl;
  branches(ps, &rg, &rl);
  // Newton polish of p(rg) = p(rl), mu(rg) = mu(rl); mu' = p'/rho.
  for (int it = 0; it < 8; ++it) {
    const double f1 = e.p(rg) - e.p(rl), f2 = e.mu(rg) - e.mu(rl);
    const double j11 = e.dp(rg), j12 = -e.dp(rl), j21 = e.dp(rg) / rg, j22 = -e.dp(rl) / rl;
    const double det = j11 * j22 - j12 * j21;
    if (det == 0.0) break;
    const double dg = (f1 * j22 - f2 * j12) / det, dl = (j11 * f2 - j21 * f1) / det;
    rg -= dg;
    rl -= dl;
    if (std::fabs(dg) < 1e-16 * rg && std::fabs(dl) < 1e-16 * rl) break;
  }
  *rho_g = rg;
  *rho_l = rl;
  *p_star = 0.5 * (e.p(rg) + e.p(rl));
  return (rg > 0 && rl > rg && rl < rmax) ? 0 : -1;
}

void interface_constants(int kind, double a, double b, double R, double T, double K, double rho_g,
                         double rho_l, double p_star, double* W1, double* sigma1) {
  const Eos e{kind, a, b, R, T, K};
  const double mus = 0.5 * (e.mu(rho_g) + e.mu(rho_l));
  // w relative to its value at rho_g (zero analytically) to cancel round-off.
  const double w0 = e.psi(rho_g) - mus * rho_g + p_star;
  auto w = [&](double r) { return e.psi(r) - mus * r + p_star - w0; };
  const double kap = K * a / 2.0;  // kappa = G^2/4 with G^2 = 2 K_EOS a K_INT^2, K_INT = 1
  *sigma1 = integrate([&](double r) { return std::sqrt(std::fmax(2.0 * kap * w(r), 0.0)); }, rho_g, rho_l, 256);
  const double r5 = 0.95 * rho_g + 0.05 * rho_l, r95 = 0.05 * rho_g + 0.95 * rho_l;
  *W1 = integrate([&](double r) { return std::sqrt(kap / (2.0 * w(r))); }, r5, r95, 256);
}

static thread_local char g_err[512];

const char* thread_error() { return g_err; }

void set_thread_error(const char* msg) {
  std::snprintf(g_err, sizeof(g_err), "%s", msg);
}

int derive(const lb_params* p, lb_derived* d, char* err, size_t errlen) {
  std::memset(d, 0, sizeof(*d));
  auto fail = [&](const char* m) {
    std::snprintf(err, errlen, "%s", m);
    return LB_EINVAL;
  };
  if (!p) return fail("null parameters");
  if (p->nx < 3 || p->ny < 3) return fail("nx and ny must be >= 3");
  if (9 * (int64_t)p->nx * p->ny >= ((int64_t)1 << 31)) return fail("lattice too large: 9 nx ny must be below 2^31");
  if (p->precision < LB_FP64 || p->precision > LB_FP16S) return fail("unknown precision");
  if (p->rounding != LB_ROUND_STOCHASTIC && p->rounding != LB_ROUND_NEAREST) return fail("unknown rounding");
  if (p->layout != LB_LAYOUT_PLANES && p->layout != LB_LAYOUT_ROWS) return fail("unknown layout");
  if (p->reserved1 != 0) return fail("reserved field must be 0");
  if (p->eos != LB_EOS_VDW && p->eos != LB_EOS_CS) return fail("unknown eos");
  if (p->variant < LB_AUTO || p->variant > LB_TWO_PASS) return fail("unknown variant");
  if (!(p->eos_a > 0) || !(p->eos_b > 0) || !(p->R_gas > 0)) return fail("eos_a, eos_b, R_gas must be > 0");
  if (!(p->Tr > 0)) return fail("Tr must be > 0");
  if (!(p->K_eos > 0) || !(p->K_int > 0)) return fail("K_eos and K_int must be > 0");
  const double w = p->varpi == 0.0 ? 1.0 / 6.0 : p->varpi;
  if (!(w > 0) || w == 1.0 || std::fabs(w - 1.0 / 3.0) < 1e-12)
    return fail("varpi must be > 0 and not 1 or 1/3 (singular coefficients of Eq. 7)");
  auto rate_ok = [](double s) { return s > 0.0 && s < 2.0; };
  if (!rate_ok(p->s_p)) return fail("s_p must lie in (0, 2)");

  d->Tc = critical_temperature(p->eos, p->eos_a, p->eos_b, p->R_gas);
  d->T = p->Tr * d->Tc;
  d->rho_g = d->rho_l = d->p_star = NAN;
  d->W1 = d->sigma1 = NAN;
  if (p->Tr < 1.0) {
    if (maxwell(p->eos, p->eos_a, p->eos_b, p->R_gas, d->T, p->K_eos, &d->rho_g, &d->rho_l, &d->p_star) != 0)
      return fail("Maxwell construction failed");
    interface_constants(p->eos, p->eos_a, p->eos_b, p->R_gas, d->T, p->K_eos, d->rho_g, d->rho_l, d->p_star,
                        &d->W1, &d->sigma1);
  } else if (!(p->lam > 0) || !(p->G2 > 0)) {
    return fail("Tr >= 1 has no coexistence: give lam and G2 explicitly");
  }
  const Eos e{p->eos, p->eos_a, p->eos_b, p->R_gas, d->T, p->K_eos};
  // Eq. 22: c_s^2 = K_INT^2 d(p_EOS + K_EOS a rho^2)/drho at rho_l, c^2 = 3 c_s^2.
  if (p->Tr < 1.0) d->c2 = 3.0 * p->K_int * p->K_int * p->K_eos * e.dp_rep(d->rho_l);
  d->lam = p->lam > 0 ? p->lam : p->K_eos / d->c2;
  if (!(p->lam > 0) && !(d->c2 > 0)) return fail("lattice speed from Eq. 22 is not positive");
  // Eq. 21: G^2 = 2 K_INT^2 K_EOS a (dx = 1), carried as G^2/c^2 = G^2 lam / K_EOS.
  d->G2 = p->G2 > 0 ? p->G2 : 2.0 * p->K_int * p->K_int * p->K_eos * p->eos_a * d->lam / p->K_eos;
  if (p->lam > 0) d->c2 = p->K_eos / p->lam;

  const double k = 1.0 - w;
  d->k = k;
  d->h = 6.0 * w * (1.0 - w) / (1.0 - 3.0 * w);
  d->b = (1.0 - w) / (1.0 - 3.0 * w);
  d->beta2 = -2.0 / (1.0 - w);
  d->s_p = p->s_p;
  // Eq. 16: tau_p tau_q = (k + 1) tau_e tau_q = 1/12, tau = 1/s - 1/2.
  const double tau_p = 1.0 / p->s_p - 0.5;
  const double tau_q = 1.0 / (12.0 * tau_p);
  const double tau_e = 1.0 / (12.0 * (k + 1.0) * tau_q);
  d->s_q = p->s_q > 0 ? p->s_q : 1.0 / (tau_q + 0.5);
  d->s_e = p->s_e > 0 ? p->s_e : 1.0 / (tau_e + 0.5);
  d->s_eps = p->s_eps > 0 ? p->s_eps : d->s_e;
  d->s_0 = p->s_0 > 0 ? p->s_0 : 1.0;
  d->s_j = p->s_j > 0 ? p->s_j : 1.0;
  if (!rate_ok(d->s_q) || !rate_ok(d->s_e) || !rate_ok(d->s_eps) || !rate_ok(d->s_0) || !rate_ok(d->s_j))
    return fail("relaxation rates must lie in (0, 2)");
  if (std::isinf(p->rho_ref)) return fail("rho_ref must be finite (or NaN: the mean initial density)");
  return LB_OK;
}

}  // namespace lbm
