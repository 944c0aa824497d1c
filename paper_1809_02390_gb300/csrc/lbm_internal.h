// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/lbm.h"

namespace lbm {

// Host thermodynamics and parameter derivation (lbm_thermo.cpp).
double critical_temperature(int kind, double a, double b, double R);
int maxwell(int kind, double a, double b, double R, double T, double K, double* rho_g, double* rho_l,
            double* p_star);
void interface_constants(int kind, double a, double b, double R, double T, double K, double rho_g,
                         double rho_l, double p_star, double* W1, double* sigma1);
int derive(const lb_params* p, lb_derived* d, char* err, size_t errlen);
const char* thread_error();
void set_thread_error(const char* msg);

// Per-launch constants of the collision, precomputed on the host in FP64
// (layout identical for float and double instantiations).
template <typename real>
struct Coef {
  int eos;        // LB_EOS_VDW or LB_EOS_CS
  real G2;        // G^2 / c^2
  real lam;       // K_EOS / c^2
  real RT;        // R T
  real a;         // EOS attraction
  real bq;        // b (vdW) or b/4 (CS): the packing variable is bq * rho
  real beta2;     // Eq. 7
  // Step (2) of the execution sequence (supplement Sec. IV).
  real hk_seps, hh_sq, b_sq, hb_sq;  // k s_eps / 2, h s_q / 2, b s_q, b s_q / 2
  // Step (3): 1 - s/2 for the non-conserved moments.
  real om_e, om_eps, om_q, om_p;
  // Step (4): R entries are these constants times a velocity monomial (supplement Eqs. 34, 37, 40).
  real R11, R17, R18, R71, R77, R81, R88;
  real T1a, T1b, X1;  // 3(2-s_e)/2 (1-k), 3(2-s_e)/2 (2k+h), 9(2-s_e)/2 (2k+h)
  real T7, T7b, X7;   // (2-s_p)/2, (2-s_p) b, -3 (2-s_p) b
  real T8, X8;        // -(2-s_p) b / 2, 3 (2-s_p) b / 2
  // Step (6): S Q_m with Q_m of Eq. 14 and F~ = G S.
  real Q1, Q2, Q78;   // (s_e - k (s_e/2 - 1) s_eps)/2, -s_eps/2, s_p/12
  real rho_ref;       // storage shift
};

template <typename real>
Coef<real> make_coef(const lb_params& p, const lb_derived& d);

}  // namespace lbm
