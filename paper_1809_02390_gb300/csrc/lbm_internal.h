// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include "lbm.h"

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

}  // namespace lbm
