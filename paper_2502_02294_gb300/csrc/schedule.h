// Host FP64 background cosmology and step factors (Sec. 2.2 of arXiv 2502.02294).
//
// E(a) = sqrt(Om a^-3 + 1 - Om); growing mode D(a) = (5 Om / 2) E(a) int_0^a (a' E)^-3 da'
// (Heath 1977), evaluated by Gauss-Legendre quadrature after a' = a t^2; D' analytically.
// FastPM factors make linear growth exact: with g_p = a^3 E D' and g_f = 3 Om D / (2a),
//   K1   = (g_p(a_h) - g_p(a_0)) / g_f(a_0)      (force at a_0)
//   dtau = (D(a_1) - D(a_0)) / g_p(a_h)         (momentum at a_h)
//   K2   = (g_p(a_1) - g_p(a_h)) / g_f(a_1)      (force at a_1)
// The plain mode integrates dt = da/(aE) and dtau = da/(a^3 E) instead.
#pragma once

#include <vector>

namespace dh {

struct StepFactors {
  double a0, a1, K1, dtau, K2, pref1;   // pref1 = 3 Om / (2 a1)
  double dK1, ddtau, dK2, dpref1;       // derivatives with respect to Omega_m
};

double cosmo_E(double a, double om);
double growth_D(double a, double om);
double growth_dD(double a, double om);
double growth_gp(double a, double om);
double growth_gf(double a, double om);

StepFactors step_factors(double a0, double a1, double om, int kdk_mode);
std::vector<StepFactors> make_schedule(double a_start, double a_end, int n_steps, double om,
                                       int kdk_mode);

}  // namespace dh
