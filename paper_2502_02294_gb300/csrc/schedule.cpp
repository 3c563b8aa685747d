// Host FP64 background cosmology and FastPM step factors (Sec. 2.2 of arXiv 2502.02294).
#include "schedule.h"

#include <cmath>

namespace dh {

namespace {

// Gauss-Legendre nodes and weights on [0, 1] (Newton iteration on P_n).
struct GaussLegendre {
  std::vector<double> x, w;
  explicit GaussLegendre(int n) : x(n), w(n) {
    for (int i = 0; i < n; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
      double dp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      x[i] = 0.5 * (z + 1.0);
      w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // (2 / ((1-z^2) dp^2)) / 2
    }
  }
};

const GaussLegendre& gl() {
  static GaussLegendre g(96);
  return g;
}

double heath_integral(double a, double om) {
  // int_0^a (a'E)^-3 da' with a' = a t^2: 2 a^{5/2} t^4 (om + (1-om) a^3 t^6)^{-3/2}
  const GaussLegendre& g = gl();
  double s = 0.0;
  for (size_t i = 0; i < g.x.size(); ++i) {
    const double t = g.x[i];
    const double t2 = t * t;
    s += g.w[i] * 2.0 * std::pow(a, 2.5) * t2 * t2 *
         std::pow(om + (1.0 - om) * a * a * a * t2 * t2 * t2, -1.5);
  }
  return s;
}

template <class Fn>
double integrate(Fn f, double a0, double a1) {
  const GaussLegendre& g = gl();
  double s = 0.0;
  for (size_t i = 0; i < g.x.size(); ++i) s += g.w[i] * f(a0 + (a1 - a0) * g.x[i]);
  return (a1 - a0) * s;
}

struct Factors {
  double K1, dtau, K2, pref1;
};

Factors factors(double a0, double a1, double om, int kdk_mode) {
  const double ah = 0.5 * (a0 + a1);
  Factors f;
  if (kdk_mode == 0) {
    f.K1 = (growth_gp(ah, om) - growth_gp(a0, om)) / growth_gf(a0, om);
    f.dtau = (growth_D(a1, om) - growth_D(a0, om)) / growth_gp(ah, om);
    f.K2 = (growth_gp(a1, om) - growth_gp(ah, om)) / growth_gf(a1, om);
  } else {
    auto dt = [om](double a) { return 1.0 / (a * cosmo_E(a, om)); };
    auto dtau = [om](double a) { return 1.0 / (a * a * a * cosmo_E(a, om)); };
    f.K1 = integrate(dt, a0, ah);
    f.dtau = integrate(dtau, a0, a1);
    f.K2 = integrate(dt, ah, a1);
  }
  f.pref1 = 1.5 * om / a1;
  return f;
}

}  // namespace

double cosmo_E(double a, double om) { return std::sqrt(om / (a * a * a) + 1.0 - om); }

double growth_D(double a, double om) { return 2.5 * om * cosmo_E(a, om) * heath_integral(a, om); }

double growth_dD(double a, double om) {
  const double E = cosmo_E(a, om);
  const double dE = -1.5 * om / (a * a * a * a) / E;
  const double aE = a * E;
  return 2.5 * om * (dE * heath_integral(a, om) + E / (aE * aE * aE));
}

double growth_gp(double a, double om) { return a * a * a * cosmo_E(a, om) * growth_dD(a, om); }

double growth_gf(double a, double om) { return 1.5 * om * growth_D(a, om) / a; }

StepFactors step_factors(double a0, double a1, double om, int kdk_mode) {
  const Factors f = factors(a0, a1, om, kdk_mode);
  const double h = 1e-5 * om;
  const Factors fp = factors(a0, a1, om + h, kdk_mode);
  const Factors fm = factors(a0, a1, om - h, kdk_mode);
  StepFactors s;
  s.a0 = a0;
  s.a1 = a1;
  s.K1 = f.K1;
  s.dtau = f.dtau;
  s.K2 = f.K2;
  s.pref1 = f.pref1;
  s.dK1 = (fp.K1 - fm.K1) / (2 * h);
  s.ddtau = (fp.dtau - fm.dtau) / (2 * h);
  s.dK2 = (fp.K2 - fm.K2) / (2 * h);
  s.dpref1 = 1.5 / a1;
  return s;
}

std::vector<StepFactors> make_schedule(double a_start, double a_end, int n_steps, double om,
                                       int kdk_mode) {
  std::vector<StepFactors> out;
  out.reserve(n_steps);
  for (int i = 0; i < n_steps; ++i) {
    const double a0 = a_start + (a_end - a_start) * i / n_steps;
    const double a1 = a_start + (a_end - a_start) * (i + 1) / n_steps;
    out.push_back(step_factors(a0, a1, om, kdk_mode));
  }
  return out;
}

}  // namespace dh
