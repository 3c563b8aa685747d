"""Background cosmology and the FastPM step factors (oracle, float64, torch CPU).

Units: length Mpc/h (comoving), velocity 100 km/s, time 1/H0, so H0 = 1. Flat LCDM without
radiation: E(a) = H(a)/H0 = sqrt(Om a^-3 + 1 - Om).

The paper (Sec. 2.2) evolves dark matter with a FastPM particle-mesh solver whose
"modified kick-drift-kick" factors are chosen so that linear (Zel'dovich) growth is
reproduced exactly for any step size. With momentum p = a^2 dx/dt, the linear solution is
x = q + D(a) s0, p = g_p(a) s0, g = g_f(a) s0, where

    g_p(a) = a^3 E(a) D'(a),     g_f(a) = (3/2) Om D(a) / a,

and d g_p / dt = g_f is the linear growth equation. A kick with the force taken at a_c
from a0 to a1 then uses (g_p(a1) - g_p(a0)) / g_f(a_c), and a drift with the momentum taken
at a_c uses (D(a1) - D(a0)) / g_p(a_c).

D(a) is the growing mode in closed form (Heath 1977):
    D(a) = (5 Om / 2) E(a) \\int_0^a da' / (a' E(a'))^3,
normalised so that D -> a as a -> 0. The integral is evaluated with Gauss-Legendre
quadrature after the substitution a' = a t^2, which makes the integrand analytic on [0, 1].

All functions accept Om as a python float or a 0-d float64 tensor (with requires_grad for
gradients with respect to Om).
"""
from __future__ import annotations

import numpy as np
import torch

_DT = torch.float64
_GL_T, _GL_W = np.polynomial.legendre.leggauss(96)
# map Gauss-Legendre nodes from [-1, 1] to [0, 1]
_GL_T = torch.tensor(0.5 * (_GL_T + 1.0), dtype=_DT)
_GL_W = torch.tensor(0.5 * _GL_W, dtype=_DT)


def _t(x):
    return x if torch.is_tensor(x) else torch.tensor(float(x), dtype=_DT)


def hubble_E(a, om):
    """E(a) = H/H0 for flat LCDM."""
    a, om = _t(a), _t(om)
    return torch.sqrt(om * a ** -3 + (1.0 - om))


def dE_da(a, om):
    a, om = _t(a), _t(om)
    return -1.5 * om * a ** -4 / hubble_E(a, om)


def _heath_integral(a, om):
    """I(a) = int_0^a (a' E(a'))^-3 da', via a' = a t^2:
    (a'E)^-3 = a'^{3/2} (Om + (1-Om) a'^3)^{-3/2}, da' = 2 a t dt  ->
    I = int_0^1 2 a^{5/2} t^4 (Om + (1-Om) a^3 t^6)^{-3/2} dt."""
    a, om = _t(a), _t(om)
    t = _GL_T
    integrand = 2.0 * a ** 2.5 * t ** 4 * (om + (1.0 - om) * a ** 3 * t ** 6) ** -1.5
    return (integrand * _GL_W).sum()


def growth_D(a, om):
    """Linear growth factor D(a) (growing mode, D ~ a at early times)."""
    a, om = _t(a), _t(om)
    return 2.5 * om * hubble_E(a, om) * _heath_integral(a, om)


def growth_dD_da(a, om):
    """dD/da from differentiating the closed form: (5 Om/2)(E' I + E (aE)^-3)."""
    a, om = _t(a), _t(om)
    E = hubble_E(a, om)
    return 2.5 * om * (dE_da(a, om) * _heath_integral(a, om) + E * (a * E) ** -3)


def g_p(a, om):
    """Momentum growth factor g_p = a^3 E D' (p = g_p s0 in linear theory)."""
    a, om = _t(a), _t(om)
    return a ** 3 * hubble_E(a, om) * growth_dD_da(a, om)


def g_f(a, om):
    """Force growth factor g_f = (3/2) Om D / a (g = g_f s0 in linear theory)."""
    a, om = _t(a), _t(om)
    return 1.5 * om * growth_D(a, om) / a


def growth_rate_f(a, om):
    """f = dlnD/dlna."""
    a = _t(a)
    return a * growth_dD_da(a, om) / growth_D(a, om)


def _gl_integral(fn, a0, a1):
    """int_{a0}^{a1} fn(a) da with 96-point Gauss-Legendre (fn smooth on the interval)."""
    a0, a1 = _t(a0), _t(a1)
    x = a0 + (a1 - a0) * _GL_T
    return (a1 - a0) * (fn(x) * _GL_W).sum()


def step_factors(a0, a1, om, kdk_mode: str = "fastpm"):
    """Factors of one kick-drift-kick step from a0 to a1 (a_h = arithmetic midpoint).

    Returns a dict of 0-d tensors:
      K1   first half-kick, force at a0         (p += K1 g(a0))
      dtau drift / hydro step in tau (dtau = dt/a^2), momentum at a_h   (x += dtau p)
      K2   second half-kick, force at a1        (p += K2 g(a1))
      pref1 Poisson prefactor 3 Om / (2 a1) for the force at a1
    fastpm: the FastPM factors (exact for linear growth, Sec. 2.2).
    plain:  K = int dt = int da/(aE), dtau = int da/(a^3 E).
    """
    a0, a1, om = _t(a0), _t(a1), _t(om)
    ah = 0.5 * (a0 + a1)
    if kdk_mode == "fastpm":
        K1 = (g_p(ah, om) - g_p(a0, om)) / g_f(a0, om)
        dtau = (growth_D(a1, om) - growth_D(a0, om)) / g_p(ah, om)
        K2 = (g_p(a1, om) - g_p(ah, om)) / g_f(a1, om)
    elif kdk_mode == "plain":
        K1 = _gl_integral(lambda a: 1.0 / (a * hubble_E(a, om)), a0, ah)
        dtau = _gl_integral(lambda a: 1.0 / (a ** 3 * hubble_E(a, om)), a0, a1)
        K2 = _gl_integral(lambda a: 1.0 / (a * hubble_E(a, om)), ah, a1)
    else:
        raise ValueError(kdk_mode)
    return {"K1": K1, "dtau": dtau, "K2": K2, "pref1": 1.5 * om / a1}


def poisson_prefactor(a, om):
    """3 Om / (2 a): del^2 phi = (3 Om / 2a) delta_tot in these units."""
    return 1.5 * _t(om) / _t(a)


def scale_factors(a_start: float, a_end: float, n_steps: int):
    """Uniform-in-a schedule a_0..a_n (Sec. 2.3.3: a predefined global schedule)."""
    return [a_start + (a_end - a_start) * i / n_steps for i in range(n_steps + 1)]
