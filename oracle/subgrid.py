"""Stochastic star formation and energy injection (oracle, float64, torch CPU).

Sec. 2.4.1 (toy model): cells denser than a threshold and colder than T_c form stars with a
probability set by the rate Pi_0; each event heats its own gas by the specific energy E_0.
Sec. 2.4.2 (differentiation): the class probability uses sigmoid thresholds,

    pi_0(rho, T) = Pi_0 sigma((delta - delta_c) / w_delta) sigma((T_c - T) / w_T),

and the discrete draw is relaxed with Gumbel-softmax at temperature tau (Eq.
gumbelsoftmax), with the Gumbel(0, 1) pair (g_0, g_1) treated as an input (Eq. reparam):

    zhat = exp((ln pi_0 + g_0)/tau) / (exp((ln pi_0 + g_0)/tau) + exp((ln(1 - pi_0) + g_1)/tau))
         = sigma(l / tau),   l = ln pi_0 - ln(1 - pi_0) + g_0 - g_1.

The second line is the same number written so that it neither overflows nor takes the log
of an underflowed pi_0: ln pi_0 = ln Pi_0 + log sigma(x1) + log sigma(x2) with
log sigma(x) = -softplus(-x), and ln(1 - pi_0) = log1p(-pi_0). The hard (tau -> 0) event is
l > 0, the Gumbel-max sample of the Bernoulli(pi_0) variable.

Readings of what the paper leaves open: delta = rho / rho_gas_mean - 1 with rho_gas_mean =
f_b; T = (gamma - 1) mu m_p e / k_B from the specific internal energy
e = (eps - |m|^2/(2 rho)) / (a^2 rho); E_0 is a specific energy in (100 km/s)^2 added to
the cell's own e times zhat (the forward pass injects the relaxed zhat); w_delta, w_T are
fixed hyper-parameters. The UV-background temperature floor T_0 (rho / rho_gas_mean)^(gamma_T
- 1) is applied after the injection, e <- max(e, e_floor) (d/de at a tie goes to e), and
only when T_0 > 0 (T_0 = 0: no UV background, as in the paper, which has no heating term).
"""
from __future__ import annotations

import torch

K_B = 1.380649e-23          # J/K (exact, SI 2019)
M_P = 1.67262192595e-27     # kg (CODATA 2022)
V_UNIT = 1.0e5              # m/s: code velocity unit 100 km/s


def t_per_e(gamma: float, mu: float) -> float:
    """Temperature [K] per unit specific internal energy [(100 km/s)^2]."""
    return (gamma - 1.0) * mu * M_P * V_UNIT ** 2 / K_B


def _log_sigmoid(x):
    return -torch.nn.functional.softplus(-x)


def subgrid(U, a, prm, g0, g1):
    """One subgrid update at scale factor a.

    U: [5, n, n, n]; prm: dict with gamma, mu, f_b, delta_c, Pi0, E0, T_c, w_delta, w_T, tau,
    T0_uv, gamma_uv (tensors or floats); g0, g1: Gumbel draws [n, n, n].
    Returns (U_new, zhat, events(bool)).
    """
    gamma = prm["gamma"]
    rho, m, eps = U[0], U[1:4], U[4]
    ke = (m * m).sum(0) / (2.0 * rho)
    e = (eps - ke) / (a * a * rho)
    tpe = t_per_e(gamma, prm["mu"])
    T = tpe * e
    delta = rho / prm["f_b"] - 1.0
    x1 = (delta - prm["delta_c"]) / prm["w_delta"]
    x2 = (prm["T_c"] - T) / prm["w_T"]
    lnpi = torch.log(torch.as_tensor(prm["Pi0"], dtype=rho.dtype)) + _log_sigmoid(x1) + _log_sigmoid(x2)
    pi0 = torch.exp(lnpi)
    logit = lnpi - torch.log1p(-pi0) + g0 - g1
    zhat = torch.sigmoid(logit / prm["tau"])
    events = logit.detach() > 0
    e1 = e + prm["E0"] * zhat
    if bool((torch.as_tensor(prm["T0_uv"]) > 0).all()):  # a float, or a tensor (per cell)
        e_floor = (prm["T0_uv"] / tpe) * (rho / prm["f_b"]) ** (prm["gamma_uv"] - 1.0)
        e2 = torch.where(e1 >= e_floor, e1, e_floor)
    else:
        e2 = e1
    eps_new = ke + a * a * rho * e2
    return torch.cat([U[:4], eps_new[None]]), zhat, events


def gumbel_softmax_literal(pi0, g0, g1, tau):
    """Eq. gumbelsoftmax exactly as printed (overflows for small tau; used only to pin the
    stable form above)."""
    a = torch.exp((torch.log(pi0) + g0) / tau)
    b = torch.exp((torch.log(1.0 - pi0) + g1) / tau)
    return a / (a + b)
