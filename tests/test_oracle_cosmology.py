"""Pins of the oracle's background cosmology and FastPM step factors (Sec. 2.2).

Each check is against something other than the oracle's own formulas: the Einstein-de
Sitter closed form, two published fitting formulas for LCDM growth, the growth ODE itself
(by finite differences) and the defining property of the FastPM factors (exact linear
growth for any step size)."""
import math

import pytest
import torch

from oracle import cosmology as C


@pytest.mark.parametrize("a", [0.05, 0.1, 0.37, 1.0])
def test_einstein_de_sitter_closed_form(a):
    # Om = 1: D = a, D' = 1, E = a^-3/2 -> g_p = a^3 a^-3/2 = a^3/2, g_f = 3/2
    assert abs(C.growth_D(a, 1.0).item() - a) < 1e-12
    assert abs(C.growth_dD_da(a, 1.0).item() - 1.0) < 1e-12
    assert abs(C.g_p(a, 1.0).item() - a ** 1.5) < 1e-12
    assert abs(C.g_f(a, 1.0).item() - 1.5) < 1e-12


def test_growth_suppression_carroll_press_turner():
    # Carroll, Press & Turner (1992) fitting formula for D(a=1)/a in flat LCDM (~1% accurate)
    om, ol = 0.3, 0.7
    cpt = 2.5 * om / (om ** (4.0 / 7.0) - ol + (1 + om / 2) * (1 + ol / 70))
    assert abs(C.growth_D(1.0, om).item() / cpt - 1.0) < 0.01


@pytest.mark.parametrize("a", [0.5, 1.0])
def test_growth_rate_linder_index(a):
    # Linder (2005): f = Om(a)^0.55, a fit good to better than 1% in LCDM
    om = 0.3
    oma = om * a ** -3 / C.hubble_E(a, om).item() ** 2
    assert abs(C.growth_rate_f(a, om).item() / oma ** 0.55 - 1.0) < 0.01


def test_early_time_normalisation():
    assert abs(C.growth_D(1e-3, 0.3).item() / 1e-3 - 1.0) < 1e-5


@pytest.mark.parametrize("a", [0.07, 0.3, 0.9])
def test_growth_ode_by_finite_differences(a):
    # d g_p / dt = g_f, i.e. (d g_p / da) a E(a) = g_f(a); and D' matches a central FD of D
    om, h = 0.3, 1e-5
    dgp = (C.g_p(a + h, om) - C.g_p(a - h, om)).item() / (2 * h)
    lhs = dgp * a * C.hubble_E(a, om).item()
    assert abs(lhs / C.g_f(a, om).item() - 1.0) < 1e-8
    dD = (C.growth_D(a + h, om) - C.growth_D(a - h, om)).item() / (2 * h)
    assert abs(dD / C.growth_dD_da(a, om).item() - 1.0) < 1e-8


def test_fastpm_kdk_exact_for_linear_growth():
    # Linear theory: x = D s0, p = g_p s0, force g = g_f s0. Kick-drift-kick with the
    # FastPM factors must reproduce it exactly after any number of coarse steps.
    om, s0 = 0.3, 0.7
    a = C.scale_factors(0.05, 1.0, 7)
    x = C.growth_D(a[0], om).item() * s0
    p = C.g_p(a[0], om).item() * s0
    for a0, a1 in zip(a[:-1], a[1:]):
        f = C.step_factors(a0, a1, om, "fastpm")
        # force of the linear solution at the current position: g = g_f(a) x / D(a)
        p += f["K1"].item() * C.g_f(a0, om).item() * x / C.growth_D(a0, om).item()
        x += f["dtau"].item() * p
        p += f["K2"].item() * C.g_f(a1, om).item() * x / C.growth_D(a1, om).item()
        assert abs(x / (C.growth_D(a1, om).item() * s0) - 1.0) < 1e-12
        assert abs(p / (C.g_p(a1, om).item() * s0) - 1.0) < 1e-12


def test_plain_factors_converge_to_fastpm():
    # The FastPM kicks weight the force by its linear growth over the half step, so they
    # differ from int dt at first order in da; the drift (D(a1)-D(a0))/g_p(a_h) is a
    # midpoint rule for int dt/a^2 and agrees at second order.
    om = 0.3
    rel = {}
    for da in (0.02, 0.01):
        f = C.step_factors(0.5, 0.5 + da, om, "fastpm")
        g = C.step_factors(0.5, 0.5 + da, om, "plain")
        rel[da] = {k: abs(f[k].item() / g[k].item() - 1.0) for k in ("K1", "K2", "dtau")}
    for k in ("K1", "K2"):
        assert rel[0.01][k] < 0.1 * 0.01
        assert 1.8 < rel[0.02][k] / rel[0.01][k] < 2.2
    assert rel[0.01]["dtau"] < 0.01 ** 2
    assert 3.6 < rel[0.02]["dtau"] / rel[0.01]["dtau"] < 4.4


def test_factors_differentiable_in_omega_m():
    om = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    f = C.step_factors(0.2, 0.25, om)
    (g,) = torch.autograd.grad(f["dtau"], om)
    h = 1e-6
    fd = (C.step_factors(0.2, 0.25, 0.3 + h)["dtau"] - C.step_factors(0.2, 0.25, 0.3 - h)["dtau"]).item() / (2 * h)
    assert abs(g.item() / fd - 1.0) < 1e-6
