"""Pins of the oracle's full step (DM + gas + subgrid) and of its spectra and gradients.

* Uniform universe: nothing moves and the specific internal energy falls exactly as a^-2
  (adiabatic expansion at gamma = 5/3: the energy-equation source vanishes, Eq. ev).
* Exact conservation over a run: gas mass, and total (DM + gas) momentum.
* A single small mode grows like D(a) in DM and gas alike (linear theory, Sec. 2.2).
* Subgrid trend (Sec. 2.4.1): a higher density threshold gives fewer star-formation events.
* Power spectrum: Parseval, a single mode lands in one bin with its amplitude, r_c = +-1.
* Gradients: reverse mode through whole runs equals central finite differences.
"""
import math

import numpy as np
import pytest
import torch

from oracle import cosmology as C
from oracle import pm, sim, spectra
from oracle.subgrid import t_per_e

DT = torch.float64


def test_uniform_universe_adiabatic_cooling():
    prm = sim.Params(n=8, box=8.0, n_steps=6, a_start=0.1, a_end=0.7).as_dict()
    st = sim.run(torch.zeros(8, 8, 8, dtype=DT), prm)
    U = st["U"]
    assert st["s"].abs().max() == 0 and st["p"].abs().max() == 0
    a = prm["a_end"]
    e = (U[4] - (U[1:4] ** 2).sum(0) / (2 * U[0])) / (a * a * U[0])
    e0 = prm["T_init"] / t_per_e(prm["gamma"], prm["mu"])
    assert torch.allclose(e * a * a, torch.full_like(e, e0 * prm["a_start"] ** 2), rtol=1e-12)


def test_run_conserves_gas_mass_and_total_momentum():
    prm = sim.Params(n=16, box=16.0, n_steps=8, a_start=0.1, a_end=0.6, rms_ref=0.2,
                     subgrid_on=1, T0_uv=1e4).as_dict()
    noise = sim.noise_field(prm)
    st0 = sim.init_state(noise, prm)
    st = sim.run(noise, prm)
    fb = sim.f_baryon(prm)
    mom = lambda s: (1 - fb) * s["p"].sum(1) + s["U"][1:4].sum((1, 2, 3))
    assert abs(st["U"][0].sum() - st0["U"][0].sum()) < 1e-12 * st0["U"][0].sum()
    scale = (1 - fb) * st["p"].abs().sum() + st["U"][1:4].abs().sum()
    assert (mom(st) - mom(st0)).abs().max() < 1e-12 * scale


@pytest.mark.slow
def test_single_mode_linear_growth():
    n, box = 32, 32.0
    prm = sim.Params(n=n, box=box, n_steps=16, a_start=0.1, a_end=0.5, T_init=100.0).as_dict()
    z, y, x = torch.meshgrid(*(torch.arange(n, dtype=DT),) * 3, indexing="ij")
    # white noise whose shaped field is one Fourier mode along x (k = 2 pi / L)
    noise = 0.011 * torch.cos(2 * math.pi * x / n)   # delta ~ 0.01 at a_start, ~0.05 at a_end
    st0 = sim.init_state(noise, prm)
    st = sim.run(noise, prm)

    def amp(field):
        return torch.fft.rfftn(field)[0, 0, 1].abs().item()

    fb = sim.f_baryon(prm)
    g0 = amp(st0["U"][0] / fb - 1)
    g1 = amp(st["U"][0] / fb - 1)
    dm1 = amp(pm.deposit(st["s"], torch.ones(n ** 3, dtype=DT), n, box) - 1)
    growth = (C.growth_D(prm["a_end"], 0.3) / C.growth_D(prm["a_start"], 0.3)).item()
    assert abs(g1 / g0 / growth - 1) < 0.02
    assert abs(g1 / dm1 - 1) < 0.03


def test_higher_threshold_fewer_events():
    base = dict(n=16, box=16.0, n_steps=6, a_start=0.2, a_end=0.8, rms_ref=0.3,
                subgrid_on=1, Pi0=0.3, T_c=1e6, w_T=5e4)
    counts = []
    for dc in (0.0, 0.5, 2.0):
        prm = sim.Params(**base, delta_c=dc, w_delta=0.05 * max(dc, 0.2)).as_dict()
        st = sim.run(sim.noise_field(prm), prm)
        counts.append(sum(int(e.sum()) for e in st["events"]))
    assert counts[0] > counts[1] > counts[2]


def test_power_spectrum_parseval_and_single_mode():
    n, box = 16, 10.0
    f = torch.randn(n, n, n, dtype=DT, generator=torch.Generator().manual_seed(0))
    f -= f.mean()
    k, P, nm = spectra.power_spectrum(f, box, nbins=n)
    # sum_k |f_k|^2 = N^3 sum_x f^2 ; P = L^3 |f_k|^2 / N^6
    total = (P * nm).sum().item() * n ** 6 / box ** 3
    assert abs(total / (n ** 3 * (f ** 2).sum().item()) - 1) < 1e-12
    z, y, x = torch.meshgrid(*(torch.arange(n, dtype=DT),) * 3, indexing="ij")
    g = 0.7 * torch.cos(2 * math.pi * (2 * x + y) / n)
    k, P, nm = spectra.power_spectrum(g, box, nbins=n)
    b = round(math.sqrt(5))  # |k| / k_f = sqrt(2^2 + 1^2)
    nz = torch.nonzero(P > 1e-20).flatten().tolist()
    assert nz == [b - 1]
    # two modes (+-k) of |g_k| = 0.35 N^3 each among nm[b-1] modes in the bin
    expect = 2 * (0.35 * n ** 3) ** 2 * box ** 3 / n ** 6 / nm[b - 1].item()
    assert abs(P[b - 1].item() / expect - 1) < 1e-12
    r = spectra.cross_correlation(f, f, box)
    assert torch.allclose(r[nm > 0], torch.ones_like(r[nm > 0]), atol=1e-12)
    r = spectra.cross_correlation(f, -f, box)
    assert torch.allclose(r[nm > 0], -torch.ones_like(r[nm > 0]), atol=1e-12)


def _fd_check(fun, x, direction, h):
    """Reverse-mode derivative along `direction` and the central difference closest to it
    over steps h, h/10, h/100. The scheme has kinks (limiter gate, CIC cell edges, |v|,
    the UV-floor max) and a large step can straddle one; a small step cannot, in practice."""
    x = x.detach().clone().requires_grad_(True)
    val = fun(x)
    (g,) = torch.autograd.grad(val, x)
    ad = (g * direction).sum().item()
    best = None
    for hh in (h, h / 10, h / 100):
        fd = (fun(x.detach() + hh * direction) - fun(x.detach() - hh * direction)).item() / (2 * hh)
        if best is None or abs(fd - ad) < abs(best - ad):
            best = fd
    return ad, best


def test_gradient_wrt_initial_noise_matches_finite_differences():
    prm = sim.Params(n=8, box=8.0, n_steps=4, a_start=0.1, a_end=0.3, rms_ref=0.15,
                     subgrid_on=1, delta_c=0.2, w_delta=0.1, T_c=1e6, w_T=1e5, Pi0=0.2,
                     T0_uv=5e3).as_dict()
    noise = sim.noise_field(prm)
    target = sim.run(sim.noise_field(dict(prm, seed=2)), prm)["U"][0].detach()
    fun = lambda w: sim.mse_density(sim.run(w, prm)["U"], target)
    d = torch.randn(noise.shape, dtype=DT, generator=torch.Generator().manual_seed(3))
    ad, fd = _fd_check(fun, noise, d, 1e-5)
    assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-14


@pytest.mark.parametrize("name", ["omega_m", "sigma8", "delta_c", "Pi0", "E0", "T0_uv", "gamma_uv"])
def test_gradient_wrt_parameters_matches_finite_differences(name):
    base = dict(n=8, box=8.0, n_steps=4, a_start=0.1, a_end=0.3, rms_ref=0.15, subgrid_on=1,
                delta_c=0.2, w_delta=0.1, T_c=1e6, w_T=1e5, Pi0=0.2, T0_uv=5e3)
    prm = sim.Params(**base).as_dict()
    noise = sim.noise_field(prm)
    target = sim.run(sim.noise_field(dict(prm, seed=2)), prm)["U"][0].detach()

    def fun(v):
        q = dict(prm)
        q[name] = v
        st = sim.run(noise, q)
        return sim.mse_density(st["U"], target) + 1e-3 * st["U"][4].mean()

    x0 = torch.tensor(float(prm[name]), dtype=DT)
    ad, fd = _fd_check(fun, x0, torch.tensor(1.0, dtype=DT), 1e-6 * max(abs(x0.item()), 1e-2))
    assert abs(ad - fd) <= 1e-5 * abs(fd) + 1e-12


def test_fli_posterior_is_the_wiener_filter_for_a_linear_forward():
    """With gravity, hydro and subgrid off and no steps, the final gas density is the
    initial rho = f_b (1 + delta_L(s)), linear in s: delta_k = A_k s_k with A_k = C sqrt(P_k)
    per Fourier mode. The posterior 1/2 [|d - rho|^2 / sigma^2 + |s|^2] is then a quadratic
    whose minimiser is the Wiener filter s_k = f_b A_k d'_k / (sigma^2 + f_b^2 A_k^2),
    d' = d - f_b, and whose gradient is s - f_b A (d' - f_b A s) / sigma^2 (the test's own
    FFTs); the oracle's reverse-mode gradient must equal it and vanish at the minimiser."""
    n, box, sig = 8, 8.0, 0.02
    prm = sim.Params(n=n, box=box, n_steps=1, gravity_on=0, hydro_on=0, subgrid_on=0,
                     rms_ref=0.2).as_dict()
    fb = prm["omega_b"] / prm["omega_m"]
    g = np.random.default_rng(9)
    # A_k from the response to one mode at a time is avoided: A is diagonal in Fourier
    # space, so its multiplier is the transfer of an impulse
    imp = torch.zeros(n, n, n, dtype=DT)
    imp[0, 0, 0] = 1.0
    d_imp = sim.run(imp, prm, n_steps=0)["U"][0] / fb - 1.0       # delta_L of an impulse
    A = np.fft.fftn(d_imp.numpy()).real                           # real, even multiplier
    assert np.abs(np.fft.fftn(d_imp.numpy()).imag).max() < 1e-14
    d = fb * (1 + 0.3 * g.normal(size=(n, n, n)))
    dp = np.fft.fftn(d - fb)
    s_star = np.fft.ifftn(fb * A * dp / (sig ** 2 + fb ** 2 * A ** 2)).real
    Ls, gs = sim.fli_value_and_grad(torch.tensor(s_star), torch.tensor(d), sig, prm, n_steps=0)
    assert np.abs(gs.numpy()).max() < 1e-9 * np.abs(s_star).max() / sig ** 2
    s1 = g.normal(size=(n, n, n))
    L1, g1 = sim.fli_value_and_grad(torch.tensor(s1), torch.tensor(d), sig, prm, n_steps=0)
    As1 = np.fft.ifftn(A * np.fft.fftn(s1)).real
    want = s1 - np.fft.ifftn(fb * A * np.fft.fftn(d - fb - fb * As1)).real / sig ** 2
    assert np.allclose(g1.numpy(), want, rtol=1e-10, atol=1e-10 * np.abs(want).max())
    L1_want = 0.5 * (((d - fb - fb * As1) ** 2).sum() / sig ** 2 + (s1 ** 2).sum())
    assert abs(L1.item() / L1_want - 1) < 1e-12
    assert L1.item() > Ls.item()


def test_thermal_observable_is_internal_energy_density():
    """eps - |m|^2/(2 rho) = a^2 rho e: for a uniform gas at T it is a^2 f_b T / t_per_e,
    with any bulk velocity (the kinetic part is removed)."""
    n, a = 4, 0.3
    prm = sim.Params(n=n, box=4.0, a_start=a, T_init=2e4).as_dict()
    s, p, U = sim.ics.initial_conditions(torch.zeros(n, n, n, dtype=DT), prm)
    fb = prm["omega_b"] / prm["omega_m"]
    want = a * a * fb * 2e4 / t_per_e(prm["gamma"], prm["mu"])
    assert torch.allclose(sim.observable(U, "thermal"), torch.full((n, n, n), want, dtype=DT),
                          rtol=1e-12)
    U2 = U.clone()
    U2[1] = 0.3 * U2[0]
    U2[4] = U2[4] + 0.5 * U2[1] ** 2 / U2[0]
    assert torch.allclose(sim.observable(U2, "thermal"), sim.observable(U, "thermal"), rtol=1e-12)
