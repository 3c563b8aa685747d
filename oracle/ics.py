"""Initial conditions: Gaussian realisation and Zel'dovich displacement (oracle, float64).

Sec. 2.1: a Gaussian realisation of the linear density field is displaced with Lagrangian
perturbation theory to the starting redshift; DM and gas start from the same linear field.
The paper's Eisenstein-Hu spectrum is replaced by the synthetic shape

    P(k) = A k^-2 exp(-(k / k_c)^2),   k_c = kc_frac * k_Nyquist,  k_Nyquist = pi N / L,

normalised on the grid: the expected cell rms of the linear contrast at a_start is
rms_ref (sigma8 / sigma8_ref) D(a_start; Om) / D(a_ref; Om_ref).

With white noise w (N(0, 1) per cell) and numpy's FFT conventions:
    delta_i = ifft( C sqrt(P(k)) fft(w) ),   C = rms * sqrt(N^3 / sum_{k != 0} P(k)),
so E[delta_i^2] = rms^2. Zel'dovich (1LPT): psi_k = i k delta_k / k^2 (so -div psi = delta_i),
gradient factor zeroed at the Nyquist index. DM: s = psi, p = (g_p(a_i) / D(a_i)) psi.
Gas on the same lattice: rho = f_b (1 + delta_i), m = rho p, eps = a_i^2 rho e_init +
|m|^2 / (2 rho) with e_init = T_init / t_per_e.
"""
from __future__ import annotations

import numpy as np
import torch

from . import cosmology as cosmo
from .pm import wavenumbers
from .subgrid import t_per_e

_DT = torch.float64


def spectrum_shape(n: int, box: float, kc_frac: float):
    """sqrt of P(k)/A on the half-complex grid, and sum over the FULL grid of P(k)/A."""
    (kx, ky, kz), _ = wavenumbers(n, box)
    k = torch.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    kc = kc_frac * np.pi * n / box
    ksafe = torch.where(k > 0, k, torch.ones_like(k))
    P = torch.where(k > 0, ksafe ** -2 * torch.exp(-(ksafe / kc) ** 2), torch.zeros_like(k))
    # full-grid sum: interior kx planes appear twice (k and -k)
    w = torch.full((n // 2 + 1,), 2.0, dtype=_DT)
    w[0] = 1.0
    if n % 2 == 0:
        w[-1] = 1.0
    total = (P * w.reshape(1, 1, -1)).sum()
    return torch.sqrt(P), total


def rms_target(prm):
    return (prm["rms_ref"] * prm["sigma8"] / prm["sigma8_ref"]
            * cosmo.growth_D(prm["a_start"], prm["omega_m"])
            / cosmo.growth_D(prm["a_ref"], prm["omega_m_ref"]))


def linear_field(noise, prm):
    """delta_i and psi (3, n, n, n) from white noise [n, n, n]."""
    n, box = prm["n"], prm["box"]
    sqrtP, total = spectrum_shape(n, box, prm["kc_frac"])
    C = rms_target(prm) * torch.sqrt(n ** 3 / total)
    dk = torch.fft.rfftn(noise, dim=(-3, -2, -1)) * (C * sqrtP)
    delta = torch.fft.irfftn(dk, s=(n, n, n), dim=(-3, -2, -1))
    (kx, ky, kz), grads = wavenumbers(n, box)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2safe = torch.where(k2 > 0, k2, torch.ones_like(k2))
    invk2 = torch.where(k2 > 0, 1.0 / k2safe, torch.zeros_like(k2))
    psi = torch.stack([torch.fft.irfftn(1j * kj * invk2 * dk, s=(n, n, n), dim=(-3, -2, -1))
                       for kj in grads])
    return delta, psi


def initial_conditions(noise, prm):
    """Returns s (3, n^3), p (3, n^3), U (5, n, n, n) at a_start."""
    n = prm["n"]
    om, a0 = prm["omega_m"], prm["a_start"]
    f_b = prm["omega_b"] / om
    delta, psi = linear_field(noise, prm)
    s = psi.reshape(3, n ** 3)
    p = (cosmo.g_p(a0, om) / cosmo.growth_D(a0, om)) * s
    rho = f_b * (1.0 + delta)
    m = rho[None] * p.reshape(3, n, n, n)
    e0 = prm["T_init"] / t_per_e(prm["gamma"], prm["mu"])
    eps = a0 * a0 * rho * e0 + (m * m).sum(0) / (2.0 * rho)
    U = torch.cat([rho[None], m, eps[None]])
    return s, p, U
