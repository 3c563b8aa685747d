"""Particle-mesh gravity, kicks and drift (oracle, float64, torch CPU).

Sec. 2.2: dark matter is sampled by N-body particles obeying dx/dt = u/a, d(au)/dt = g
(Eq. dm_hamil), with g = -grad(phi) from a particle-mesh Poisson solve (FastPM). With
p = a u = a^2 dx/dt and the drift time d tau = dt/a^2 this is dx/dtau = p, dp/dt = g.
The gas feels the same field through the source S_g = (0, rho g, a rho U.g) of Eq.
conservation; in (rho, m = rho p, eps) and over a kick of length K = int g dt at frozen
rho and g this integrates exactly to

    m   <- m + rho g K,
    eps <- eps + K m.g + K^2 rho |g|^2 / 2          (eps - |m|^2/(2 rho) is unchanged).

Mesh: node j sits at x = j dx and coincides with gas cell j. Particles are stored in
Lagrangian order (index = (qz N + qy) N + qx) as displacements s from their lattice site
q = (qx, qy, qz) dx, so x = q + s (periodic). Cloud-in-cell weights per axis from
t = s/dx: i = q + floor(t), f = t - floor(t), weights (1 - f, f) on nodes (i, i + 1) mod N.
With ``index_fp32=True`` the cell decision floor(t) is taken on t computed in float32
(t32 = fl32(s32 * fl32(N/L))), the precision of the GPU kernels, so both sides pick the
same cells; the weights stay float64.

Poisson (in these units, H0 = 1): del^2 phi = (3 Om / 2a) delta_tot, delta_tot = rho_dm +
rho_gas - 1 (densities in units of the mean total matter density). Spectrally
g_k = i k (3 Om / 2a) delta_k / k^2, k = 0 removed, and the gradient factor k_j set to 0 at
the Nyquist index of axis j.
"""
from __future__ import annotations

import numpy as np
import torch

_DT = torch.float64


def lattice(n: int):
    """Integer lattice coordinates (qx, qy, qz) of particles 0..n^3-1, Lagrangian order."""
    idx = torch.arange(n ** 3, dtype=torch.int64)
    return torch.stack([idx % n, (idx // n) % n, idx // (n * n)])


def cic_cells(s, n: int, box: float, index_fp32: bool = False):
    """Base node index (3, np) int64 and fractions (3, np) float64 of each particle."""
    q = lattice(n)
    t = s / (box / n)
    if index_fp32:
        inv_dx = np.float32(n / box)
        t32 = s.detach().cpu().numpy().astype(np.float32) * inv_dx  # one fp32 multiply
        fl = torch.from_numpy(np.floor(t32).astype(np.int64))
    else:
        fl = torch.floor(t.detach()).to(torch.int64)
    f = t - fl.to(_DT)
    return q + fl, f


def _corners(base, f, n):
    """Yield (flat node index, weight) for the 8 CIC corners."""
    for oz in (0, 1):
        wz = f[2] if oz else 1.0 - f[2]
        iz = (base[2] + oz) % n
        for oy in (0, 1):
            wy = f[1] if oy else 1.0 - f[1]
            iy = (base[1] + oy) % n
            for ox in (0, 1):
                wx = f[0] if ox else 1.0 - f[0]
                ix = (base[0] + ox) % n
                yield (iz * n + iy) * n + ix, wx * wy * wz


def deposit(s, values, n: int, box: float, index_fp32: bool = False):
    """CIC scatter of per-particle values onto the n^3 mesh: returns [n, n, n]."""
    base, f = cic_cells(s, n, box, index_fp32)
    out = torch.zeros(n ** 3, dtype=_DT)
    for idx, w in _corners(base, f, n):
        out = out.index_add(0, idx, w * values)
    return out.reshape(n, n, n)


def interp(grid, s, n: int, box: float, index_fp32: bool = False):
    """CIC readout of a mesh field [..., n, n, n] at particle positions: [..., np]."""
    base, f = cic_cells(s, n, box, index_fp32)
    flat = grid.reshape(*grid.shape[:-3], n ** 3)
    out = 0.0
    for idx, w in _corners(base, f, n):
        out = out + w * flat[..., idx]
    return out


def wavenumbers(n: int, box: float):
    """k_x (rfft axis), k_y, k_z broadcastable to the half-complex shape [n, n, n//2+1],
    plus the gradient factors with the Nyquist index zeroed."""
    kf = 2.0 * np.pi / box
    full = np.fft.fftfreq(n, d=1.0 / n)          # 0..n/2-1, -n/2..-1
    half = np.arange(n // 2 + 1, dtype=np.float64)
    kz = torch.tensor(full * kf, dtype=_DT).reshape(n, 1, 1)
    ky = torch.tensor(full * kf, dtype=_DT).reshape(1, n, 1)
    kx = torch.tensor(half * kf, dtype=_DT).reshape(1, 1, n // 2 + 1)
    grad = []
    for k, idx in ((kx, half), (ky, full), (kz, full)):
        kg = k.clone()
        if n % 2 == 0:
            nyq = torch.tensor(np.abs(idx) == n // 2).reshape(k.shape)
            kg = torch.where(nyq, torch.zeros_like(kg), kg)
        grad.append(kg)
    return (kx, ky, kz), grad


def gravity(delta, pref, box: float):
    """g = -grad(phi), del^2 phi = pref * delta; returns [3, n, n, n] (x, y, z)."""
    n = delta.shape[-1]
    (kx, ky, kz), (gx, gy, gz) = wavenumbers(n, box)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2safe = torch.where(k2 > 0, k2, torch.ones_like(k2))
    G = torch.where(k2 > 0, 1.0 / k2safe, torch.zeros_like(k2))
    dk = torch.fft.rfftn(delta, dim=(-3, -2, -1))
    out = []
    for kj in (gx, gy, gz):
        gk = (1j * kj * G) * dk * pref
        out.append(torch.fft.irfftn(gk, s=(n, n, n), dim=(-3, -2, -1)))
    return torch.stack(out)


def density_contrast(s, rho_gas, f_b, n: int, box: float, index_fp32: bool = False):
    """delta_tot = (1 - f_b) * (CIC particle count per node) + rho_gas - 1."""
    count = deposit(s, torch.ones(s.shape[1], dtype=_DT), n, box, index_fp32)
    return (1.0 - f_b) * count + rho_gas - 1.0


def gas_kick(U, g, K):
    """Exact kick of the gas by a frozen field over K = int g dt."""
    rho, m, eps = U[0], U[1:4], U[4]
    m_new = m + rho * g * K
    eps_new = eps + K * (m * g).sum(0) + 0.5 * K * K * rho * (g * g).sum(0)
    return torch.cat([rho[None], m_new, eps_new[None]])


def particle_kick(p, s, g, K, box: float, index_fp32: bool = False):
    n = g.shape[-1]
    return p + K * interp(g, s, n, box, index_fp32)


def drift(s, p, dtau):
    return s + dtau * p
