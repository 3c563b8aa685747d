"""Relaxing TVD sweep for the comoving Euler equations (oracle, float64, torch CPU).

State per cell U = (rho, m_x, m_y, m_z, eps), tensor shape [5, Nz, Ny, Nx] (C order, x
fastest), periodic in every direction.

Comoving variables (Sec. 2.3, Eq. conservation): rho is the comoving gas density,
m = a rho U (U the peculiar velocity), eps = a^2 rho E with E = e + U^2/2. Written in the
drift time d tau = dt / a^2, Eqs. cont / momentum / ev become the plain Euler equations in
(rho, m, eps) with the pressure-like quantity

    P = a^2 p = (gamma - 1) (eps - |m|^2 / (2 rho)),

because the expansion term a adot (2 - 3(gamma - 1)) rho e of the energy equation vanishes
for gamma = 5/3 (the paper's Eq. ev after its simplification). Gravity enters as a
separate source (module ``pm``).

One sweep along direction d (Sec. 2.3.1-2.3.2, following the Trac & Pen relaxing scheme the
paper cites):
  * velocity v = m_d / rho, sound speed c_s = sqrt(gamma P / rho), freezing speed
    c = |v| + c_s per cell;
  * flux F = (m_d, m_x v + P [d == x], m_y v + P [d == y], m_z v + P [d == z], (eps + P) v);
  * right / left moving fluxes F^R = (c U + F) / 2, F^L = (c U - F) / 2, F = F^R - F^L;
  * half step (Eq. TVD_halfstep) with first-order upwind face fluxes
    F_{i+1/2} = F^R_i - F^L_{i+1};
  * full step (Eq. TVD_fullstep) from U^n with second-order face fluxes computed on the
    half-step state: F^R_{i+1/2} = F^R_i + phi((F^R_i - F^R_{i-1})/2, (F^R_{i+1} - F^R_i)/2),
    and its mirror image F^L_{i+1/2} = F^L_{i+1} - phi((F^L_{i+1} - F^L_i)/2,
    (F^L_{i+2} - F^L_{i+1})/2), limited component by component;
  * limiter: the paper's harmonic-mean van Leer form 2ab/(a + b + eps), gated to zero when
    a b <= 0 (standard van Leer; the ungated form is unstable where a ~ -b), with eps
    signed like a + b so the denominator never vanishes.

Conventions at kinks (they fix the reverse-mode gradient): d|v|/dv = 0 at v = 0; c_s = 0 and
its derivative 0 where gamma P / rho <= 0; the gated limiter and its derivative are 0 where
a b <= 0.
"""
from __future__ import annotations

import torch

# tensor dim of each sweep direction and the momentum field carried along it
_AXIS = {"x": (3, 1), "y": (2, 2), "z": (1, 3)}

# Strang permutation cycle: step n uses ORDERS[n % 6] (Sec. 2.3.2: "XYZZYX, ZXYYXZ, YZXXZY")
ORDERS = ("xyz", "zyx", "zxy", "yxz", "yzx", "xzy")

LIMITER_EPS = 1e-30


def pressure(U, gamma):
    rho, m, eps = U[0], U[1:4], U[4]
    return (gamma - 1.0) * (eps - (m * m).sum(0) / (2.0 * rho))


def _sound_speed(P, rho, gamma):
    cs2 = gamma * P / rho
    pos = cs2 > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, cs2, torch.ones_like(cs2))),
                       torch.zeros_like(cs2))


def split_fluxes(U, d: str, gamma: float):
    """Right and left moving fluxes (F^R, F^L) of every cell for a sweep along d."""
    _, f = _AXIS[d]
    rho, eps = U[0], U[4]
    md = U[f]
    v = md / rho
    P = pressure(U, gamma)
    c = torch.abs(v) + _sound_speed(P, rho, gamma)
    F = [md]
    for k in (1, 2, 3):
        F.append(U[k] * v + (P if k == f else 0.0))
    F.append((eps + P) * v)
    F = torch.stack(F)
    cU = c * U
    return 0.5 * (cU + F), 0.5 * (cU - F)


def vanleer(a, b, eps: float = LIMITER_EPS):
    """Gated harmonic-mean limiter 2 max(ab, 0) / (a + b + copysign(eps, a + b))."""
    ab = a * b
    num = torch.where(ab > 0, ab, torch.zeros_like(ab))
    s = a + b
    return 2.0 * num / (s + torch.copysign(torch.full_like(s, eps), s.detach()))


def sweep(U, d: str, nu, gamma: float, eps: float = LIMITER_EPS):
    """One relaxing-TVD sweep along d; nu = dtau / dx (may be a 0-d tensor)."""
    ax, _ = _AXIS[d]

    def nb(x, k):  # x[i + k] at position i (periodic)
        return torch.roll(x, shifts=-k, dims=ax)

    # half step: first-order upwind face fluxes F_{i+1/2} = F^R_i - F^L_{i+1}
    FR, FL = split_fluxes(U, d, gamma)
    Fface = FR - nb(FL, 1)
    Uh = U - 0.5 * nu * (Fface - nb(Fface, -1))
    # full step: second-order limited face fluxes on the half-step state
    FRh, FLh = split_fluxes(Uh, d, gamma)
    FRface = FRh + vanleer(0.5 * (FRh - nb(FRh, -1)), 0.5 * (nb(FRh, 1) - FRh), eps)
    FL1, FL2 = nb(FLh, 1), nb(FLh, 2)
    FLface = FL1 - vanleer(0.5 * (FL1 - FLh), 0.5 * (FL2 - FL1), eps)
    F2 = FRface - FLface
    return U - nu * (F2 - nb(F2, -1))


def hydro_step(U, step_index: int, nu, gamma: float, eps: float = LIMITER_EPS):
    """Three Strang-split sweeps, each with the full step, in the order of the cycle."""
    for d in ORDERS[step_index % 6]:
        U = sweep(U, d, nu, gamma, eps)
    return U


def signal_speed_max(U, gamma: float):
    """max over cells and directions of |v_d| + c_s (Eq. dt: dt <= C_max dx / (|v| + c_s))."""
    rho = U[0]
    P = pressure(U, gamma)
    cs = _sound_speed(P, rho, gamma)
    vmax = torch.stack([torch.abs(U[k] / rho) for k in (1, 2, 3)]).amax(0)
    return float((vmax + cs).max())


def cfl_number(U, dtau, dx, gamma: float):
    """C = max(|v| + c_s) dtau / dx."""
    return signal_speed_max(U, gamma) * float(dtau) / dx
