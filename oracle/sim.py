"""One time step and a run of the coupled DM + gas + subgrid system (oracle, float64).

Step n takes the state from a_n to a_{n+1} (uniform in a; a_h the midpoint). The paper
fixes the ingredients (Sec. 2.2 FastPM kick-drift-kick for the dark matter, Sec. 2.3.2
Strang-split relaxing TVD sweeps for the gas, Sec. 2.4 subgrid model) but not their
interleaving; the reading used here applies the same kick-drift-kick to DM and gas:

  1. half kick of DM momenta and gas (m, eps) with g(a_n)         K1 (force at a_n)
  2. drift of DM positions                                        dtau (momentum at a_h)
  3. three hydro sweeps of length dtau in the order ORDERS[n % 6]
  4. subgrid star formation at a_{n+1} with Philox draws of step n
  5. CIC deposit of DM + gas density, spectral Poisson solve -> g(a_{n+1})
  6. half kick of DM and gas with g(a_{n+1})                      K2 (force at a_{n+1})

Diagnostics that do not feed back (Sec. 2.4.1): the star mesh accumulates zhat, and the
dark-matter auxiliary field accumulates the CIC readout of each step's zhat at the drifted
particle positions.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict, field
import math

import numpy as np
import torch

from . import cosmology as cosmo
from . import hydro, pm, ics, philox
from .subgrid import subgrid as subgrid_update

_DT = torch.float64


@dataclass
class Params:
    n: int = 32
    box: float = 32.0                 # Mpc/h
    omega_m: float = 0.3
    omega_b: float = 0.049
    h: float = 0.7                    # does not enter: lengths in Mpc/h, velocities 100 km/s
    sigma8: float = 0.8
    gamma: float = 5.0 / 3.0
    mu: float = 0.6
    T_init: float = 1.0e4             # K
    a_start: float = 0.1
    a_end: float = 0.5
    n_steps: int = 20
    ckpt_every: int = 6
    subgrid_on: int = 0
    delta_c: float = 100.0
    Pi0: float = 0.05
    E0: float = 0.03                  # (100 km/s)^2
    T_c: float = 3.0e4                # K
    w_delta: float = 5.0
    w_T: float = 1500.0
    tau: float = 0.1
    T0_uv: float = 0.0                # K; 0 disables the floor
    gamma_uv: float = 1.4
    seed: int = 1
    kdk_mode: str = "fastpm"
    rms_ref: float = 0.05
    a_ref: float = 0.1
    sigma8_ref: float = 0.8
    omega_m_ref: float = 0.3
    kc_frac: float = 0.5
    limiter_eps: float = 1e-30
    gravity_on: int = 1
    hydro_on: int = 1
    instance: int = 0

    def as_dict(self):
        return asdict(self)


def _as_prm(prm):
    return prm.as_dict() if isinstance(prm, Params) else dict(prm)


def schedule(prm):
    """Per-step dicts (a0, a1, K1, dtau, K2, pref1) as 0-d float64 tensors."""
    a = cosmo.scale_factors(prm["a_start"], prm["a_end"], prm["n_steps"])
    out = []
    for i in range(prm["n_steps"]):
        f = cosmo.step_factors(a[i], a[i + 1], prm["omega_m"], prm["kdk_mode"])
        f["a0"], f["a1"] = a[i], a[i + 1]
        out.append(f)
    return out


def f_baryon(prm):
    return prm["omega_b"] / prm["omega_m"]


def force(s, rho_gas, prm, a):
    n, box = prm["n"], prm["box"]
    if not prm["gravity_on"]:
        return torch.zeros(3, n, n, n, dtype=_DT)
    delta = pm.density_contrast(s, rho_gas, f_baryon(prm), n, box)
    return pm.gravity(delta, cosmo.poisson_prefactor(a, prm["omega_m"]), box)


def subgrid_params(prm):
    return {k: prm[k] for k in ("gamma", "mu", "delta_c", "Pi0", "E0", "T_c", "w_delta",
                                "w_T", "tau", "T0_uv", "gamma_uv")} | {"f_b": f_baryon(prm)}


def init_state(noise, prm):
    prm = _as_prm(prm)
    s, p, U = ics.initial_conditions(noise, prm)
    n = prm["n"]
    return {"s": s, "p": p, "U": U, "g": force(s, U[0], prm, prm["a_start"]), "step": 0,
            "star": torch.zeros(n, n, n, dtype=_DT), "aux": torch.zeros(n ** 3, dtype=_DT),
            "events": []}


def step(state, prm, sched=None):
    """Advance the state by one step (returns a new dict)."""
    prm = _as_prm(prm)
    n, box = prm["n"], prm["box"]
    i = state["step"]
    f = (sched or schedule(prm))[i]
    s, p, U, g = state["s"], state["p"], state["U"], state["g"]
    if prm["gravity_on"]:
        p = pm.particle_kick(p, s, g, f["K1"], box)
        U = pm.gas_kick(U, g, f["K1"])
    s = pm.drift(s, p, f["dtau"])
    if prm["hydro_on"]:
        U = hydro.hydro_step(U, i, f["dtau"] / (box / n), prm["gamma"], prm["limiter_eps"])
    star, aux, events = state["star"], state["aux"], list(state["events"])
    if prm["subgrid_on"]:
        g0, g1 = philox.gumbel_pair(prm["seed"], n ** 3, i, prm["instance"])
        g0 = torch.tensor(g0.reshape(n, n, n), dtype=_DT)
        g1 = torch.tensor(g1.reshape(n, n, n), dtype=_DT)
        U, zhat, ev = subgrid_update(U, f["a1"], subgrid_params(prm), g0, g1)
        star = star + zhat.detach()
        aux = aux + pm.interp(zhat.detach(), s.detach(), n, box)
        events.append(ev)
    g = force(s, U[0], prm, f["a1"])
    if prm["gravity_on"]:
        p = pm.particle_kick(p, s, g, f["K2"], box)
        U = pm.gas_kick(U, g, f["K2"])
    return {"s": s, "p": p, "U": U, "g": g, "step": i + 1, "star": star, "aux": aux,
            "events": events}


def run(noise, prm, n_steps: int | None = None, callback=None):
    prm = _as_prm(prm)
    sched = schedule(prm)
    st = init_state(noise, prm)
    for _ in range(prm["n_steps"] if n_steps is None else n_steps):
        st = step(st, prm, sched)
        if callback is not None:
            callback(st)
    return st


def noise_field(prm):
    """The run's white noise from its Philox seed (tag 0)."""
    prm = _as_prm(prm)
    return torch.tensor(philox.white_noise(prm["seed"], prm["n"], prm["instance"]), dtype=_DT)


def mse_density(U, target):
    """Mean squared difference of the gas density (config-2 loss)."""
    return ((U[0] - target) ** 2).mean()


def observable(U, kind: str = "density"):
    """Observed field of the final gas state (Sec. 3): the density, or ("thermal") the
    internal energy density eps - |m|^2 / (2 rho) = a^2 rho e, proportional to the
    gas-mass-weighted temperature rho T of the delta_b T probe of Sec. 3.2."""
    if kind == "density":
        return U[0]
    if kind == "thermal":
        return U[4] - (U[1:4] ** 2).sum(0) / (2.0 * U[0])
    raise ValueError(kind)


def fli_value_and_grad(noise, data, sigma_noise, prm, n_steps: int | None = None,
                       kind: str = "density"):
    """Posterior of field-level inference (Sec. 3.2) at the amplitudes `noise` and its
    gradient by reverse mode through the whole run (float64)."""
    s = noise.detach().clone().requires_grad_(True)
    U = run(s, prm, n_steps)["U"]
    L = fli_loss(U, data, sigma_noise, s, kind)
    (g,) = torch.autograd.grad(L, s)
    return L.detach(), g


def fli_loss(U, data, sigma_noise, noise, kind: str = "density"):
    """Negative log posterior of field-level inference (Sec. 3.2):
    1/2 sum[(d - F(s))^2 / N + |s|^2], F the observable of the final gas state and s the
    white noise."""
    return 0.5 * (((data - observable(U, kind)) ** 2).sum() / sigma_noise ** 2 +
                  (noise ** 2).sum())
