"""Pins of the oracle's relaxing TVD hydro (Sec. 2.3.1-2.3.4).

* Sod shock tube against the exact Riemann solution (textbook two-rarefaction/shock solver,
  Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4): L1 error falls
  with resolution and the shock sits within 2 cells of the exact position.
* Exact conservation of mass, momentum and energy per sweep in a periodic box.
* A uniform state, at rest or moving, is reproduced exactly.
* Sedov-Taylor blast: shock radius phi_0 (E_0 t^2 / rho_1)^(1/5), phi_0 = 1.15 (Eq. sedov),
  front within 2 cells and angular scatter below 1 cell (the paper's own result, Sec. 2.3.4).
"""
import math

import numpy as np
import pytest
import torch

from oracle import hydro

DT = torch.float64


# ---------------------------------------------------------------- exact Riemann solver
def _exact_riemann(WL, WR, gamma, xi):
    """Exact solution (rho, u, p) of the 1-D Riemann problem at similarity coords xi=x/t."""
    rl, ul, pl = WL
    rr, ur, pr = WR
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)

    def fK(p, rK, pK, cK):
        if p > pK:  # shock
            A, B = 2 / ((gamma + 1) * rK), (gamma - 1) / (gamma + 1) * pK
            return (p - pK) * math.sqrt(A / (p + B))
        return 2 * cK / (gamma - 1) * ((p / pK) ** ((gamma - 1) / (2 * gamma)) - 1)

    f = lambda p: fK(p, rl, pl, cl) + fK(p, rr, pr, cr) + ur - ul
    lo, hi = 1e-12, 10 * max(pl, pr)
    for _ in range(200):  # bisection: f is monotone increasing in p
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
    ps = 0.5 * (lo + hi)
    us = 0.5 * (ul + ur) + 0.5 * (fK(ps, rr, pr, cr) - fK(ps, rl, pl, cl))
    g1 = (gamma - 1) / (gamma + 1)
    out = np.zeros((3, len(xi)))
    for i, s in enumerate(xi):
        if s < us:  # left of contact
            if ps > pl:
                SL = ul - cl * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
                W = (rl, ul, pl) if s < SL else (rl * (ps / pl + g1) / (g1 * ps / pl + 1), us, ps)
            else:
                csl = cl * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                if s < ul - cl:
                    W = (rl, ul, pl)
                elif s > us - csl:
                    W = (rl * (ps / pl) ** (1 / gamma), us, ps)
                else:
                    r = rl * (2 / (gamma + 1) + g1 / cl * (ul - s)) ** (2 / (gamma - 1))
                    u = 2 / (gamma + 1) * (cl + (gamma - 1) / 2 * ul + s)
                    W = (r, u, pl * (r / rl) ** gamma)
        else:
            if ps > pr:
                SR = ur + cr * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
                W = (rr, ur, pr) if s > SR else (rr * (ps / pr + g1) / (g1 * ps / pr + 1), us, ps)
            else:
                csr = cr * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                if s > ur + cr:
                    W = (rr, ur, pr)
                elif s < us + csr:
                    W = (rr * (ps / pr) ** (1 / gamma), us, ps)
                else:
                    r = rr * (2 / (gamma + 1) - g1 / cr * (ur - s)) ** (2 / (gamma - 1))
                    u = 2 / (gamma + 1) * (-cr + (gamma - 1) / 2 * ur + s)
                    W = (r, u, pr * (r / rr) ** gamma)
        out[:, i] = W
    return out, ps, us


def _to_U(rho, u, p, gamma):
    n = len(rho)
    U = np.zeros((5, 1, 1, n))
    U[0, 0, 0] = rho
    U[1, 0, 0] = rho * u
    U[4, 0, 0] = p / (gamma - 1) + 0.5 * rho * u * u
    return torch.tensor(U, dtype=DT)


def _sod(n, t_end=0.2, gamma=1.4):
    """Sod on a periodic domain of length 2: left state on [0,1), right on [1,2). The
    mirrored problem at x = 0 = 2 stays outside the window [0.6, 1.5] until t = 0.2."""
    L = 2.0
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    left = x < 1.0
    U = _to_U(np.where(left, 1.0, 0.125), np.zeros(n), np.where(left, 1.0, 0.1), gamma)
    nsteps = int(math.ceil(t_end / (0.3 * dx / 2.2)))
    nu = (t_end / nsteps) / dx
    for _ in range(nsteps):
        U = hydro.sweep(U, "x", nu, gamma)
    return x, U[0, 0, 0].numpy()


def test_sod_against_exact_riemann_solution():
    gamma = 1.4
    errs = {}
    for n in (200, 400, 800):
        x, rho = _sod(n)
        win = (x > 0.6) & (x < 1.5)
        ex, ps, us = _exact_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), gamma, (x[win] - 1.0) / 0.2)
        errs[n] = np.abs(rho[win] - ex[0]).sum() * (2.0 / n)
        if n == 800:
            # shock position: exact right-shock speed (Toro eq. 4.59) and post-shock density
            cr = math.sqrt(gamma * 0.1 / 0.125)
            S = cr * math.sqrt((gamma + 1) / (2 * gamma) * ps / 0.1 + (gamma - 1) / (2 * gamma))
            g1 = (gamma - 1) / (gamma + 1)
            r2 = 0.125 * (ps / 0.1 + g1) / (g1 * ps / 0.1 + 1)
            xs_exact = 1.0 + S * 0.2
            half = 0.5 * (0.125 + r2)
            xr = x[win]
            i = np.where((rho[win][:-1] > half) & (rho[win][1:] <= half))[0][-1]
            xs = xr[i] + (rho[win][i] - half) / (rho[win][i] - rho[win][i + 1]) * (xr[i + 1] - xr[i])
            assert abs(xs - xs_exact) < 2 * (2.0 / n)
            assert abs(ps - 0.30313) < 1e-4 and abs(us - 0.92745) < 1e-4  # Toro table 4.2 test 1
    assert errs[400] < errs[200] and errs[800] < errs[400]
    assert errs[800] < 0.01


def _random_state(shape, seed):
    g = torch.Generator().manual_seed(seed)
    n = shape
    rho = 1.0 + 0.3 * torch.rand(n, generator=g, dtype=DT)
    m = 0.3 * (torch.rand((3,) + n, generator=g, dtype=DT) - 0.5)
    P = 0.5 + 0.3 * torch.rand(n, generator=g, dtype=DT)
    eps = P / (5 / 3 - 1) + (m * m).sum(0) / (2 * rho)
    return torch.cat([rho[None], m, eps[None]])


@pytest.mark.parametrize("d", ["x", "y", "z"])
def test_sweep_conserves_totals(d):
    U = _random_state((6, 7, 8), 1)
    V = hydro.sweep(U, d, 0.2, 5 / 3)
    tot0, tot1 = U.sum((1, 2, 3)), V.sum((1, 2, 3))
    assert torch.allclose(tot0, tot1, rtol=0, atol=1e-12 * U.abs().sum().item())
    assert (V - U).abs().max() > 1e-3  # it did something


def test_uniform_states_are_fixed_points():
    for vel in ((0, 0, 0), (0.3, -0.2, 0.1)):
        U = torch.zeros(5, 4, 5, 6, dtype=DT)
        U[0] = 1.3
        for k in range(3):
            U[1 + k] = 1.3 * vel[k]
        U[4] = 0.7 + 0.5 * 1.3 * sum(v * v for v in vel)
        V = hydro.hydro_step(U, 1, 0.3, 5 / 3)
        assert torch.equal(V, U) or (V - U).abs().max() < 1e-15


def test_strang_cycle_matches_paper_string():
    # "XYZZYX, ZXYYXZ, YZXXZY": each group of six letters is a step and its reverse
    s = "".join(hydro.ORDERS).upper()
    assert s == "XYZZYXZXYYXZYZXXZY"


@pytest.mark.slow
def test_sedov_taylor_blast():
    gamma, n = 5.0 / 3.0, 64
    rho1, E0, p_bg = 1.0, 1.0e4, 1e-6
    U = torch.zeros(5, n, n, n, dtype=DT)
    U[0] = rho1
    U[4] = p_bg / (gamma - 1)
    c = n // 2
    U[4, c, c, c] += E0                      # energy in the central cell (dx = 1)
    r_target = 12.0
    t_end = math.sqrt((r_target / 1.15) ** 5 * rho1 / E0)
    t, step = 0.0, 0
    while t < t_end - 1e-12:
        vmax = hydro.signal_speed_max(U, gamma)
        dt = min(0.3 / vmax, t_end - t)
        U = hydro.hydro_step(U, step, dt, gamma)
        t += dt
        step += 1
    # shock radius along 48 random directions: radius of the density maximum
    from scipy.ndimage import map_coordinates
    rng = np.random.default_rng(0)
    dirs = rng.normal(size=(48, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = np.arange(2.0, 20.0, 0.05)
    rho = U[0].numpy()
    radii = []
    for d in dirs:
        pts = c + d[:, None] * r[None, :]
        prof = map_coordinates(rho, pts, order=1)
        radii.append(r[np.argmax(prof)])
    radii = np.array(radii)
    r_exact = 1.15 * (E0 * t_end ** 2 / rho1) ** 0.2
    assert abs(radii.mean() - r_exact) < 2.0
    assert radii.std() < 1.0
    # mass and energy conserved by the whole run
    assert abs(U[0].sum().item() - rho1 * n ** 3) < 1e-8 * n ** 3
    assert abs(U[4].sum().item() - (E0 + p_bg / (gamma - 1) * n ** 3)) < 1e-8 * E0
