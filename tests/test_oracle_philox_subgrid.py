"""Pins of the oracle's Philox generator, Gumbel draws and subgrid model (Sec. 2.4)."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import philox, subgrid
from oracle.sim import Params, subgrid_params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(w, 16) for w in line.split()])
    return rows


def test_philox_known_answers():
    for r in _kat():
        out = philox.philox4x32_10([np.uint64(c) for c in r[0:4]], r[4:6])
        assert [int(o) for o in out] == r[6:10]


def test_uniform_exact_in_float32_and_open_interval():
    x = np.array([0, 1, 511, 512, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    u = philox.uniform_from_word(x)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u[0] == 2.0 ** -24 and u[4] == 1.0 - 2.0 ** -24


def test_gumbel_moments():
    # Gumbel(0,1): mean = Euler-Mascheroni constant, variance = pi^2 / 6
    g0, g1 = philox.gumbel_pair(seed=11, n_cells=1 << 20, step=3)
    for g in (g0, g1):
        assert abs(g.mean() - 0.5772156649) < 4 * math.sqrt(math.pi ** 2 / 6 / g.size)
        assert abs(g.var() / (math.pi ** 2 / 6) - 1.0) < 0.01
    assert abs(np.corrcoef(g0, g1)[0, 1]) < 0.005


def test_white_noise_moments():
    w = philox.white_noise(seed=5, n=64)
    assert abs(w.mean()) < 4 / math.sqrt(w.size)
    assert abs(w.var() - 1.0) < 0.01
    assert abs(((w ** 4).mean()) / 3.0 - 1.0) < 0.03


def _cells(n=32, seed=0):
    """Random gas cells spanning the sigmoid transitions (rho near delta_c, T near T_c)."""
    rng = np.random.default_rng(seed)
    prm = subgrid_params(Params().as_dict() | {"T0_uv": 0.0})
    fb = prm["f_b"]
    tpe = subgrid.t_per_e(prm["gamma"], prm["mu"])
    a = 0.5
    rho = fb * (1 + prm["delta_c"] + prm["w_delta"] * rng.normal(size=(n, n, n)) * 3)
    m = rng.normal(size=(3, n, n, n)) * 0.1 * rho
    T = prm["T_c"] + prm["w_T"] * 3 * rng.normal(size=(n, n, n))
    e = T / tpe
    eps = a * a * rho * e + (m * m).sum(0) / (2 * rho)
    U = torch.tensor(np.concatenate([rho[None], m, eps[None]]), dtype=torch.float64)
    return U, prm, a


def test_stable_form_matches_printed_gumbel_softmax():
    U, prm, a = _cells(16)
    g0, g1 = philox.gumbel_pair(3, 16 ** 3, 0)
    g0 = torch.tensor(g0.reshape(U.shape[1:])); g1 = torch.tensor(g1.reshape(U.shape[1:]))
    _, zhat, _ = subgrid.subgrid(U, a, prm, g0, g1)
    # recompute pi_0 directly from its definition and apply the printed Eq. gumbelsoftmax
    tpe = subgrid.t_per_e(prm["gamma"], prm["mu"])
    rho, m, eps = U[0], U[1:4], U[4]
    e = (eps - (m * m).sum(0) / (2 * rho)) / (a * a * rho)
    sig = lambda x: 1 / (1 + torch.exp(-x))
    pi0 = prm["Pi0"] * sig((rho / prm["f_b"] - 1 - prm["delta_c"]) / prm["w_delta"]) \
        * sig((prm["T_c"] - tpe * e) / prm["w_T"])
    lit = subgrid.gumbel_softmax_literal(pi0, g0, g1, prm["tau"])
    ok = torch.isfinite(lit)
    assert ok.float().mean() > 0.9
    assert torch.allclose(zhat[ok], lit[ok], rtol=1e-10, atol=1e-12)


def test_event_frequency_equals_pi0():
    # Gumbel-max: P(ln pi0 + g0 > ln(1-pi0) + g1) = pi0 exactly; binomial test over 2^20 draws
    n = 1 << 20
    for pi0 in (0.02, 0.3, 0.75):
        g0, g1 = philox.gumbel_pair(7, n, step=int(pi0 * 100))
        ev = (math.log(pi0) + g0) > (math.log1p(-pi0) + g1)
        sd = math.sqrt(pi0 * (1 - pi0) / n)
        assert abs(ev.mean() - pi0) < 4.5 * sd


def test_zero_temperature_limit_gives_hard_events():
    U, prm, a = _cells(16, seed=1)
    g0, g1 = philox.gumbel_pair(3, 16 ** 3, 5)
    g0 = torch.tensor(g0.reshape(U.shape[1:])); g1 = torch.tensor(g1.reshape(U.shape[1:]))
    prm = dict(prm, tau=1e-6)
    _, zhat, events = subgrid.subgrid(U, a, prm, g0, g1)
    far = (zhat < 1e-3) | (zhat > 1 - 1e-3)
    assert far.float().mean() > 0.99
    assert torch.equal((zhat[far] > 0.5), events[far])


def test_sharp_threshold_limit():
    # widths -> 0: pi0 -> Pi0 [delta > delta_c][T < T_c]; with tau small the injected energy
    # follows that indicator exactly where the Gumbel margin is not tiny
    U, prm, a = _cells(16, seed=2)
    prm = dict(prm, w_delta=1e-9, w_T=1e-9, Pi0=0.999999, tau=1e-3)
    g = torch.zeros(U.shape[1:], dtype=torch.float64)
    Unew, zhat, _ = subgrid.subgrid(U, a, prm, g, g)
    tpe = subgrid.t_per_e(prm["gamma"], prm["mu"])
    rho, m, eps = U[0], U[1:4], U[4]
    e = (eps - (m * m).sum(0) / (2 * rho)) / (a * a * rho)
    ind = (rho / prm["f_b"] - 1 > prm["delta_c"]) & (tpe * e < prm["T_c"])
    assert torch.equal(zhat > 0.5, ind)
    de = (Unew[4] - U[4]) / (a * a * rho)
    assert torch.allclose(de[ind], torch.full_like(de[ind], prm["E0"]), rtol=1e-6)
    assert torch.all(de[~ind].abs() < 1e-9)


def test_uv_floor_sets_minimum_temperature():
    U, prm, a = _cells(8, seed=3)
    prm = dict(prm, T0_uv=5e4, gamma_uv=1.4, Pi0=1e-12)
    g = torch.zeros(U.shape[1:], dtype=torch.float64)
    Unew, _, _ = subgrid.subgrid(U, a, prm, g, g)
    tpe = subgrid.t_per_e(prm["gamma"], prm["mu"])
    rho, m = Unew[0], Unew[1:4]
    T = tpe * (Unew[4] - (m * m).sum(0) / (2 * rho)) / (a * a * rho)
    Tf = 5e4 * (rho / prm["f_b"]) ** 0.4
    assert torch.all(T >= Tf * (1 - 1e-12))


def test_temperature_conversion_value():
    # T = (gamma-1) mu m_p e / k_B: 1e4 K at mu=0.6, gamma=5/3 is e ~ 0.0206 (100 km/s)^2
    e = 1e4 / subgrid.t_per_e(5 / 3, 0.6)
    assert abs(e - 0.020636) < 2e-6
