"""Pins of the oracle's particle-mesh gravity, kicks and drift (Sec. 2.2).

* Single Fourier mode: g equals the closed-form gradient of the Poisson solution.
* Momentum conservation: sum over the mesh of delta * g vanishes (k <-> -k symmetry).
* CIC deposit: brute-force definition on a tiny grid, mass conservation, node/midpoint cases;
  readout is the transpose of deposit; readout is exact for fields linear within a cell.
* Gas kick: internal energy unchanged and two kicks compose exactly.
* Zel'dovich pancake: a plane wave evolved with the PM and FastPM factors follows
  x = q + D(a) psi(q) before shell crossing.
"""
import itertools
import math

import numpy as np
import pytest
import torch

from oracle import cosmology as C
from oracle import pm

DT = torch.float64


def _grid_x(n, box):
    x = torch.arange(n, dtype=DT) * (box / n)
    return torch.meshgrid(x, x, x, indexing="ij")  # z, y, x


@pytest.mark.parametrize("mode", [(1, 0, 0), (0, 2, 1), (3, -1, 2)])
def test_single_mode_poisson(mode):
    n, box, pref = 16, 20.0, 0.73
    z, y, x = _grid_x(n, box)
    kv = [2 * math.pi / box * m for m in mode]  # (kx, ky, kz)
    phase = kv[0] * x + kv[1] * y + kv[2] * z
    delta = 0.3 * torch.cos(phase)
    g = pm.gravity(delta, pref, box)
    k2 = sum(k * k for k in kv)
    # phi = -pref 0.3 cos / k^2 ; g = -grad phi = -pref 0.3 k sin / k^2
    for j in range(3):
        ref = -pref * 0.3 * kv[j] / k2 * torch.sin(phase)
        assert torch.allclose(g[j], ref, atol=1e-13)


def test_momentum_conservation():
    n, box = 12, 12.0
    delta = torch.randn(n, n, n, dtype=DT, generator=torch.Generator().manual_seed(0))
    delta -= delta.mean()
    g = pm.gravity(delta, 1.0, box)
    tot = (delta[None] * g).sum((1, 2, 3))
    assert tot.abs().max() < 1e-12 * delta.abs().sum()


def _brute_deposit(x_cells, vals, n):
    """Definition of CIC: each particle spreads its value over the 8 nodes around it with
    weights prod_d (1 - |X_d - node_d|), periodic."""
    out = np.zeros((n, n, n))
    for X, v in zip(x_cells, vals):
        base = np.floor(X).astype(int)
        for o in itertools.product((0, 1), repeat=3):
            node = base + np.array(o)
            w = np.prod(1.0 - np.abs(X - node))
            ix, iy, iz = node % n
            out[iz, iy, ix] += w * v
    return out


def test_deposit_matches_brute_force_and_conserves_mass():
    n, box = 6, 9.0
    rng = np.random.default_rng(3)
    s = torch.tensor(rng.uniform(-4, 4, size=(3, n ** 3)), dtype=DT)
    vals = torch.tensor(rng.uniform(0.5, 2, size=n ** 3), dtype=DT)
    got = pm.deposit(s, vals, n, box).numpy()
    q = pm.lattice(n).numpy().astype(float)
    X = (q + s.numpy() / (box / n)).T
    ref = _brute_deposit(X, vals.numpy(), n)
    assert np.allclose(got, ref, atol=1e-13)
    assert abs(got.sum() - vals.sum().item()) < 1e-12


def test_deposit_special_positions():
    n, box = 4, 4.0
    s = torch.zeros(3, n ** 3, dtype=DT)
    one = pm.deposit(s, torch.ones(n ** 3, dtype=DT), n, box)
    assert torch.equal(one, torch.ones(n, n, n, dtype=DT))        # lattice -> uniform
    s[0, 0] = 0.5                                                   # particle 0 at x = 0.5
    d = pm.deposit(s, torch.ones(n ** 3, dtype=DT), n, box)
    assert d[0, 0, 0].item() == 0.5 and d[0, 0, 1].item() == 1.5


def test_readout_is_transpose_of_deposit():
    n, box = 8, 5.0
    g = torch.Generator().manual_seed(1)
    s = 3 * torch.randn(3, n ** 3, dtype=DT, generator=g)
    w = torch.randn(n ** 3, dtype=DT, generator=g)
    f = torch.randn(n, n, n, dtype=DT, generator=g)
    lhs = (pm.deposit(s, w, n, box) * f).sum()
    rhs = (w * pm.interp(f, s, n, box)).sum()
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_readout_exact_for_affine_field_inside_cell():
    n, box = 8, 8.0
    z, y, x = _grid_x(n, box)
    f = 0.3 + 0.5 * x - 0.2 * y + 0.7 * z
    rng = np.random.default_rng(2)
    s = torch.tensor(rng.uniform(0, 0.99, size=(3, n ** 3)), dtype=DT)
    q = pm.lattice(n).to(DT)
    inside = (q < n - 1).all(0)                  # no periodic wrap between the two nodes
    X = q + s
    ref = 0.3 + 0.5 * X[0] - 0.2 * X[1] + 0.7 * X[2]
    got = pm.interp(f, s, n, box)
    assert torch.allclose(got[inside], ref[inside], atol=1e-13)


def test_fp32_cell_decision_agrees_away_from_boundaries():
    n, box = 8, 8.0
    rng = np.random.default_rng(5)
    s = torch.tensor(rng.uniform(-3, 3, size=(3, n ** 3)).astype(np.float32).astype(np.float64))
    b64, f64 = pm.cic_cells(s, n, box, index_fp32=False)
    b32, f32 = pm.cic_cells(s, n, box, index_fp32=True)
    assert torch.equal(b64, b32)
    assert torch.allclose(f64, f32, atol=1e-12)


def test_gas_kick_exact_composition_and_internal_energy():
    g_ = torch.Generator().manual_seed(4)
    U = torch.rand(5, 3, 3, 3, dtype=DT, generator=g_) + 0.5
    g = torch.randn(3, 3, 3, 3, dtype=DT, generator=g_)
    eint = lambda V: V[4] - (V[1:4] ** 2).sum(0) / (2 * V[0])
    V = pm.gas_kick(U, g, 0.37)
    assert torch.allclose(eint(V), eint(U), atol=1e-13)
    W = pm.gas_kick(pm.gas_kick(U, g, 0.2), g, 0.17)
    assert torch.allclose(V, W, atol=1e-13)


def _pancake(n, box=32.0, om=0.3):
    k = 2 * math.pi / box
    a = C.scale_factors(0.1, 0.5, 20)
    B = 0.5 / C.growth_D(a[-1], om).item()
    q = pm.lattice(n).to(DT) * (box / n)
    psi = torch.zeros(3, n ** 3, dtype=DT)
    psi[0] = B / k * torch.sin(k * q[0])
    s = C.growth_D(a[0], om) * psi
    p = C.g_p(a[0], om) * psi
    zero = torch.zeros(n, n, n, dtype=DT)

    def force(s, at):
        delta = pm.density_contrast(s, zero, 0.0, n, box)
        return pm.gravity(delta, C.poisson_prefactor(at, om), box)

    g = force(s, a[0])
    for a0, a1 in zip(a[:-1], a[1:]):
        f = C.step_factors(a0, a1, om)
        p = pm.particle_kick(p, s, g, f["K1"], box)
        s = pm.drift(s, p, f["dtau"])
        g = force(s, a1)
        p = pm.particle_kick(p, s, g, f["K2"], box)
    ref_s = C.growth_D(a[-1], om) * psi[0]
    ref_p = C.g_p(a[-1], om) * psi[0]
    es = ((s[0] - ref_s).abs().max() / ref_s.abs().max()).item()
    ep = ((p[0] - ref_p).abs().max() / ref_p.abs().max()).item()
    return es, ep, s[1:].abs().max().item()


@pytest.mark.slow
def test_zeldovich_pancake_before_shell_crossing():
    # DM only (f_b = 0, no gas): psi_x(q) = (B/k) sin(k q_x), delta_L = -D B cos(k q_x).
    # Shell crossing at D B = 1; B D(a_end) = 0.5 keeps the run well before it. Particles
    # start on the mesh nodes, where CIC deposit of sub-cell displacements is a one-sided
    # difference: the error is first order in k dx, so it must halve when dx halves.
    es32, ep32, t32 = _pancake(32)
    es64, ep64, t64 = _pancake(64)
    assert es32 < 0.06 and ep32 < 0.08
    assert 0.4 < es64 / es32 < 0.6 and 0.4 < ep64 / ep32 < 0.6
    assert t32 < 1e-12 and t64 < 1e-12          # plane symmetry kept
