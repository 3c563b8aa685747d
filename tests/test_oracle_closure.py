"""Pins of the closure oracle (oracle/closure.py): convolution, GELU, network, Adam, and the
coarse/fine pairing operators, each against an independent fact."""
import math

import numpy as np
import pytest
import torch

from oracle import closure as oc

DT = torch.float64


def _rand(shape, seed):
    return torch.from_numpy(np.random.default_rng(seed).standard_normal(shape))


def test_conv_matches_bruteforce_loops():
    h = _rand((3, 4, 4, 4), 1)
    W = _rand((27, 3, 2), 2)
    assert torch.allclose(oc.conv_periodic(h, W), oc.conv_bruteforce(h, W), atol=1e-12)


def test_conv_tap_convention():
    """A single tap t with offset (dx, dy, dz) reads the input at v + offset."""
    n = 5
    h = _rand((1, n, n, n), 3)
    for t, (dx, dy, dz) in [(14, (1, 0, 0)), (16, (0, 1, 0)), (22, (0, 0, 1)), (0, (-1, -1, -1))]:
        W = torch.zeros(27, 1, 1, dtype=DT)
        W[t, 0, 0] = 1.0
        want = torch.roll(h, shifts=(-dz, -dy, -dx), dims=(1, 2, 3))
        assert torch.allclose(oc.conv_periodic(h, W), want)


def test_conv_translation_equivariant():
    h = _rand((4, 6, 6, 6), 4)
    W = _rand((27, 4, 3), 5)
    a = oc.conv_periodic(torch.roll(h, (1, -2, 3), (1, 2, 3)), W)
    b = torch.roll(oc.conv_periodic(h, W), (1, -2, 3), (1, 2, 3))
    assert torch.allclose(a, b, atol=1e-12)


def test_gelu_values():
    z = torch.tensor([0.0, 1.0, -1.0, 8.0, -8.0], dtype=DT)
    g = oc.gelu(z)
    assert g[0] == 0.0
    assert abs(g[1].item() - 0.841344746068543) < 1e-14  # Phi(1), standard normal table
    assert abs(g[1].item() - g[2].item() - 1.0) < 1e-15    # GELU(x) - GELU(-x) = x
    assert abs(g[3].item() - 8.0) < 1e-12 and abs(g[4].item()) < 1e-12


def test_bf16_rounding():
    x = torch.tensor([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 3.14159], dtype=DT)
    q = oc.bf16(x)
    assert q[0] == 1.0 and q[1] == 1.0                 # tie to even
    assert q[2] == 1.0 + 2 ** -7                       # tie to even (upwards)
    assert abs(q[3].item() - 3.140625) < 1e-15         # 8 significant bits


def test_zero_network_is_identity():
    n = 4
    gas = torch.rand(5, n, n, n, dtype=DT) + 0.5
    w = np.zeros(oc.N_WEIGHTS, dtype=np.float32)
    out = oc.apply(gas, w, [0.1] * 5, [2.0] * 5, [0.3] * 5)
    assert torch.equal(out, gas)


def test_weight_count_and_layout():
    assert oc.N_WEIGHTS == 27 * 5 * 16 + 16 + 2 * (27 * 16 * 16 + 16) + 27 * 16 * 5 + 5
    w = np.arange(oc.N_WEIGHTS, dtype=np.float64)
    layers = oc.unpack(w)
    assert layers[0][0][1, 2, 3].item() == 1 * 5 * 16 + 2 * 16 + 3
    assert layers[0][1][0].item() == 27 * 5 * 16
    assert layers[3][1][-1].item() == oc.N_WEIGHTS - 1


def test_network_gradient_matches_finite_differences():
    n = 4
    x = _rand((5, n, n, n), 6)
    w = oc.he_init(7).astype(np.float64)
    w[-5:] = 0.1
    tgt = _rand((5, n, n, n), 8) * 0.1
    wt = torch.tensor(w, requires_grad=True)
    L = oc.mse_loss(oc.network(x, oc.unpack_t(wt), quantise=False), tgt)
    g, = torch.autograd.grad(L, wt)
    rng = np.random.default_rng(9)
    for i in rng.choice(oc.N_WEIGHTS, 12, replace=False):
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fp = oc.mse_loss(oc.network(x, wp, quantise=False), tgt).item()
        fm = oc.mse_loss(oc.network(x, wm, quantise=False), tgt).item()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[i].item()) < 1e-7 + 1e-5 * abs(fd), (i, fd, g[i].item())


def test_adam_first_step_and_convergence():
    p = np.array([3.0, -2.0, 0.5])
    g = np.array([0.7, -1e-3, 40.0])
    p1, m, v = oc.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step: m_hat / sqrt(v_hat) = sign(g)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-7)
    # f(p) = |p|^2 / 2 is minimised
    x, m, v = np.array([1.0, -1.0]), np.zeros(2), np.zeros(2)
    for t in range(1, 3001):
        x, m, v = oc.adam(x, x, m, v, t, lr=0.01)
    assert np.abs(x).max() < 0.05


@pytest.mark.parametrize("n_c", [4, 5, 6])
def test_refine_noise_interpolates_coarse_values(n_c):
    w = np.random.default_rng(n_c).standard_normal((n_c, n_c, n_c))
    wf = oc.refine_noise(w, 2 * n_c, 1.5)
    assert np.allclose(wf[::2, ::2, ::2], 1.5 * w, atol=1e-12)


def test_refine_noise_keeps_a_cosine_mode():
    n_c, n_f = 8, 16
    x_c = np.arange(n_c) / n_c
    x_f = np.arange(n_f) / n_f
    c = np.cos(2 * np.pi * 3 * x_c)[None, None, :] * np.ones((n_c, n_c, 1))
    f = np.cos(2 * np.pi * 3 * x_f)[None, None, :] * np.ones((n_f, n_f, 1))
    assert np.allclose(oc.refine_noise(c, n_f, 1.0), f, atol=1e-12)
    # a Nyquist mode of the coarse grid becomes the band-limited cos(pi x / dx_c)
    c = np.cos(np.pi * np.arange(n_c))[None, :, None] * np.ones((n_c, 1, n_c))
    f = np.cos(np.pi * np.arange(n_f) / 2)[None, :, None] * np.ones((n_f, 1, n_f))
    assert np.allclose(oc.refine_noise(c, n_f, 1.0), f, atol=1e-12)


def test_restrict_gas_constant_total_and_transfer():
    n_f = 8
    const = torch.full((5, n_f, n_f, n_f), 2.5, dtype=DT)
    assert torch.allclose(oc.restrict_gas(const), torch.full((5, 4, 4, 4), 2.5, dtype=DT))
    g = _rand((5, n_f, n_f, n_f), 10)
    assert torch.allclose(oc.restrict_gas(g).sum((1, 2, 3)) * 8, g.sum((1, 2, 3)), atol=1e-10)
    # tent filter transfer 1/2 + cos(k dx_f)/2 on a cosine along x
    k = 2 * np.pi * 2 / n_f
    xf = torch.arange(n_f, dtype=DT)
    fine = torch.cos(k * xf).expand(5, n_f, n_f, n_f)
    want = torch.cos(k * 2 * torch.arange(4, dtype=DT)) * (0.5 + 0.5 * math.cos(k))
    got = oc.restrict_gas(fine)
    assert torch.allclose(got, want.expand(5, 4, 4, 4), atol=1e-12)


def test_restrict_particles_picks_even_lattice_sites():
    n_f = 6
    q = torch.arange(n_f ** 3, dtype=DT)
    part = torch.stack([q + 1000 * c for c in range(6)])
    out = oc.restrict_particles(part, n_f)
    for qz, qy, qx in [(0, 0, 0), (1, 2, 0), (2, 1, 2)]:
        i_c = (qz * 3 + qy) * 3 + qx
        i_f = ((2 * qz) * n_f + 2 * qy) * n_f + 2 * qx
        assert torch.equal(out[:, i_c], part[:, i_f])


def test_network_window_matches_periodic_network():
    n = 10
    x = _rand((5, n, n, n), 11)
    w = oc.he_init(12).astype(np.float64)
    w[-5:] = 0.05
    y = oc.network(x, w)
    for (z0, y0, x0) in [(0, 0, 0), (9, 3, 5), (4, 9, 1)]:
        idx = [torch.arange(c - 4, c + 5) % n for c in (z0, y0, x0)]
        win = x[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
        assert torch.allclose(oc.network_window(win, w), y[:, z0, y0, x0], atol=1e-12)
