"""Learned closure on GB300 (tcgen05 bfloat16 convolutions) against the FP64 oracle.

Tolerances. The oracle rounds inputs, weights and hidden activations to bfloat16 at the
same points as the kernels and accumulates in float64; the kernels accumulate in float32.
What remains are float32 sums of 432 products (relative ~1e-6) and the rare activation
that lands on the other side of a bfloat16 rounding boundary (one bfloat16 ulp, 2^-8
relative, in a few voxels): 2e-3 relative L2 covers both with margin. The weight gradient
is taken by the kernels with the back-propagated signal also in bfloat16 (2^-9 relative
rounding per element at each of the three layers it passes), against the oracle's exact
float64 gradient of the same quantised forward: 2e-2 relative L2 per layer.
"""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import f32, lib, need_gpu, rel_l2
from oracle import closure as oc

pytestmark = pytest.mark.gpu
DT = torch.float64
MU = [0.15, 0.0, 0.0, 0.0, 1.5e-4]
SIGMA = [0.05, 0.01, 0.01, 0.01, 5e-5]
SCALE = [0.01, 0.002, 0.002, 0.002, 0.003]


@pytest.fixture(scope="module")
def dh():
    need_gpu()
    return lib()


def _weights(seed, bias=0.05):
    w = oc.he_init(seed)
    layers = oc.unpack(w)
    # non-zero biases so that every term of the layer is exercised
    out, o = w.copy(), 0
    for ci, co in oc.LAYERS:
        o += 27 * ci * co
        out[o:o + co] = bias * np.linspace(-1, 1, co)
        o += co
    return out


def _gas(n, seed, B=None):
    if B is None:
        return f32(synth.gas_state(n, seed))
    arr = np.stack([synth.gas_state(n, seed + b) for b in range(B)])
    return f32(arr)


def _closure(dh, w):
    c = dh.Closure(w)
    c.set_norm(MU, SIGMA, SCALE)
    return c


def _x(gas_o):
    mu = torch.tensor(MU, dtype=DT)[:, None, None, None]
    sg = torch.tensor(SIGMA, dtype=DT)[:, None, None, None]
    return (gas_o - mu) / sg


@pytest.mark.parametrize("n", [4, 12, 33, 64])
def test_forward_matches_oracle(dh, n):
    w = _weights(1)
    c = _closure(dh, w)
    gas, gas_o = _gas(n, 3)
    y = c.forward(gas)
    c.status()
    want = oc.network(_x(gas_o), w)
    assert rel_l2(y, want) < 2e-3, rel_l2(y, want)
    c.close()


@pytest.mark.parametrize("n", [128, 130])
def test_forward_sampled_voxels_large_grids(dh, n):
    """n >= 128 keeps tiles inside lines (130: a partial second tile per line)."""
    w = _weights(2)
    c = _closure(dh, w)
    gas, gas_o = _gas(n, 4)
    y = c.forward(gas).double().cpu()
    c.status()
    x = _x(gas_o)
    rng = np.random.default_rng(5)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (5, 127, 128 % n), (n // 2, 1, n - 2)]
    pts += [tuple(rng.integers(0, n, 3)) for _ in range(24)]
    got, want = [], []
    for z0, y0, x0 in pts:
        idx = [torch.arange(q - 4, q + 5) % n for q in (z0, y0, x0)]
        win = x[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
        want.append(oc.network_window(win, w))
        got.append(y[:, z0, y0, x0])
    assert rel_l2(torch.stack(got), torch.stack(want)) < 2e-3
    c.close()


def test_forward_five_tiles_per_line(dh):
    """n = 513: five 128-position tiles per line (one line per CTA), the most tiles per plane
    the grid sizes accepted by the host produce; the accumulator ring then holds six plane
    slots per tile in 480 of the 512 TMEM columns. The input repeats a 57^3 field nine
    times per axis, so each sampled voxel's 9^3 window comes from the small field."""
    n, m = 513, 57
    w = _weights(12)
    c = _closure(dh, w)
    base, base_o = _gas(m, 13)
    gas = base.repeat(1, n // m, n // m, n // m).contiguous()
    y = c.forward(gas)
    c.status()
    x = _x(base_o)
    rng = np.random.default_rng(14)
    # every tile of a line (x = 0, 128, ..., 512), both sides of the CTAs' plane columns
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (102, 5, 127), (103, 6, 128), (205, 500, 255),
           (206, 1, 256), (308, 2, 383), (309, 3, 384), (411, 4, 511), (412, 7, 512)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(20)]
    got, want = [], []
    for z0, y0, x0 in pts:
        idx = [torch.arange(q - 4, q + 5) % m for q in (z0 % m, y0 % m, x0 % m)]
        win = x[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
        want.append(oc.network_window(win, w))
        got.append(y[:, z0, y0, x0].double().cpu())
    assert rel_l2(torch.stack(got), torch.stack(want)) < 2e-3
    c.close()


def test_batched_forward_and_apply(dh):
    n, B = 16, 3
    w = _weights(6)
    c = _closure(dh, w)
    gas, gas_o = _gas(n, 7, B)
    y = c.forward(gas)
    for b in range(B):
        assert rel_l2(y[b], oc.network(_x(gas_o[b]), w)) < 2e-3
    g2 = gas.clone()
    c.apply(g2)
    for b in range(B):
        want = oc.apply(gas_o[b], w, MU, SIGMA, SCALE)
        assert rel_l2(g2[b] - gas[b], want - gas_o[b]) < 2e-3
    c.status()
    c.close()


def test_zero_weights_are_the_identity(dh):
    n = 12
    c = _closure(dh, None)
    gas, _ = _gas(n, 8)
    g2 = gas.clone()
    c.apply(g2)
    assert torch.equal(g2, gas)
    assert torch.count_nonzero(c.forward(gas)) == 0
    c.close()


def test_weights_round_trip(dh):
    w = _weights(9)
    c = dh.Closure(w)
    assert np.array_equal(c.weights(), w)
    c.close()


@pytest.mark.parametrize("n", [8, 20, 33])
def test_gradient_matches_oracle(dh, n):
    w = _weights(10)
    c = _closure(dh, w)
    gas, gas_o = _gas(n, 11)
    tgt, tgt_o = f32(synth.gas_state(n, 12))
    loss, g = c.gradient(gas, tgt)
    wt = torch.tensor(w.astype(np.float64), requires_grad=True)
    layers = oc.unpack_t(wt)
    # quantised forward, rounding as the identity in the reverse pass
    q = lambda a: a + (oc.bf16(a.detach()) - a.detach())
    h = q(_x(gas_o))
    for l, (W, b) in enumerate(layers):
        z = oc.conv_periodic(h, q(W)) + b[:, None, None, None]
        h = q(oc.gelu(z)) if l < 3 else z
    sc = torch.tensor(SCALE, dtype=DT)[:, None, None, None]
    L = oc.mse_loss(h, (tgt_o - gas_o) / sc)
    go, = torch.autograd.grad(L, wt)
    assert abs(loss - L.item()) < 2e-3 * L.item()
    o = 0
    for ci, co in oc.LAYERS:
        k = 27 * ci * co + co
        assert rel_l2(g[o:o + k], go[o:o + k]) < 2e-2, (ci, co, rel_l2(g[o:o + k], go[o:o + k]))
        o += k
    c.close()


def test_training_step_is_adam_and_reduces_loss(dh):
    n = 16
    w = _weights(13)
    c = _closure(dh, w)
    gas, _ = _gas(n, 14)
    # a learnable target: a local function of the input (density contrast feedback)
    tgt = gas.clone()
    tgt[0] += 0.2 * (gas[0] - gas[0].mean())
    l0, g0 = c.gradient(gas, tgt)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    c.train_step(gas, tgt, 1e-3, loss)
    w1 = c.weights()
    # first bias-corrected Adam step: -lr g / (|g| + eps)
    nz = np.abs(g0) > 1e-4 * np.abs(g0).max()
    want = -1e-3 * g0[nz] / (np.abs(g0[nz]) + 1e-8)
    assert np.allclose((w1 - w)[nz], want, atol=1e-6)
    assert abs(loss.item() - l0) < 1e-3 * l0
    for _ in range(100):
        c.train_step(gas, tgt, 3e-3, loss)
    l1, _ = c.gradient(gas, tgt)
    assert l1 < 0.8 * l0, (l0, l1)
    c.status()
    c.close()


def test_refine_noise_matches_oracle(dh):
    for n_c in (8, 9):
        w, w_o = f32(synth.white_noise(n_c, 20 + n_c))
        got = dh.refine_noise(w, 2 * n_c, 0.7)
        want = oc.refine_noise(w_o.numpy(), 2 * n_c, 0.7)
        assert rel_l2(got, torch.from_numpy(want)) < 1e-5
        assert rel_l2(got[::2, ::2, ::2], 0.7 * w_o) < 1e-5


def test_restrictions_match_oracle(dh):
    n_f, B = 16, 2
    g, g_o = f32(np.stack([synth.gas_state(n_f, 30 + b) for b in range(B)]))
    got = dh.restrict_gas(g)
    for b in range(B):
        assert rel_l2(got[b], oc.restrict_gas(g_o[b])) < 1e-6
    p, p_o = f32(np.stack([synth.field(n_f, 40 + b, shape=(6, n_f ** 3)) for b in range(B)]))
    got = dh.restrict_particles(p, n_f)
    for b in range(B):
        assert torch.equal(got[b].cpu().double(), oc.restrict_particles(p_o[b], n_f))


def test_closure_inside_the_solver(dh):
    """sim_step with a closure = the plain step followed by the closure (same kernels), and
    the adjoint refuses while a closure is set."""
    n = 16
    p = dh.default_params(n=n, box=16.0, n_steps=4, a_start=0.1, a_end=0.3, rms_ref=0.15)
    noise, _ = f32(synth.white_noise(n, 50))
    w = _weights(15)
    c = _closure(dh, w)
    plain = dh.Simulation(p, noise)
    corr = dh.Simulation(p, noise)
    corr.set_closure(c)
    plain.step()
    corr.step()
    g = plain.state()["gas"].clone()
    c.apply(g)
    assert torch.equal(corr.state()["gas"], g)
    assert not torch.equal(corr.state()["gas"], plain.state()["gas"])
    with pytest.raises(dh.SimError):
        corr.step_adjoint(torch.zeros(5, n, n, n, device="cuda"), torch.zeros(6, n ** 3, device="cuda"))
    corr.set_closure(None)
    corr.reset()
    plain.reset()
    corr.run()
    plain.run()
    assert torch.equal(corr.state()["gas"], plain.state()["gas"])
    for s in (plain, corr):
        s.close()
    c.close()
