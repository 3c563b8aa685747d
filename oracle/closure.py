"""Learned closure: a small 3-D convolutional correction applied after each step (oracle).

Sec. 4 lists "solver-in-the-loop" refinement among the uses a differentiable solver opens:
a network, trained against better-resolved runs, corrects the coarse solution at every
step. The network here is the one the parameter-sampling studies call for: four periodic
3x3x3 convolutions 5 -> 16 -> 16 -> 16 -> 5 with GELU between them, acting as a residual
correction of the five gas fields on normalised inputs:

    x  = q((u - mu) / sigma)                    (per field; q = round to bfloat16)
    h1 = q(GELU(conv(x,  W1) + b1))
    h2 = q(GELU(conv(h1, W2) + b2))
    h3 = q(GELU(conv(h2, W3) + b3))
    y  = conv(h3, W4) + b4                       (float, 5 channels)
    u' = u + s * y                               (per field scale s)

with conv(h, W)[v, co] = sum over the 27 taps t and input channels ci of
h[v + off(t), ci] W[t, ci, co] (cross-correlation, periodic in every axis), tap
t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1) for the offset (dx, dy, dz) in {-1, 0, 1}^3,
GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, the weights W rounded to bfloat16
before use and the biases b kept as given (float32 values). Arithmetic is float64 here,
the reference for a float32-accumulating kernel: the quantisation points q are part of
the definition, the accumulation precision is not. The gradient is torch's reverse mode of this float64
arithmetic with the rounding treated as the identity.

Weight vector (flat float32, the layout the C ABI uses): for layers l = 1..4 with
(Cin, Cout) = (5, 16), (16, 16), (16, 16), (16, 5): W_l[t][ci][co] (27 Cin Cout values,
co fastest) followed by b_l[co].

Also here: the coarse/fine pairing of the training runs -- the band-limited (Fourier)
interpolation of coarse white noise onto a grid twice as fine, the tent restriction of a
fine gas state, and the subsampling of fine particles onto the coarse lattice.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F

LAYERS = ((5, 16), (16, 16), (16, 16), (16, 5))
N_WEIGHTS = sum(27 * ci * co + co for ci, co in LAYERS)  # 18197
_DT = torch.float64


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    return torch.as_tensor(x, dtype=_DT).to(torch.bfloat16).to(_DT)


def gelu(z):
    return 0.5 * z * (1.0 + torch.erf(z / math.sqrt(2.0)))


def unpack(wvec):
    """Flat weight vector -> [(W [27, Cin, Cout], b [Cout]) per layer], float64."""
    w = torch.as_tensor(np.asarray(wvec, dtype=np.float64))
    out, o = [], 0
    for ci, co in LAYERS:
        W = w[o:o + 27 * ci * co].reshape(27, ci, co)
        o += 27 * ci * co
        b = w[o:o + co]
        o += co
        out.append((W, b))
    assert o == w.numel()
    return out


def unpack_t(w):
    """unpack() for a float64 torch tensor (keeps the autograd graph)."""
    out, o = [], 0
    for ci, co in LAYERS:
        W = w[o:o + 27 * ci * co].reshape(27, ci, co)
        o += 27 * ci * co
        out.append((W, w[o:o + co]))
        o += co
    return out


def conv_periodic(h, W):
    """h [C_in, n, n, n] (z, y, x), W [27, C_in, C_out] -> [C_out, n, n, n].

    Written with torch's conv3d on a circularly padded input: kernel element
    (kz, ky, kx) multiplies h[z + kz - 1, y + ky - 1, x + kx - 1], so tap t = 9 kz + 3 ky + kx.
    """
    ci, co = W.shape[1], W.shape[2]
    k = W.reshape(3, 3, 3, ci, co).permute(4, 3, 0, 1, 2).contiguous()  # [co, ci, kz, ky, kx]
    hp = F.pad(h.unsqueeze(0), (1, 1, 1, 1, 1, 1), mode="circular")
    return F.conv3d(hp, k)[0]


def conv_bruteforce(h, W):
    """The same cross-correlation as explicit loops (pin for conv_periodic, tiny n only)."""
    ci, n = h.shape[0], h.shape[1]
    co = W.shape[2]
    out = torch.zeros(co, n, n, n, dtype=_DT)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                for t in range(27):
                    dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
                    v = h[:, (z + dz) % n, (y + dy) % n, (x + dx) % n]
                    out[:, z, y, x] += v @ W[t]
    return out


def network(x, weights, quantise=True):
    """y [5, n, n, n] from normalised input x [5, n, n, n] (float64 tensors)."""
    q = bf16 if quantise else (lambda a: a)
    h = q(x)
    layers = unpack(weights) if not isinstance(weights, list) else weights
    for l, (W, b) in enumerate(layers):
        z = conv_periodic(h, q(W)) + b[:, None, None, None]
        h = q(gelu(z)) if l < 3 else z
    return h


def network_window(xwin, weights, quantise=True):
    """The network's output at the centre of a (2R + 1)^3 window of the input, R = 4 (one
    voxel per layer), with unpadded convolutions: xwin [5, 9, 9, 9] -> y [5] (float64).
    Equal to network() at that voxel for any periodic input (pinned in the tests); used to
    check single voxels of large grids."""
    q = bf16 if quantise else (lambda a: a)
    h = q(torch.as_tensor(xwin, dtype=_DT))
    layers = unpack(weights) if not isinstance(weights, list) else weights
    for l, (W, b) in enumerate(layers):
        ci, co = W.shape[1], W.shape[2]
        k = q(W).reshape(3, 3, 3, ci, co).permute(4, 3, 0, 1, 2).contiguous()
        z = F.conv3d(h.unsqueeze(0), k)[0] + b[:, None, None, None]
        h = q(gelu(z)) if l < 3 else z
    return h[:, 0, 0, 0]


def apply(gas, weights, mu, sigma, scale, quantise=True):
    """u' = u + s * NN((u - mu) / sigma) for gas [5, n, n, n]."""
    mu = torch.as_tensor(mu, dtype=_DT)[:, None, None, None]
    sigma = torch.as_tensor(sigma, dtype=_DT)[:, None, None, None]
    scale = torch.as_tensor(scale, dtype=_DT)[:, None, None, None]
    gas = torch.as_tensor(gas, dtype=_DT)
    x = (gas - mu) / sigma
    return gas + scale * network(x, weights, quantise)


def mse_loss(y, target):
    """L = mean over the 5 fields and all cells of (y - target)^2."""
    return ((y - target) ** 2).mean()


def adam(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) with bias correction; returns the
    new (params, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def he_init(seed: int):
    """Deterministic initial weights: N(0, 2 / (27 Cin)) for W (numpy Generator(seed)),
    zero biases, and the last layer scaled by 0.1 so the correction starts small."""
    g = np.random.default_rng(seed)
    out = []
    for l, (ci, co) in enumerate(LAYERS):
        W = g.standard_normal((27, ci, co)) * math.sqrt(2.0 / (27 * ci))
        if l == 3:
            W *= 0.1
        out.append(W.reshape(-1))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


# ------------------------------------------------------------------ coarse / fine pairing
def refine_noise(w_c, n_f: int, scale: float):
    """Band-limited interpolation of the coarse field w_c [n_c]^3 onto [n_f]^3 (n_f > n_c),
    times `scale`: keep the coarse Fourier modes, zero the rest, and split a Nyquist mode
    of an even n_c equally between +k and -k on the fine grid (so the interpolant is real
    and passes through every coarse value)."""
    w_c = np.asarray(w_c, dtype=np.float64)
    n_c = w_c.shape[0]
    Wc = np.fft.fftn(w_c)
    Wf = np.zeros((n_f, n_f, n_f), dtype=np.complex128)
    kc = np.fft.fftfreq(n_c, 1.0 / n_c).astype(int)  # signed coarse indices
    for iz, kz in enumerate(kc):
        for iy, ky in enumerate(kc):
            for ix, kx in enumerate(kc):
                val = Wc[iz, iy, ix]
                targets = [()]
                for k in (kz, ky, kx):
                    if n_c % 2 == 0 and abs(k) == n_c // 2:
                        opts = [(k, 0.5), (-k, 0.5)]
                    else:
                        opts = [(k, 1.0)]
                    targets = [t + (o,) for t in targets for o in opts]
                for (z, fz), (y, fy), (x, fx) in targets:
                    Wf[z % n_f, y % n_f, x % n_f] += val * fz * fy * fx
    w_f = np.fft.ifftn(Wf).real * (n_f ** 3 / n_c ** 3)
    return scale * w_f


def restrict_gas(gas_f):
    """Fine gas [5, 2n]^3 -> coarse [5, n]^3 with the tent weights (1/4, 1/2, 1/4) per axis
    around fine cell 2j (coarse cell j and fine cell 2j share the node j dx_c); the total
    of every field is preserved up to the factor 8 of the cell volume."""
    g = torch.as_tensor(gas_f, dtype=_DT)
    w = torch.tensor([0.25, 0.5, 0.25], dtype=_DT)
    for axis in (1, 2, 3):
        g = (w[0] * torch.roll(g, 1, axis) + w[1] * g + w[2] * torch.roll(g, -1, axis))
    return g[:, ::2, ::2, ::2].contiguous()


def restrict_particles(part_f, n_f: int):
    """Fine particles [6, n_f^3] (Lagrangian order) -> the coarse lattice's particles: the
    fine particle at lattice site 2q is the coarse particle at q (same Lagrangian point)."""
    p = torch.as_tensor(part_f, dtype=_DT).reshape(6, n_f, n_f, n_f)
    return p[:, ::2, ::2, ::2].reshape(6, -1).contiguous()
