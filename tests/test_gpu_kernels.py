"""GPU parity of each kernel against the FP64 oracle on identical float32 inputs.

Tolerances (relative L2 over a field unless stated): 1e-5 for forward kernels (the per-step
bar), 1e-4 for adjoints (longer FP32 chains; both are far below any modelling error).
Integer work (Philox words, CIC cell decisions, event bits outside the decision guard band)
is compared exactly.
"""
import math

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import f32, gas, lib, need_gpu, rel_l2
from oracle import hydro, philox as ophilox, pm, spectra, subgrid as osub
from oracle.sim import Params, subgrid_params

pytestmark = pytest.mark.gpu

GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def dh():
    need_gpu()
    return lib()


def _nu(U, frac=0.4):
    return frac / hydro.signal_speed_max(U, GAMMA)


@pytest.mark.parametrize("n", [8, 12, 48, 64, 70, 128])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sweep_forward(dh, n, axis):
    Ug, Uo = f32(gas(n, seed=n + axis))
    nu = _nu(Uo)
    got = dh.sweep(Ug, axis, nu)
    want = hydro.sweep(Uo, "xyz"[axis], nu, GAMMA)
    for k in range(5):
        assert rel_l2(got[k], want[k]) < 1e-5, (k, rel_l2(got[k], want[k]))


def test_sweep_sharp_fronts_and_uniform(dh):
    # Sod-like jump along each axis plus an exactly uniform block (stays exactly uniform)
    n = 32
    U = gas(n, seed=3, rho_rel=0.0, vel=0.0)
    U[0, :, :, : n // 2] *= 8.0
    U[4, :, :, : n // 2] *= 10.0
    Ug, Uo = f32(U)
    for axis in range(3):
        got = dh.sweep(Ug, axis, 0.3)
        want = hydro.sweep(Uo, "xyz"[axis], 0.3, GAMMA)
        for k in (0, 4):
            assert rel_l2(got[k], want[k]) < 1e-5
    Uu = np.zeros((5, 16, 16, 16))
    Uu[0], Uu[1], Uu[4] = 0.3, 0.03, 0.01
    Ug, _ = f32(Uu)
    for axis in range(3):
        assert torch.equal(dh.sweep(Ug, axis, 0.7), Ug)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 20, 64, 70])
@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
def test_sweep_forms_match_oracle(dh, n, variant):
    """Every kernel form (tile, marching in 32- and 16-cell segments or in the segment length
    fitted to whole waves; x adjoint via transposed copies; the paired packed-FP32x2 forward
    form for y / z on even grids) against the oracle, on grids
    smaller than the stencil (2, 3, 5 cells: every halo wraps onto the line itself) and on
    grids with a ragged last tile and segment.

    The forms evaluate the same expressions in different orders (gather vs scatter of the
    face terms), and the marching form's face block runs in packed FP32x2 instructions,
    which round every product separately where scalar code may contract a product into an
    FMA; the compiler's contraction choices in the inlined forward recompute differ between
    kernels too. Their adjoints agree to 1.0-1.7e-6 relative L2, except where a limiter
    argument lies within float32 rounding of zero and one form's recompute takes the other
    branch (measured: 4 adjacent cells of 343,000 at n = 70, 32-cell segments, z axis:
    1.4e-3 overall). The forms are therefore compared like the oracle: 5e-6 outside the
    0.1 % worst cells (at least one) and 1e-2 overall.
    Against the float64 oracle a face whose limiter arguments straddle zero within float32
    rounding takes the other branch in a few isolated cells (e.g. one cell at n = 20, seed
    101, y axis: 3.4e-3 overall); the oracle bar is therefore 1e-4 outside the 0.1 %
    worst cells (at least one) and 1e-2 overall."""
    Ug, Uo = f32(gas(n, seed=5 * n + variant))
    lam_g, lam_o = f32(synth.field(n, seed=98, shape=(5, n, n, n)))
    nu = _nu(Uo)
    for axis in range(3):
        got = dh.sweep(Ug, axis, nu, variant=variant)
        want = hydro.sweep(Uo, "xyz"[axis], nu, GAMMA)
        for k in range(5):
            assert rel_l2(got[k], want[k]) < 1e-5, (axis, k, rel_l2(got[k], want[k]))
        gl, dnu = dh.sweep_adjoint(Ug, lam_g, axis, nu, variant=variant)
        ref_form, dnu_ref = dh.sweep_adjoint(Ug, lam_g, axis, nu, variant=1)
        X = Uo.clone().requires_grad_(True)
        nut = torch.tensor(nu, dtype=torch.float64, requires_grad=True)
        out = (hydro.sweep(X, "xyz"[axis], nut, GAMMA) * lam_o).sum()
        gx, gnu = torch.autograd.grad(out, (X, nut))
        for k in range(5):
            df = (gl[k] - ref_form[k]).double().cpu().flatten()
            assert df.norm().item() < 1e-2 * ref_form[k].double().norm().item(), (axis, k, "forms differ")
            kf = torch.ones_like(df, dtype=torch.bool)
            kf[torch.topk(df.abs(), max(1, df.numel() // 1000)).indices] = False
            assert df[kf].norm().item() < 5e-6 * ref_form[k].double().norm().item(), \
                (axis, k, "forms differ outside worst cells")
            err = rel_l2(gl[k], gx[k])
            assert err < 1e-2, (axis, k, err)
            d = (gl[k].double().cpu() - gx[k]).flatten()
            keep = torch.ones_like(d, dtype=torch.bool)
            keep[torch.topk(d.abs(), max(1, d.numel() // 1000)).indices] = False
            assert d[keep].norm().item() < 1e-4 * gx[k].norm().item(), (axis, k, "outside worst cells")
        # d/dnu sums face terms that largely cancel: a face whose limiter argument one form
        # rounds to the other branch moves it by up to ~1e-2 (measured 7e-3 at n = 70), so the
        # forms and the oracle are held to 1e-2 of it
        assert abs(dnu.item() - dnu_ref.item()) < 1e-2 * abs(dnu_ref.item())
        assert abs(dnu.item() - gnu.item()) < 1e-2 * abs(gnu.item())


@pytest.mark.parametrize("variant", [2, 4, 5])
def test_x_adjoint_marching_forms_128(dh, variant):
    """The marching x adjoint (on x <-> y transposed copies) at the benchmark's n = 128,
    where its segments are fitted to whole waves: against the tile form and the oracle with
    the bars of the forms test."""
    n, axis = 128, 0
    Ug, Uo = f32(gas(n, seed=77))
    lam_g, lam_o = f32(synth.field(n, seed=78, shape=(5, n, n, n)))
    nu = _nu(Uo)
    gl, dnu = dh.sweep_adjoint(Ug, lam_g, axis, nu, variant=variant)
    ref_form, dnu_ref = dh.sweep_adjoint(Ug, lam_g, axis, nu, variant=1)
    X = Uo.clone().requires_grad_(True)
    nut = torch.tensor(nu, dtype=torch.float64, requires_grad=True)
    out = (hydro.sweep(X, "x", nut, GAMMA) * lam_o).sum()
    gx, gnu = torch.autograd.grad(out, (X, nut))
    for k in range(5):
        df = (gl[k] - ref_form[k]).double().cpu().flatten()
        kf = torch.ones_like(df, dtype=torch.bool)
        kf[torch.topk(df.abs(), max(1, df.numel() // 1000)).indices] = False
        assert df[kf].norm().item() < 5e-6 * ref_form[k].double().norm().item(), (k, "forms differ")
        d = (gl[k].double().cpu() - gx[k]).flatten()
        keep = torch.ones_like(d, dtype=torch.bool)
        keep[torch.topk(d.abs(), max(1, d.numel() // 1000)).indices] = False
        assert d[keep].norm().item() < 1e-4 * gx[k].norm().item(), (k, "outside worst cells")
        assert rel_l2(gl[k], gx[k]) < 1e-2
    assert abs(dnu.item() - dnu_ref.item()) < 1e-2 * abs(dnu_ref.item())
    assert abs(dnu.item() - gnu.item()) < 1e-2 * abs(gnu.item())


@pytest.mark.parametrize("n", [8, 20, 48, 64])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sweep_adjoint(dh, n, axis):
    Ug, Uo = f32(gas(n, seed=7 * n + axis))
    lam_g, lam_o = f32(synth.field(n, seed=99, shape=(5, n, n, n)))
    nu = _nu(Uo)
    got, dnu = dh.sweep_adjoint(Ug, lam_g, axis, nu)
    X = Uo.clone().requires_grad_(True)
    nut = torch.tensor(nu, dtype=torch.float64, requires_grad=True)
    out = (hydro.sweep(X, "xyz"[axis], nut, GAMMA) * lam_o).sum()
    gx, gnu = torch.autograd.grad(out, (X, nut))
    for k in range(5):
        assert rel_l2(got[k], gx[k]) < 1e-4, (k, rel_l2(got[k], gx[k]))
    assert abs(dnu.item() - gnu.item()) < 1e-4 * abs(gnu.item())


def _positions(n, seed, scale):
    s = synth.displacements(n, seed, scale)
    # a few particles exactly on nodes and exactly half way, and far outside the box
    s[:, :5] = 0.0
    s[0, 5:10] = 0.5 * (10.0 / n)
    s[:, 10:12] = -3.0 * (10.0 / n) * n
    return s


@pytest.mark.parametrize("n", [2, 3, 8, 16, 33])
def test_deposit_and_readout(dh, n):
    box = 10.0
    sg, so = f32(_positions(n, 5, 2.5 * box / n))
    vg, vo = f32(synth.rng(6).uniform(0.5, 2.0, size=n ** 3))
    got = dh.deposit_cic(sg, n, box, values=vg)
    want = pm.deposit(so, vo, n, box, index_fp32=True)
    assert (got.double().cpu() - want).abs().max().item() < 2e-6 * want.abs().max().item()
    # mass is conserved to the fixed-point resolution
    assert abs(got.double().sum().item() - vo.sum().item()) < 1e-4
    fg, fo = f32(synth.field(n, 8, shape=(3, n, n, n)))
    got = dh.interp_cic(fg, sg, n, box)
    want = pm.interp(fo, so, n, box, index_fp32=True)
    assert rel_l2(got, want) < 1e-6


def test_deposit_deterministic(dh):
    n, box = 32, 32.0
    sg, _ = f32(_positions(n, 9, 3.0))
    a = dh.deposit_cic(sg, n, box)
    b = dh.deposit_cic(sg, n, box)
    assert torch.equal(a, b)


@pytest.mark.parametrize("n", [8, 16, 48, 64])
def test_gravity_and_adjoint(dh, n):
    box, pref = 1.3 * n, 0.77
    dg, do = f32(synth.field(n, 11))
    got = dh.gravity(dg, box, pref)
    want = pm.gravity(do, pref, box)
    assert rel_l2(got, want) < 1e-5
    lg, lo = f32(synth.field(n, 12, shape=(3, n, n, n)))
    got = dh.gravity_adjoint(lg, box, pref)
    X = do.clone().requires_grad_(True)
    (gx,) = torch.autograd.grad((pm.gravity(X, pref, box) * lo).sum(), X)
    assert rel_l2(got, gx) < 1e-5


def _subgrid_state(n, seed):
    prm = Params(T0_uv=8e3, gamma_uv=1.3, delta_c=1.5, w_delta=0.3, T_c=2e4, w_T=3e3,
                 Pi0=0.3, E0=0.03, seed=77).as_dict()
    sp = subgrid_params(prm)
    a = 0.4
    rng = synth.rng(seed)
    rho = sp["f_b"] * (1 + prm["delta_c"] + 3 * prm["w_delta"] * rng.normal(size=(n, n, n)))
    rho = np.abs(rho) + 0.01
    m = 0.05 * rho * rng.normal(size=(3, n, n, n))
    T = prm["T_c"] + 3 * prm["w_T"] * rng.normal(size=(n, n, n))
    e = np.abs(T) / osub.t_per_e(GAMMA, 0.6)
    eps = a * a * rho * e + (m * m).sum(0) / (2 * rho)
    return np.concatenate([rho[None], m, eps[None]]), prm, sp, a


@pytest.mark.parametrize("n", [16, 30])
def test_subgrid_forward_and_events(dh, n):
    U, prm, sp, a = _subgrid_state(n, 4)
    step = 3
    p = dh.default_params(**{k: prm[k] for k in ("delta_c", "w_delta", "T_c", "w_T", "Pi0", "E0",
                                                 "T0_uv", "gamma_uv", "tau", "seed")})
    Ug, Uo = f32(U)
    zh, ev = dh.subgrid(Ug, a, p, step)
    g0, g1 = ophilox.gumbel_pair(prm["seed"], n ** 3, step)
    g0 = torch.tensor(g0.reshape(n, n, n)); g1 = torch.tensor(g1.reshape(n, n, n))
    Uw, zw, evw = osub.subgrid(Uo, a, sp, g0, g1)
    assert rel_l2(Ug[4], Uw[4]) < 1e-5
    assert torch.equal(Ug[:4].cpu(), torch.from_numpy(U[:4].astype(np.float32)))
    assert (zh.double().cpu() - zw).abs().max() < 1e-4
    # event bits: exact outside a guard band of the decision variable
    bits = ev.cpu().numpy().view(np.uint32)
    got = np.unpackbits(bits.view(np.uint8), bitorder="little")[: n ** 3].astype(bool)
    rho, m = Uo[0], Uo[1:4]
    e = (Uo[4] - (m * m).sum(0) / (2 * rho)) / (a * a * rho)
    x1 = (rho / sp["f_b"] - 1 - sp["delta_c"]) / sp["w_delta"]
    x2 = (sp["T_c"] - osub.t_per_e(GAMMA, 0.6) * e) / sp["w_T"]
    lnpi = math.log(sp["Pi0"]) - torch.nn.functional.softplus(-x1) - torch.nn.functional.softplus(-x2)
    logit = (lnpi - torch.log1p(-torch.exp(lnpi)) + g0 - g1).flatten().numpy()
    far = np.abs(logit) > 1e-4
    assert far.mean() > 0.99
    assert np.array_equal(got[far], evw.flatten().numpy()[far])
    assert 0.02 < got.mean() < 0.98


def test_subgrid_adjoint(dh):
    n = 16
    U, prm, sp, a = _subgrid_state(n, 5)
    step = 2
    p = dh.default_params(**{k: prm[k] for k in ("delta_c", "w_delta", "T_c", "w_T", "Pi0", "E0",
                                                 "T0_uv", "gamma_uv", "tau", "seed")})
    Ug, Uo = f32(U)
    lg, lo = f32(synth.field(n, 21, shape=(5, n, n, n)))
    lam = lg.clone()
    dpar, dfb = dh.subgrid_adjoint(Ug, lam, a, p, step)
    g0, g1 = ophilox.gumbel_pair(prm["seed"], n ** 3, step)
    g0 = torch.tensor(g0.reshape(n, n, n)); g1 = torch.tensor(g1.reshape(n, n, n))
    names = ("delta_c", "Pi0", "E0", "T0_uv", "gamma_uv", "f_b")
    leaves = {k: torch.tensor(float(sp[k]), dtype=torch.float64, requires_grad=True) for k in names}
    X = Uo.clone().requires_grad_(True)
    sp2 = dict(sp, **leaves)
    Uw, _, _ = osub.subgrid(X, a, sp2, g0, g1)
    grads = torch.autograd.grad((Uw * lo).sum(), [X] + [leaves[k] for k in names])
    for k in range(5):
        assert rel_l2(lam[k], grads[0][k]) < 1e-4, (k, rel_l2(lam[k], grads[0][k]))
    idx = {"delta_c": 2, "Pi0": 3, "E0": 4, "T0_uv": 5, "gamma_uv": 6}
    for j, k in enumerate(names[:5]):
        want = grads[1 + j].item()
        assert abs(dpar[idx[k]].item() - want) < 1e-4 * abs(want) + 1e-9, (k, dpar[idx[k]].item(), want)
    want = grads[-1].item()
    assert abs(dfb.item() - want) < 1e-4 * abs(want)


def test_philox_words(dh):
    for seed, step, inst, tag in ((1, 0, 0, 0), (0x123456789ABCDEF, 17, 3, 1)):
        got = dh.philox(seed, step, inst, tag, 5000).cpu().numpy().view(np.uint32)
        want = np.stack(ophilox.words(seed, 5000, step, inst, tag), axis=1)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("n", [16, 24])
def test_power_spectrum(dh, n):
    box = 25.0
    ag, ao = f32(synth.field(n, 31))
    bg, bo = f32(synth.field(n, 32))
    k, P, nm = dh.power_spectrum(ag, box, n)
    kw, Pw, nw = spectra.power_spectrum(ao, box, n)
    assert torch.equal(nm.cpu(), nw)
    assert rel_l2(k, kw) < 1e-12
    assert rel_l2(P, Pw) < 1e-5
    k, P, nm = dh.power_spectrum(ag, box, n, b=bg)
    kw, Pw, nw = spectra.power_spectrum(ao, box, n, bo)
    assert (P.cpu() - Pw).abs().max() < 1e-5 * Pw.abs().max()
