"""Config-2 gradient check on the GPU: forward + adjoint at 64^3 (64^3 particles), the IC
recipe, 50 steps a = 0.1 -> 1.0 in float32; loss = MSE between the final gas density and
the final density of a run from another seed. Gradients with respect to the 64^3 white
noise (20 random directions) and to (Omega_m, sigma8) against central finite differences.

The loss is piecewise smooth: CIC cell crossings, the limiter gate, |v| and the sound-speed
clamp are kinks. Measured on this grid (12 directions, h = 1e-3, 5e-3, 2e-2):
  - 10 steps a = 0.1 -> 0.2 (before shocks): adjoint and differences agree to 6e-4 of the
    RMS directional derivative at h = 1e-3 (median 1.4e-4 relative), the gap growing with
    h as the truncation error does: the smooth regime, checked below at 2e-3 / 1e-3;
  - 50 steps a = 0.1 -> 1.0: the gap is 1-3.5% of the RMS and does not shrink with h
    (3.5%, 3.4%, 3.5%): the run crosses kinks at spacings far below any usable h, so the
    differences measure a mean slope while reverse mode gives the slope of the branch at
    the point (the float64 oracle shows the same 0.05-3% spread on 16^3 runs). Which
    kinks lie near the point also moves with the last bit of the forward's rounding. The
    50-step check therefore bars each direction at 5% of the RMS and the median relative
    gap at 2.5%.
The 50-step test here is therefore a robustness check of the adjoint against float32
differences, not the gradient bar of the workload (1e-3). That bar is checked against the
float64 oracle's reverse mode of whole runs: 50 steps a = 0.1 -> 1.0 at 16^3 and 32^3
(tests/test_gpu_parity_runs.py), shorter runs from 12^3 to 64^3 (tests/test_gpu_sim.py),
and the smooth-regime differences and float64 differences at h = 2e-6 below.
"""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import f32, lib, need_gpu, oracle_params

pytestmark = pytest.mark.gpu

N, STEPS = 64, 50


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    dh = lib()
    p = dh.default_params(n=N, box=float(N), n_steps=STEPS, a_start=0.1, a_end=1.0,
                          ckpt_every=10, seed=1)
    tsim = dh.Simulation(dh.default_params(n=N, box=float(N), n_steps=STEPS, a_start=0.1,
                                           a_end=1.0, seed=2))
    tsim.run()
    target = tsim.state()["gas"][0].contiguous().clone()
    tsim.close()
    noise = torch.from_numpy(synth.white_noise(N, 11).astype(np.float32)).cuda()
    return dh, p, noise, target


def _loss(dh, p, noise, target, n=N):
    sim = dh.Simulation(p, noise)
    sim.run()
    _, loss = sim.loss_density(target, 1.0 / n ** 3)
    return loss.item(), sim


def test_noise_gradient_robust_against_float32_differences_50_steps(setup):
    dh, p, noise, target = setup
    L0, sim = _loss(dh, p, noise, target)
    dL, _ = sim.loss_density(target, 1.0 / N ** 3)
    dnoise, _ = sim.run_adjoint(dL)
    sim.close()
    g = torch.Generator().manual_seed(123)
    h = 5e-3
    ads, fds = [], []
    for k in range(20):
        d = torch.randn(N, N, N, generator=g).cuda()
        ads.append((dnoise.double() * d.double()).sum().item())
        lp, s1 = _loss(dh, p, (noise + h * d).contiguous(), target)
        s1.close()
        lm, s2 = _loss(dh, p, (noise - h * d).contiguous(), target)
        s2.close()
        fds.append((lp - lm) / (2 * h))
    ads, fds = np.array(ads), np.array(fds)
    scale = np.sqrt(np.mean(fds ** 2))
    assert np.all(np.abs(ads - fds) <= 0.05 * scale), np.abs(ads - fds) / scale
    assert np.median(np.abs(ads - fds) / np.abs(fds)) < 0.025, np.abs(ads - fds) / np.abs(fds)


def test_noise_gradient_matches_finite_differences_smooth_regime():
    """64^3, 10 steps a = 0.1 -> 0.2 (before shell crossing and shocks), h = 1e-3."""
    need_gpu()
    dh = lib()
    steps, a1 = 10, 0.2
    p = dh.default_params(n=N, box=float(N), n_steps=steps, a_start=0.1, a_end=a1,
                          ckpt_every=5, seed=1)
    tsim = dh.Simulation(dh.default_params(n=N, box=float(N), n_steps=steps, a_start=0.1,
                                           a_end=a1, seed=2))
    tsim.run()
    target = tsim.state()["gas"][0].contiguous().clone()
    tsim.close()
    noise = torch.from_numpy(synth.white_noise(N, 11).astype(np.float32)).cuda()
    L0, sim = _loss(dh, p, noise, target)
    dL, _ = sim.loss_density(target, 1.0 / N ** 3)
    dnoise, _ = sim.run_adjoint(dL)
    sim.close()
    g = torch.Generator().manual_seed(321)
    h = 1e-3
    ads, fds = [], []
    for k in range(20):
        d = torch.randn(N, N, N, generator=g).cuda()
        ads.append((dnoise.double() * d.double()).sum().item())
        lp, s1 = _loss(dh, p, (noise + h * d).contiguous(), target)
        s1.close()
        lm, s2 = _loss(dh, p, (noise - h * d).contiguous(), target)
        s2.close()
        fds.append((lp - lm) / (2 * h))
    ads, fds = np.array(ads), np.array(fds)
    scale = np.sqrt(np.mean(fds ** 2))
    assert np.all(np.abs(ads - fds) <= 2e-3 * scale), np.abs(ads - fds) / scale
    assert np.median(np.abs(ads - fds) / np.abs(fds)) < 1e-3, np.abs(ads - fds) / np.abs(fds)


@pytest.mark.parametrize("name,idx", [("omega_m", 0), ("sigma8", 1)])
def test_parameter_gradient_matches_finite_differences(setup, name, idx):
    dh, p, noise, target = setup
    L0, sim = _loss(dh, p, noise, target)
    dL, _ = sim.loss_density(target, 1.0 / N ** 3)
    _, dpar = sim.run_adjoint(dL)
    sim.close()
    ad = dpar[idx].item()
    x0 = getattr(p, name)
    h = 1e-3 * x0
    vals = []
    for sgn in (1, -1):
        q = dh.SimParams.from_buffer_copy(p)
        setattr(q, name, x0 + sgn * h)
        v, s = _loss(dh, q, noise, target)
        s.close()
        vals.append(v)
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(ad - fd) < 1e-3 * abs(fd), (ad, fd)


def test_noise_gradient_matches_float64_finite_differences():
    """GPU adjoint of a 16^3, 50-step run (a = 0.1 -> 1) against central differences of the
    float64 oracle at h = 2e-6 on 4 random directions (within 1e-2 relative). The UV floor
    (T0 = 1e4 K, subgrid on with delta_c = 100 so that no star forms) keeps the pressure
    positive; without it the single-energy pressure of this run turns negative in ~8% of
    the cells by a = 1, where float32 and float64 gradients part (the sound-speed
    derivative diverges at P = 0)."""
    need_gpu()
    dh = lib()
    from oracle import sim as osim
    n = 16
    p = dh.default_params(n=n, box=float(n), n_steps=STEPS, a_start=0.1, a_end=1.0,
                          ckpt_every=10, seed=1, subgrid_on=1, delta_c=100.0, T0_uv=1e4,
                          gamma_uv=1.4)
    o = oracle_params(p)
    target_o = osim.run(osim.noise_field(dict(o, seed=2)), dict(o, seed=2))["U"][0]
    tg = target_o.float().cuda().contiguous()
    wg, wo = f32(synth.white_noise(n, 11))
    sim = dh.Simulation(p, wg)
    sim.run()
    dL, _ = sim.loss_density(tg, 1.0 / n ** 3)
    dnoise, _ = sim.run_adjoint(dL)
    sim.close()
    fun = lambda w: osim.mse_density(osim.run(w, o)["U"], target_o).item()
    g = torch.Generator().manual_seed(5)
    h = 2e-6
    for k in range(4):
        d = torch.randn(n, n, n, generator=g, dtype=torch.float64)
        ad = (dnoise.double().cpu() * d).sum().item()
        fd = (fun(wo + h * d) - fun(wo - h * d)) / (2 * h)
        assert abs(ad - fd) <= 1e-2 * abs(fd), (k, ad, fd)
