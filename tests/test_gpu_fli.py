"""Field-level inference (Sec. 3.2) on the GPU against the FP64 oracle.

* sim_fli_step: the posterior 1/2 [|d - rho(s)|^2 / sigma^2 + |s|^2] at s (1e-4 relative),
  its gradient through the whole checkpointed run (1e-3 relative L2, the gradient bar),
  and the Adam update, compared with the oracle's Adam applied to the same gradient
  (float32 rounding: 1e-6);
* sim_adam alone (vector and scalar paths, with and without the prior pull) against the
  oracle's Adam over three steps;
* sim_cross_correlation against the oracle's r_c(k), and its limits +1 / -1;
* a short inference in the linear regime recovers the large-scale modes of the truth.
"""
import math

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import f32, lib, need_gpu, oracle_params, rel_l2
from oracle import closure as oc, sim as osim, spectra

pytestmark = pytest.mark.gpu
DT = torch.float64
SUB = dict(subgrid_on=1, delta_c=0.3, w_delta=0.05, T_c=1e6, w_T=1e5, Pi0=0.2, T0_uv=5e3)


@pytest.fixture(scope="module")
def dh():
    need_gpu()
    return lib()


def test_fli_step_matches_oracle(dh):
    n, sig, lr = 12, 0.01, 0.05
    p = dh.default_params(n=n, box=12.0, n_steps=5, ckpt_every=2, a_start=0.1, a_end=0.35,
                          rms_ref=0.15, **SUB)
    o = oracle_params(p)
    sg, so = f32(synth.white_noise(n, 90))
    dg, do = f32(0.16 * (1 + 0.2 * synth.field(n, 91)))
    sim = dh.Simulation(p, sg)
    x = sg.clone()
    m = torch.zeros_like(x)
    v = torch.zeros_like(x)
    grad = torch.empty_like(x)
    loss = sim.fli_step(x, m, v, dg, sig, lr, 1, grad=grad)
    L, g = osim.fli_value_and_grad(so, do, sig, o)
    assert abs(loss.item() / L.item() - 1) < 1e-4, (loss.item(), L.item())
    assert rel_l2(grad, g) < 1e-3, rel_l2(grad, g)
    gg = grad.double().cpu().numpy()
    want, mw, vw = oc.adam(so.numpy(), gg, np.zeros_like(gg), np.zeros_like(gg), 1, lr)
    assert rel_l2(x, torch.tensor(want)) < 1e-6
    assert rel_l2(m, torch.tensor(mw)) < 1e-6
    assert rel_l2(v, torch.tensor(vw)) < 1e-6
    # second iteration: the handle re-runs from the updated amplitudes
    loss2 = sim.fli_step(x, m, v, dg, sig, lr, 2, grad=grad)
    L2, g2 = osim.fli_value_and_grad(torch.tensor(want), do, sig, o)
    assert abs(loss2.item() / L2.item() - 1) < 1e-4
    assert rel_l2(grad, g2) < 1e-3
    with pytest.raises(dh.SimError):
        sim.fli_step(x, m, v, dg, sig, lr, 0)
    sim.close()


@pytest.mark.parametrize("count,prior_w", [(4096, 0.0), (4096, 1.0), (1001, 1.0)])
def test_adam_matches_oracle(dh, count, prior_w):
    rng = synth.rng(count)
    x0 = rng.normal(size=count)
    xg, _ = f32(x0)
    m = torch.zeros_like(xg)
    v = torch.zeros_like(xg)
    xo, mo, vo = xg.double().cpu().numpy(), np.zeros(count), np.zeros(count)
    for t in (1, 2, 3):
        gg, go = f32(rng.normal(size=count))
        prior = torch.zeros(1, dtype=DT, device="cuda")
        gout = torch.empty_like(xg)
        x_before = xg.double().cpu().numpy()
        dh.adam(xg, gg, m, v, t, 0.01, prior_w=prior_w, grad_out=gout, prior=prior)
        gt = go.numpy() + prior_w * xo
        assert rel_l2(gout, torch.tensor(gt)) < 1e-6
        assert abs(prior.item() - 0.5 * prior_w * (x_before ** 2).sum()) <= 1e-5 * (1 + prior.item())
        xo, mo, vo = oc.adam(xo, gt, mo, vo, t, 0.01)
        assert rel_l2(xg, torch.tensor(xo)) < 1e-6, t
        assert rel_l2(v, torch.tensor(vo)) < 1e-5, t


@pytest.mark.parametrize("n", [16, 24])
def test_cross_correlation_matches_oracle(dh, n):
    box = 2.0 * n
    ag, ao = f32(synth.field(n, 5))
    bg, bo = f32(0.5 * synth.field(n, 5) + synth.field(n, 6))
    nb = n // 2
    k, rc, nm = dh.cross_correlation(ag, bg, box, nb)
    ko, _, nmo = spectra.power_spectrum(ao, box, nb)
    rco = spectra.cross_correlation(ao, bo, box, nb)
    assert torch.equal(nm.cpu(), nmo)
    assert torch.allclose(k.cpu(), ko, rtol=1e-12)
    assert (rc.cpu() - rco).abs().max().item() < 1e-6
    _, r1, _ = dh.cross_correlation(ag, ag, box, nb)
    _, r2, _ = dh.cross_correlation(ag, (-ag).contiguous(), box, nb)
    assert (r1.cpu() - 1).abs().max().item() < 1e-12
    assert (r2.cpu() + 1).abs().max().item() < 1e-12


def test_inference_recovers_large_scales_in_linear_regime(dh):
    """A 16^3 box evolved a = 0.1 -> 0.2 (linear regime); the mock is the truth's final gas
    density plus 10% noise; 60 Adam iterations from zero amplitudes."""
    n = 16
    p = dh.default_params(n=n, box=16.0, n_steps=4, ckpt_every=2, a_start=0.1, a_end=0.2,
                          rms_ref=0.1, T_init=1e5)
    truth, _ = f32(synth.white_noise(n, 300))
    ts = dh.Simulation(p, truth)
    ts.run()
    rho = ts.state()["gas"][0].clone()
    ts.close()
    sig = 0.1 * rho.std().item()
    data = (rho + sig * torch.from_numpy(synth.field(n, 301).astype(np.float32)).cuda()).contiguous()
    sim = dh.Simulation(p)
    x, losses = dh.fli_infer(sim, data, sig, 60, 0.05)
    L = losses[:, 0].cpu().numpy()
    assert L[-1] < 0.5 * L[0], (L[0], L[-1])
    _, rc, nm = dh.cross_correlation(x, truth, 16.0, 4)
    assert rc[0].item() > 0.9 and rc[1].item() > 0.8, rc.cpu().numpy()
    sim.close()


def test_thermal_posterior_matches_oracle(dh):
    """The delta_b T probe of Sec. 3.2 (internal energy density eps - |m|^2 / 2 rho), subgrid
    off as in the paper's field-level inference."""
    n = 12
    p = dh.default_params(n=n, box=12.0, n_steps=5, ckpt_every=2, a_start=0.1, a_end=0.35,
                          rms_ref=0.15, T_init=1e5)
    o = oracle_params(p)
    sg, so = f32(synth.white_noise(n, 95))
    sim = dh.Simulation(p, sg)
    sim.run()
    st = sim.state()["gas"].double().cpu()
    u = osim.observable(st, "thermal")
    sig = u.std().item()
    dg, do = f32((u + sig * torch.from_numpy(synth.field(n, 96))).numpy())
    x, xo = f32(synth.white_noise(n, 97))
    loss, grad = sim.posterior(x, dg, sig, observable=dh.OBS_THERMAL)
    L, g = osim.fli_value_and_grad(xo, do, sig, o, kind="thermal")
    assert abs(loss.item() / L.item() - 1) < 1e-4, (loss.item(), L.item())
    assert rel_l2(grad, g) < 1e-3, rel_l2(grad, g)
    # the density observable through the same entry point
    dg2, do2 = f32(0.16 * (1 + 0.2 * synth.field(n, 98)))
    loss2, grad2 = sim.posterior(x, dg2, 0.01, observable=dh.OBS_DENSITY)
    L2, g2 = osim.fli_value_and_grad(xo, do2, 0.01, o, kind="density")
    assert abs(loss2.item() / L2.item() - 1) < 1e-4
    assert rel_l2(grad2, g2) < 1e-3
    sim.close()


@pytest.mark.parametrize("snr", [1.0, 5.0])
def test_lbfgs_inference_thermal_probe(dh, snr):
    """L-BFGS (M = 8) on the thermal probe with pixel-noise variance snr x the data
    variance, in a 16^3 box evolved a = 0.1 -> 0.2: the posterior falls and the large-scale
    amplitudes are recovered (better at the lower noise)."""
    from paper_2502_02294_gb300.inference import fli_lbfgs
    n = 16
    p = dh.default_params(n=n, box=16.0, n_steps=4, ckpt_every=2, a_start=0.1, a_end=0.2,
                          rms_ref=0.1, T_init=1e5)
    truth, _ = f32(synth.white_noise(n, 310))
    ts = dh.Simulation(p, truth)
    ts.run()
    st = ts.state()["gas"].double().cpu()
    ts.close()
    u = osim.observable(st, "thermal")
    sig = math.sqrt(snr) * u.std().item()
    data, _ = f32((u + sig * torch.from_numpy(synth.field(n, 311))).numpy())
    sim = dh.Simulation(p)
    r = fli_lbfgs(sim, data, sig, torch.zeros(n, n, n, device="cuda"), dh.OBS_THERMAL,
                  max_iter=60)
    # from s = 0 the data term is 1/2 sum (signal + noise)^2 / sigma^2 ~ N (1 + snr) / (2 snr);
    # at the posterior mode it is ~ N / 2 (the noise) plus the prior of the recovered modes
    N = n ** 3
    L0, L1 = r.history[0][1], r.history[-1][1]
    _, rc, _ = dh.cross_correlation(r.x.contiguous(), truth, 16.0, 4)
    print(f"\nS/N {snr}: loss {L0:.1f} -> {L1:.1f} in {r.iterations} iterations "
          f"({r.evaluations} evaluations), r_c {rc.cpu().numpy()}")
    assert abs(L0 / (N * (1 + snr) / (2 * snr)) - 1) < 0.1, L0
    assert L1 < 0.56 * N, (L1, r.iterations)
    assert rc[0].item() > (0.8 if snr == 1.0 else 0.5), rc.cpu().numpy()
    sim.close()
