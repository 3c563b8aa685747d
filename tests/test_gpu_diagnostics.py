"""Per-step diagnostics on the GPU (sim_set_diagnostics / sim_diagnostics).

* Conservation over a run with gravity and hydro (Sec. 2.2-2.3): the gas mass is constant
  and the total momentum (gas + dark matter) is conserved, to float32 round-off, at every
  recorded step; the recorded scale factors follow the schedule.
* Each record equals the sums and minima of the state read back from the handle (float64
  sums on the host), and its event count equals the set bits of the event words.
* Records made while sim_run replays a captured graph equal those of an eager run.
* A non-finite cell is counted and left out of the sums.
"""
import math

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import f32, lib, need_gpu

pytestmark = pytest.mark.gpu
SUB = dict(subgrid_on=1, delta_c=0.3, w_delta=0.05, T_c=1e6, w_T=1e5, Pi0=0.2, T0_uv=5e3)


@pytest.fixture(scope="module")
def dh():
    need_gpu()
    return lib()


def test_run_conserves_mass_and_total_momentum(dh):
    n, steps = 24, 16
    p = dh.default_params(n=n, box=float(n), n_steps=steps, ckpt_every=4, a_start=0.1,
                          a_end=0.6, rms_ref=0.2)
    sim = dh.Simulation(p, f32(synth.white_noise(n, 12))[0])
    sim.set_diagnostics(True)
    sim.run()
    st = sim.state()
    fb = p.omega_b / p.omega_m
    cm = 1.0 - fb
    scale = st["gas"][1:4].double().abs().sum().item() + cm * st["p"].double().abs().sum().item()
    recs = [sim.diagnostics(k) for k in range(steps + 1)]
    M0 = recs[0]["mass"]
    assert abs(M0 / (fb * n ** 3) - 1) < 1e-6
    P0 = np.array([recs[0][c] + recs[0][d] for c, d in (("mx", "px"), ("my", "py"), ("mz", "pz"))])
    for k, r in enumerate(recs):
        assert abs(r["mass"] / M0 - 1) < 2e-6, (k, r["mass"], M0)
        Pk = np.array([r["mx"] + r["px"], r["my"] + r["py"], r["mz"] + r["pz"]])
        assert np.abs(Pk - P0).max() < 1e-5 * scale, (k, Pk - P0, scale)
        assert r["nonfinite"] == 0 and r["rho_min"] > 0
        want_a = p.a_start + (p.a_end - p.a_start) * k / steps
        assert abs(r["a"] - want_a) < 1e-12
    sim.close()


def test_record_equals_state_sums(dh):
    n = 16
    p = dh.default_params(n=n, box=16.0, n_steps=6, a_start=0.1, a_end=0.4, rms_ref=0.15, **SUB)
    sim = dh.Simulation(p, f32(synth.white_noise(n, 13))[0])
    sim.set_diagnostics(True)
    prev_star = sim.state()["star"].double().clone()
    total_events = 0
    for k in range(1, 4):
        sim.step()
        st = sim.state()
        r = sim.diagnostics(k)
        g = st["gas"].double()
        gam = p.gamma
        P = (gam - 1) * (st["gas"][4] - 0.5 * (st["gas"][1:4] ** 2).sum(0) / st["gas"][0])
        cm = 1 - p.omega_b / p.omega_m
        for name, want in (("mass", g[0].sum()), ("mx", g[1].sum()), ("my", g[2].sum()),
                           ("mz", g[3].sum()), ("energy", g[4].sum()),
                           ("px", cm * st["p"][0].double().sum()),
                           ("pz", cm * st["p"][2].double().sum())):
            want = want.item()
            tol = 1e-6 * (g[0].abs().sum().item() if name == "mass" else
                          g[4].abs().sum().item() if name == "energy" else
                          g[1:4].abs().sum().item() + cm * st["p"].double().abs().sum().item())
            assert abs(r[name] - want) <= tol, (k, name, r[name], want)
        assert r["rho_min"] == st["gas"][0].min().item()
        assert abs(r["p_min"] - P.min().item()) <= 1e-6 * P.abs().max().item()
        ev = int(np.unpackbits(st["events"].cpu().numpy().view(np.uint8)).sum())
        assert r["events"] == ev
        total_events += ev
        star = st["star"].double()
        assert abs(r["stars"] - (star - prev_star).sum().item()) <= 1e-5 * max(1.0, star.sum().item())
        prev_star = star.clone()
    assert total_events > 0
    sim.close()


def test_records_under_graph_replay_equal_eager(dh):
    n = 16
    p = dh.default_params(n=n, box=16.0, n_steps=8, ckpt_every=4, a_start=0.1, a_end=0.5,
                          rms_ref=0.15, **SUB)
    wg = f32(synth.white_noise(n, 14))[0]
    out = []
    for graphs in (False, True):
        sim = dh.Simulation(p, wg)
        sim.set_graphs(graphs)
        sim.set_diagnostics(True)
        for rep in range(2):           # graphs: capture, then replay
            sim.reinit(wg)
            sim.run()
            out.append([sim.diagnostics(k) for k in range(9)])
        sim.close()
    for recs in out[1:]:
        for a, b in zip(out[0], recs):
            assert a == b


def test_non_finite_cell_is_counted(dh):
    n = 16
    p = dh.default_params(n=n, box=16.0, n_steps=4, a_start=0.1, a_end=0.3, rms_ref=0.1,
                          gravity_on=0)
    sim = dh.Simulation(p, f32(synth.white_noise(n, 4))[0])
    st = sim.state()
    gas = st["gas"].cpu().numpy().copy()
    part = torch.cat([st["s"], st["p"]]).cpu().numpy()
    gas[4, 1, 2, 3] = float("nan")
    sim.set_state(f32(gas)[0], f32(part)[0], 0)
    sim.set_diagnostics(True)
    sim.step()
    r0 = sim.diagnostics(0)
    assert r0["nonfinite"] == 1
    assert math.isfinite(r0["mass"]) and math.isfinite(r0["energy"])
    r1 = sim.diagnostics(1)
    assert r1["nonfinite"] >= 1
    sim.close()
