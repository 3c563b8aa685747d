"""GPU parity of the whole path (ICs, steps, runs, adjoints) against the FP64 oracle.

Bars: per step relative L2 <= 1e-5 for density, momentum and energy (and particle
displacement / momentum) from the same float32 state; <= 1e-3 after a full run from the
same white noise; gradients through the C ABI within 1e-3 (relative L2 / relative) of the
oracle's reverse mode, which is itself pinned against finite differences.
"""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import f32, lib, need_gpu, oracle_params, rel_l2
from oracle import ics as oics, philox as ophilox, sim as osim

pytestmark = pytest.mark.gpu
DT = torch.float64


@pytest.fixture(scope="module")
def dh():
    need_gpu()
    return lib()


def _oracle_state(st, o, a):
    s = st["s"].double().cpu()
    U = st["gas"].double().cpu()
    return {"s": s, "p": st["p"].double().cpu(), "U": U, "g": osim.force(s, U[0], o, a),
            "step": st["step"], "star": torch.zeros(U.shape[1:], dtype=DT),
            "aux": torch.zeros(s.shape[1], dtype=DT), "events": []}


# subgrid settings that form stars in these small boxes; every configuration below keeps the
# oracle's CFL number under 0.3 and the density above 0.15 of the mean (checked on the CPU)
SUB = dict(subgrid_on=1, delta_c=0.3, w_delta=0.05, T_c=1e6, w_T=1e5, Pi0=0.2, T0_uv=5e3)


@pytest.mark.parametrize("n", [16, 24])
def test_initial_conditions(dh, n):
    p = dh.default_params(n=n, box=float(n), rms_ref=0.2)
    wg, wo = f32(synth.white_noise(n, 3))
    sim = dh.Simulation(p, wg)
    st = sim.state()
    s, pp, U = oics.initial_conditions(wo, oracle_params(p))
    assert rel_l2(st["s"], s) < 1e-5
    assert rel_l2(st["p"], pp) < 1e-5
    for k in range(5):
        assert rel_l2(st["gas"][k], U[k]) < 1e-5, k
    sim.close()


def test_philox_noise_matches_oracle(dh):
    n = 16
    p = dh.default_params(n=n, box=16.0, seed=12345)
    a = dh.Simulation(p)                      # noise drawn on the device
    wg, _ = f32(ophilox.white_noise(12345, n))
    b = dh.Simulation(p, wg)                  # the oracle's draw passed in
    sa, sb = a.state(), b.state()
    for key in ("gas", "s", "p"):
        assert rel_l2(sa[key], sb[key]) < 2e-6


@pytest.mark.parametrize("n,sub", [(16, False), (16, True), (20, True)])
def test_single_step_parity(dh, n, sub):
    kw = dict(n=n, box=float(n), n_steps=6, a_start=0.1, a_end=0.4, rms_ref=0.15)
    if sub:
        kw.update(SUB)
    p = dh.default_params(**kw)
    o = oracle_params(p)
    sim = dh.Simulation(p, f32(synth.white_noise(n, 1))[0])
    for i in range(3):   # three different Strang orders
        st0 = sim.state()
        sim.step()
        st1 = sim.state()
        a_i = o["a_start"] + (o["a_end"] - o["a_start"]) * i / o["n_steps"]
        ref = osim.step(_oracle_state(st0, o, a_i), o)
        for k in range(5):
            assert rel_l2(st1["gas"][k], ref["U"][k]) < 1e-5, (i, k, rel_l2(st1["gas"][k], ref["U"][k]))
        assert rel_l2(st1["s"], ref["s"]) < 1e-5
        assert rel_l2(st1["p"], ref["p"]) < 1e-5
    sim.close()


def test_config1_forward_run(dh):
    """32^3, box 32 Mpc/h, 20 steps a = 0.1 -> 0.5, no subgrid: final state vs oracle."""
    n = 32
    p = dh.default_params(n=n, box=32.0, n_steps=20, a_start=0.1, a_end=0.5)
    wg, wo = f32(synth.white_noise(n, 1))
    sim = dh.Simulation(p, wg)
    sim.run()
    st = sim.state()
    ref = osim.run(wo, oracle_params(p))
    for k in range(5):
        assert rel_l2(st["gas"][k], ref["U"][k]) < 1e-3, (k, rel_l2(st["gas"][k], ref["U"][k]))
    assert rel_l2(st["s"], ref["s"]) < 1e-3
    # the hard-event and cell-index decisions are taken on each side's own state here, so
    # only the state itself is compared; kernel-level tests compare the decisions exactly
    sim.close()


def test_run_is_deterministic_and_resettable(dh):
    n = 24
    p = dh.default_params(n=n, box=24.0, n_steps=8, a_start=0.1, a_end=0.5, rms_ref=0.15, **SUB)
    sim = dh.Simulation(p)
    sim.run()
    a = sim.state()
    sim.reset()
    sim.run()
    b = sim.state()
    for key in ("gas", "s", "p", "star", "aux", "events"):
        assert torch.equal(a[key], b[key]), key
    sim.close()


# Without the UV floor the gas cools adiabatically while its bulk flow grows; at Mach >> 10
# the single-energy pressure P = (gamma-1)(eps - |m|^2/2rho) is a small difference of large
# numbers and the sound-speed derivative gamma/(2 c_s rho) diverges where P -> 0, so float32
# and float64 gradients part there. The subgrid-off cases start warmer (T_init = 1e5 K) to
# stay away from P ~ 0; the cold regime is exercised by the forward-parity tests.
WARM = dict(T_init=1e5)


@pytest.mark.parametrize("n,sub", [(12, True), (12, False), (64, False)])
def test_step_adjoint_matches_oracle_reverse_mode(dh, n, sub):
    p = dh.default_params(n=n, box=float(n), n_steps=4, a_start=0.1, a_end=0.3,
                          rms_ref=0.15 if n < 32 else 0.05, **(SUB if sub else WARM))
    o = oracle_params(p)
    sim = dh.Simulation(p, f32(synth.white_noise(n, 2))[0])
    sim.step()
    st0 = sim.state()
    sim.step()
    lam_gas, lg_o = f32(synth.field(n, 40, shape=(5, n, n, n)))
    lam_part, lp_o = f32(synth.field(n, 41, shape=(6, n ** 3)) * 0.1)
    dpar = torch.zeros(dh.NPARAMS, dtype=torch.float64, device="cuda")
    sim.step_adjoint(lam_gas, lam_part, dpar)
    # oracle: differentiate one step from the same float32 state (g(a_1) recomputed inside)
    a1 = osim.schedule(o)[0]["a1"]

    def oracle_grad(U0, s0, p0):
        U = U0.clone().requires_grad_(True)
        s = s0.clone().requires_grad_(True)
        pp = p0.clone().requires_grad_(True)
        om = torch.tensor(o["omega_m"], dtype=DT, requires_grad=True)
        oo = dict(o, omega_m=om)
        state = {"s": s, "p": pp, "U": U, "g": osim.force(s, U[0], oo, a1), "step": 1,
                 "star": torch.zeros(n, n, n, dtype=DT), "aux": torch.zeros(n ** 3, dtype=DT),
                 "events": []}
        out = osim.step(state, oo)
        L = (out["U"] * lg_o).sum() + (out["s"] * lp_o[:3]).sum() + (out["p"] * lp_o[3:]).sum()
        return torch.autograd.grad(L, (U, s, pp, om))

    X = (st0["gas"].double().cpu(), st0["s"].double().cpu(), st0["p"].double().cpu())
    gU, gs, gp, gom = oracle_grad(*X)
    # The reverse mode of a step has kinks (limiter gates, CIC cell edges). The float32
    # forward rounds every intermediate state (kicked gas, half step, fluxes), and where a
    # flux difference is near zero that flips a gate, so the two gradients differ in a few
    # isolated cells. The oracle's own gradient moves as much when its input moves by 1e-6
    # relative: that floor is measured here and the GPU must agree within
    # max(1e-3, 3 x floor) overall and within 1e-4 outside the 0.1 % worst cells.
    gen = torch.Generator().manual_seed(0)
    Xp = [x * (1 + 1e-6 * torch.randn(x.shape, generator=gen, dtype=DT)) for x in X]
    fU, fs, fp, _ = oracle_grad(*Xp)
    for k in range(5):
        err = rel_l2(lam_gas[k], gU[k])
        assert err < max(1e-3, 3 * rel_l2(fU[k], gU[k])), (k, err, rel_l2(fU[k], gU[k]))
        d = (lam_gas[k].double().cpu() - gU[k]).flatten()
        keep = torch.ones_like(d, dtype=torch.bool)
        keep[torch.topk(d.abs(), max(1, d.numel() // 1000)).indices] = False
        assert d[keep].norm().item() < 1e-4 * gU[k].norm().item(), (k, "outside worst cells")
    assert rel_l2(lam_part[:3], gs) < max(1e-3, 3 * rel_l2(fs, gs))
    assert rel_l2(lam_part[3:], gp) < max(1e-3, 3 * rel_l2(fp, gp))
    assert abs(dpar[0].item() - gom.item()) < 1e-3 * abs(gom.item())


@pytest.mark.parametrize("ckpt,sub", [(2, True), (5, True), (2, False)])
def test_run_adjoint_matches_oracle_reverse_mode(dh, ckpt, sub):
    n = 12
    p = dh.default_params(n=n, box=12.0, n_steps=5, ckpt_every=ckpt, a_start=0.1, a_end=0.35,
                          rms_ref=0.15, **(SUB if sub else WARM))
    o = oracle_params(p)
    wg, wo = f32(synth.white_noise(n, 5))
    tg, to = f32(0.16 * (1 + 0.2 * synth.field(n, 7)))
    sim = dh.Simulation(p, wg)
    sim.run()
    st = sim.state()
    dL = (2.0 / n ** 3) * (st["gas"][0] - tg)
    dL_dgas = torch.zeros(5, n, n, n, device="cuda")
    dL_dgas[0] = dL
    dnoise, dpar = sim.run_adjoint(dL_dgas.contiguous())
    names = ["omega_m", "sigma8", "delta_c", "Pi0", "E0", "T0_uv", "gamma_uv"]
    leaves = {k: torch.tensor(float(o[k]), dtype=DT, requires_grad=True) for k in names}
    X = wo.clone().requires_grad_(True)
    out = osim.run(X, dict(o, **leaves))
    L = osim.mse_density(out["U"], to)
    grads = torch.autograd.grad(L, [X] + [leaves[k] for k in names], allow_unused=True)
    assert rel_l2(dnoise, grads[0]) < 1e-3, rel_l2(dnoise, grads[0])
    for j, k in enumerate(names):
        want = 0.0 if grads[1 + j] is None else grads[1 + j].item()
        assert abs(dpar[j].item() - want) <= 1e-3 * abs(want) + 1e-10, (k, dpar[j].item(), want)


@pytest.mark.parametrize("n,steps,sub", [(40, 4, True), (64, 3, False)])
def test_run_adjoint_multi_tile(dh, n, steps, sub):
    """Grids spanning several sweep tiles along every axis (forward tiles of 32, adjoint
    tiles of 16 along y and z), a ragged last tile at n = 40, two checkpoint segments."""
    kw = dict(n=n, box=float(n), n_steps=steps, ckpt_every=2, a_start=0.1, a_end=0.25,
              rms_ref=0.15 if n < 48 else 0.05)
    kw.update(SUB if sub else WARM)
    p = dh.default_params(**kw)
    o = oracle_params(p)
    wg, wo = f32(synth.white_noise(n, 15))
    tg, to = f32(0.16 * (1 + 0.2 * synth.field(n, 16)))
    sim = dh.Simulation(p, wg)
    sim.run()
    st = sim.state()
    dL_dgas = torch.zeros(5, n, n, n, device="cuda")
    dL_dgas[0] = (2.0 / n ** 3) * (st["gas"][0] - tg)
    dnoise, dpar = sim.run_adjoint(dL_dgas.contiguous())
    X = wo.clone().requires_grad_(True)
    om = torch.tensor(o["omega_m"], dtype=DT, requires_grad=True)
    out = osim.run(X, dict(o, omega_m=om))
    L = osim.mse_density(out["U"], to)
    gX, gom = torch.autograd.grad(L, (X, om))
    assert rel_l2(dnoise, gX) < 1e-3, rel_l2(dnoise, gX)
    assert abs(dpar[0].item() - gom.item()) <= 1e-3 * abs(gom.item())
    sim.close()


def test_cfl_matches_oracle(dh):
    n = 16
    p = dh.default_params(n=n, box=16.0, rms_ref=0.3)
    sim = dh.Simulation(p, f32(synth.white_noise(n, 8))[0])
    st = sim.state()
    from oracle import hydro
    want = hydro.cfl_number(st["gas"].double().cpu(), sim.schedule(0)["dtau"], 1.0, p.gamma)
    assert abs(sim.cfl() / want - 1) < 1e-5


def test_graph_replay_matches_eager(dh):
    """sim_run / sim_run_adjoint captured into CUDA graphs and replayed give the same bits
    as eager execution, on the first (capturing) call and on later replays."""
    n = 24
    p = dh.default_params(n=n, box=24.0, n_steps=6, ckpt_every=4, a_start=0.1, a_end=0.4,
                          rms_ref=0.15, **SUB)
    wg, _ = f32(synth.white_noise(n, 21))
    tg, _ = f32(0.16 * (1 + 0.2 * synth.field(n, 22)))
    stream = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(stream):
        for graphs in (0, 1):
            sim = dh.Simulation(p, wg)
            assert dh.lib.sim_set_graphs(sim.h, graphs) == 0
            dnoise = torch.empty(n, n, n, device="cuda")
            dpar = torch.zeros(dh.NPARAMS, dtype=torch.float64, device="cuda")
            dL = torch.empty(5, n, n, n, device="cuda")
            loss = torch.empty(1, dtype=torch.float64, device="cuda")
            for rep in range(3):
                sim.reinit(wg)
                sim.run()
                sim.loss_density(tg, 1.0 / n ** 3, out=dL, loss=loss)
                assert dh.lib.sim_run_adjoint(sim.h, dh.api._ptr(dL), None, dh.api._ptr(dnoise),
                                              dh.api._ptr(dpar)) == 0
                stream.synchronize()
                outs.append((graphs, rep, sim.state()["gas"].clone(), dnoise.clone(), dpar.clone()))
            sim.close()
    # the forward pass is bitwise reproducible (fixed-point deposit); the reverse pass
    # scatters particle adjoints with float atomics, so its sums vary at round-off level
    ref = outs[0]
    for g, rep, gas, dn, dp in outs[1:]:
        assert torch.equal(gas, ref[2]), (g, rep)
        assert rel_l2(dn, ref[3]) < 1e-5, (g, rep)
        assert rel_l2(dp, ref[4]) < 1e-5, (g, rep)


@pytest.mark.parametrize("graphs", [0, 1])
def test_runs_record_their_last_segments(dh, graphs):
    """Once a handle holds a tape (after its first reverse pass), sim_run records its last
    checkpoint segments as it goes (sim_set_tape_recording: 1 by default, 0 none, -1 all) and
    the next sim_run_adjoint recomputes none of them: every run's state, stars, events and
    diagnostics are those of a run without the tape, the gradients agree (float atomics in
    the reverse pass: 1e-5), and the reverse pass launches fewer kernels. A tape grown for
    more segments drops what the run before recorded on the old one."""
    n = 16
    p = dh.default_params(n=n, box=16.0, n_steps=10, ckpt_every=4, a_start=0.1, a_end=0.4,
                          rms_ref=0.15, **SUB)
    wg, _ = f32(synth.white_noise(n, 23))
    tg, _ = f32(0.16 * (1 + 0.2 * synth.field(n, 24)))
    sim = dh.Simulation(p, wg)
    sim.set_graphs(bool(graphs))
    sim.set_diagnostics(True)
    runs = []
    # segments [0, 4), [4, 8), [8, 10); the recording set before each run
    for segs in (1, 1, 0, -1, -1):
        sim.set_tape_recording(segs)
        sim.reset()
        sim.run()
        st = {k: v.clone() for k, v in sim.state().items() if torch.is_tensor(v)}
        diag = [sim.diagnostics(k) for k in range(p.n_steps + 1)]
        dL, _ = sim.loss_density(tg, 1.0 / n ** 3)
        torch.cuda.synchronize()
        l0 = dh.lib.sim_kernel_launches()
        dnoise, dpar = sim.run_adjoint(dL)
        torch.cuda.synchronize()
        runs.append((st, diag, dnoise.clone(), dpar.clone(), dh.lib.sim_kernel_launches() - l0))
    ref = runs[0]
    for st, diag, dn, dp, _ in runs[1:]:
        for k in ref[0]:
            assert torch.equal(st[k], ref[0][k]), k
        assert diag == ref[1]
        assert rel_l2(dn, ref[2]) < 1e-5
        assert rel_l2(dp, ref[3]) < 1e-5
    L = [r[4] for r in runs]
    # no tape yet; last segment recorded; nothing recorded; recorded on the old tape, which
    # the adjoint then grows (recording dropped); all three segments recorded
    assert L[1] < L[0] and L[2] == L[0] and L[3] == L[0] and L[4] < L[1], L
    sim.close()
