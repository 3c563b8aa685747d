"""Batched instances (sim_init_batch), sweep-variant autotuning and handle groups on GB300.

A batch of B instances runs every kernel of the step once for all B; each instance must
evolve as a B = 1 handle with the same parameters. The forward state is compared bit for
bit (the deposit is fixed point and every kernel computes an instance exactly as a single
launch would); the reverse pass sums particle adjoints with float atomics, so gradients are
compared at round-off level.
"""
import pytest
import torch

import synth
from gpu_helpers import f32, lib, need_gpu, rel_l2

pytestmark = pytest.mark.gpu

SUB = dict(subgrid_on=1, delta_c=0.3, w_delta=0.05, T_c=1e6, w_T=1e5, Pi0=0.2, T0_uv=5e3)


@pytest.fixture(scope="module")
def dh():
    need_gpu()
    return lib()


def _params(dh, n, count, n_steps=6, **kw):
    """Instances differing in cosmology, subgrid parameters and Philox seed / instance."""
    draws = synth.uniform_params(11, count, {"omega_m": (0.27, 0.33), "sigma8": (0.75, 0.85),
                                             "delta_c": (0.2, 0.4), "Pi0": (0.1, 0.3),
                                             "T0_uv": (3e3, 8e3), "gamma_uv": (1.2, 1.6)})
    out = []
    for b, d in enumerate(draws):
        base = dict(n=n, box=float(n), n_steps=n_steps, ckpt_every=4, a_start=0.1, a_end=0.4,
                    rms_ref=0.15, seed=100 + b, instance=b)
        base.update(SUB)
        base.update(kw)
        base.update(d)
        out.append(dh.default_params(**base))
    return out


def _noise(n, B, seed=5):
    return torch.stack([f32(synth.white_noise(n, seed + b))[0] for b in range(B)])


def test_batch_forward_matches_single_instances_bitwise(dh):
    n, B = 16, 3
    ps = _params(dh, n, B)
    noise = _noise(n, B)
    bat = dh.Simulation(ps, noise.contiguous())
    bat.run()
    sb = bat.state()
    for b in range(B):
        one = dh.Simulation(ps[b], noise[b].contiguous())
        one.run()
        s1 = one.state()
        for key in ("gas", "s", "p", "star", "aux", "events"):
            assert torch.equal(sb[key][b], s1[key]), (b, key)
        one.close()
    bat.close()


def test_batch_noise_from_philox_per_instance(dh):
    """noise = NULL draws each instance's white noise from its own (seed, instance)."""
    n, B = 12, 2
    ps = _params(dh, n, B)
    bat = dh.Simulation(ps, None)
    sb = bat.state()
    for b in range(B):
        one = dh.Simulation(ps[b], None)
        assert torch.equal(sb["gas"][b], one.state()["gas"]), b
        one.close()
    assert not torch.equal(sb["gas"][0], sb["gas"][1])
    bat.close()


def test_batch_gradients_match_single_instances(dh):
    n, B = 16, 3
    ps = _params(dh, n, B)
    noise = _noise(n, B)
    tgt = torch.stack([f32(0.16 * (1 + 0.2 * synth.field(n, 30 + b)))[0] for b in range(B)])
    bat = dh.Simulation(ps, noise.contiguous())
    bat.run()
    dL, loss = bat.loss_density(tgt.contiguous(), 1.0 / n ** 3)
    dnb, dpb = bat.run_adjoint(dL)
    for b in range(B):
        one = dh.Simulation(ps[b], noise[b].contiguous())
        one.run()
        dL1, loss1 = one.loss_density(tgt[b].contiguous(), 1.0 / n ** 3)
        assert torch.equal(loss[b:b + 1], loss1) or abs(loss[b].item() - loss1.item()) < 1e-12
        dn1, dp1 = one.run_adjoint(dL1)
        assert rel_l2(dnb[b], dn1) < 1e-5, b
        assert rel_l2(dpb[b], dp1) < 1e-5, b
        one.close()
    bat.close()


def test_batch_step_adjoint_matches_single(dh):
    n, B = 12, 2
    ps = _params(dh, n, B, n_steps=3)
    noise = _noise(n, B)
    bat = dh.Simulation(ps, noise.contiguous())
    bat.step()
    lg = torch.stack([f32(synth.field(n, 40 + b, shape=(5, n, n, n)))[0] for b in range(B)])
    lp = torch.stack([f32(0.1 * synth.field(n, 50 + b, shape=(6, n ** 3)))[0] for b in range(B)])
    lgb, lpb = lg.clone(), lp.clone()
    dpb = torch.zeros(B, dh.NPARAMS, dtype=torch.float64, device="cuda")
    bat.step_adjoint(lgb, lpb, dpb)
    for b in range(B):
        one = dh.Simulation(ps[b], noise[b].contiguous())
        one.step()
        g1, p1 = lg[b].clone(), lp[b].clone()
        d1 = torch.zeros(dh.NPARAMS, dtype=torch.float64, device="cuda")
        one.step_adjoint(g1, p1, d1)
        # the reverse pass scatters particle adjoints with float atomics: round-off level
        assert rel_l2(lgb[b], g1) < 1e-5, b
        assert rel_l2(lpb[b], p1) < 1e-5, b
        assert rel_l2(dpb[b], d1) < 1e-5, b
        one.close()
    bat.close()


def test_batch_rejects_mismatched_shared_fields(dh):
    ps = _params(dh, 12, 2)
    ps[1].n_steps = ps[0].n_steps + 1
    with pytest.raises(dh.SimError):
        dh.Simulation(ps)


@pytest.mark.parametrize("n", [32, 48])
def test_autotune_and_variants_agree(dh, n):
    """Every sweep variant computes the same update; the autotuner picks one per axis."""
    B = 2
    ps = _params(dh, n, B, n_steps=3, rms_ref=0.05)
    noise = _noise(n, B)
    results = []
    for mode in ("default", "tile", "march32", "march16", "marchfit", "pair", "auto"):
        sim = dh.Simulation(ps, noise.contiguous())
        if mode == "auto":
            fwd, adj = sim.autotune(reps=2)
            assert fwd[0] == 1 and all(v in (1, 2, 3, 4, 5) for v in fwd)
            assert all(v in (1, 2, 3, 4) for v in adj)
        elif mode != "default":
            v = {"tile": 1, "march32": 2, "march16": 3, "marchfit": 4, "pair": 5}[mode]
            sim.set_sweep_variants([v] * 3, [v] * 3)
        sim.run()
        st = sim.state()
        dL = torch.zeros(B, 5, n, n, n, device="cuda")
        dL[:, 0] = st["gas"][:, 0] - st["gas"][:, 0].mean()
        dn, dp = sim.run_adjoint(dL.contiguous())
        results.append((mode, st["gas"].clone(), dn.clone(), dp.clone()))
        sim.close()
    ref = results[0]
    for mode, gas, dn, dp in results[1:]:
        assert rel_l2(gas, ref[1]) < 1e-6, mode
        assert rel_l2(dn, ref[2]) < 1e-5, mode
        assert rel_l2(dp, ref[3]) < 1e-5, mode


def test_group_of_uneven_batches(dh):
    """Two batches of different grid sizes captured as one graph: first call (capture) and
    replay after a reset give the members' own results."""
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sizes = (16, 24)
        members, solo = [], []
        for n in sizes:
            ps = _params(dh, n, 2)
            noise = _noise(n, 2, seed=7 * n)
            members.append(dh.Simulation(ps, noise.contiguous()))
            solo.append(dh.Simulation(ps, noise.contiguous()))
        grp = dh.Group(members)
        dls = []
        for m, n in zip(solo, sizes):
            m.run()
            st = m.state()
            dL = torch.zeros(2, 5, n, n, n, device="cuda")
            dL[:, 0] = st["gas"][:, 0] - 0.16
            dls.append(dL.contiguous())
        ref = [(m.state()["gas"].clone(), m.run_adjoint(dl, want_noise=False)[1].clone())
               for m, dl in zip(solo, dls)]
        for rep in range(2):
            grp.reset()
            grp.run()
            outs = grp.run_adjoint(dls)
            stream.synchronize()
            for k, m in enumerate(members):
                assert torch.equal(m.state()["gas"], ref[k][0]), (rep, k)
                assert rel_l2(outs[k], ref[k][1]) < 1e-5, (rep, k)
        grp.close()
        for m in members + solo:
            m.close()
