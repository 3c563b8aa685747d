"""Failure detection on the GPU without a GPU fault: each failure is made on the host
(an input the library must reject or flag) or by a device wait that is given no time.

* CFL watchdog: sim_run with cfl_max far below the run's CFL number stops with SIM_ECFL
  after the first step and names the step; the device stays usable.
* Non-finite state: a NaN or an infinity written into one gas cell (host input, gravity
  off so that no particle position is derived from it) is reported by sim_cfl as NaN and
  stops sim_run with SIM_ENAN.
* Tensor-core waits: the closure's pipeline waits given a zero time limit give up at once;
  the launch records SIM_ETIMEOUT, drains its own copies and MMAs, frees its tensor memory
  and returns, and the next launch with the default limit gives the same result as before.
"""
import math

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import f32, lib, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dh():
    need_gpu()
    return lib()


def test_cfl_watchdog_stops_the_run(dh):
    n = 16
    p = dh.default_params(n=n, box=16.0, n_steps=6, a_start=0.1, a_end=0.4, rms_ref=0.2,
                          cfl_max=1e-6)
    sim = dh.Simulation(p, f32(synth.white_noise(n, 3))[0])
    with pytest.raises(dh.SimError) as e:
        sim.run()
    assert e.value.status == dh.SIM_ECFL
    assert "after step 1" in str(e.value)
    sim.close()
    # the same run with a generous limit completes
    p.cfl_max = 10.0
    sim = dh.Simulation(p, f32(synth.white_noise(n, 3))[0])
    sim.run()
    assert 0 < sim.cfl() < 10.0
    sim.close()


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_gas_is_reported(dh, bad):
    n = 16
    p = dh.default_params(n=n, box=16.0, n_steps=4, a_start=0.1, a_end=0.3, rms_ref=0.1,
                          gravity_on=0, cfl_max=10.0)
    sim = dh.Simulation(p, f32(synth.white_noise(n, 4))[0])
    st = sim.state()
    assert math.isfinite(sim.cfl())
    gas = st["gas"].cpu().numpy().copy()
    part = torch.cat([st["s"], st["p"]]).cpu().numpy()
    gas[4, 3, 5, 7] = bad                     # one energy value, written on the host
    sim.set_state(f32(gas)[0], f32(part)[0], 0)
    assert math.isnan(sim.cfl())
    with pytest.raises(dh.SimError) as e:
        sim.run()
    assert e.value.status == dh.SIM_ENAN
    sim.close()


def test_closure_wait_timeout_is_reported_and_recoverable(dh):
    from oracle import closure as oc
    n = 32
    c = dh.Closure(oc.he_init(5))
    c.set_norm([0.15, 0, 0, 0, 1.5e-4], [0.05, 0.01, 0.01, 0.01, 5e-5],
               [0.01, 0.002, 0.002, 0.002, 0.003])
    g0 = f32(synth.gas_state(n, 9))[0]
    ref = c.forward(g0)
    c.status()
    c.set_wait_limit(0)
    out = c.forward(g0)
    with pytest.raises(dh.SimError) as e:
        c.status()
    assert e.value.status == dh.SIM_ETIMEOUT
    c.status()                                # the report was cleared
    c.set_wait_limit(1_000_000_000)
    again = c.forward(g0)
    c.status()
    assert torch.equal(again, ref)
    with pytest.raises(dh.SimError):
        c.set_wait_limit(-1)
    c.close()
    del out
