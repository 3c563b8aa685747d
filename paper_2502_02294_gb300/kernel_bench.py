"""Per-entry timings of the library's single-kernel entry points on an evolved state.

    python -m paper_2502_02294_gb300.kernel_bench [--n 128] [--steps 10] [--reps 10]
                                                  [--only sweep,sweep_adjoint,...] [--variant V]

Creates a simulation with the 128^3 benchmark settings (box = n Mpc/h, 100 steps
a = 0.05 -> 1.0, subgrid on), advances it `--steps` steps so that the fields have
structure, then times each entry with CUDA events on the current stream. A 512 MB buffer
is written before every repetition, so each launch starts with a cold L2. One line per
entry: average time and algorithmic GB/s (bytes an ideal single pass moves, stated per
entry below). With `--reps 1 --warmup 0` it is also the small case for profiler captures.
"""
from __future__ import annotations

import argparse
import statistics

import numpy as np
import torch

from . import api
from ._lib import CLOSURE_NWEIGHTS, default_params

# algorithmic bytes per cell (one particle per cell) of one call
BYTES_PER_CELL = {
    "sweep": 40,           # 5 float32 fields read + 5 written
    "sweep_adjoint": 60,   # state + output adjoint read, input adjoint written
    "deposit_cic": 16,     # 3 displacement floats read, 1 density float written
    "interp_cic": 36,      # 3 mesh fields + 3 displacements read, 3 values written
    "gravity": 16,         # density contrast read, 3 force components written
    "subgrid": 44,         # 5 fields read + written in place, star indicator written
    "closure_apply": 296,  # pack (20 + 32), 4 layers x (32 in + 32 out), gas 40 read+write
    "step_adjoint": None,  # one step's reverse pass (recompute + every adjoint kernel): time only
}
# useful closure flops per voxel: 2 x 27 x (5 x 16 + 16 x 16 + 16 x 16 + 16 x 5)
CLOSURE_FLOPS = 2 * 27 * (5 * 16 + 16 * 16 + 16 * 16 + 16 * 5)
BENCH = dict(n_steps=100, a_start=0.05, a_end=1.0, ckpt_every=10, subgrid_on=1,
             delta_c=100.0, Pi0=0.05, E0=0.03, T_c=3.0e4, w_delta=5.0, w_T=1500.0,
             T0_uv=1.0e4, gamma_uv=1.4, seed=1)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--only", default=",".join(k for k in BYTES_PER_CELL if k != "step_adjoint"))
    ap.add_argument("--variant", type=int, default=0,
                    help="sweep kernel form (SWEEP_*; 0 = the built-in choice)")
    args = ap.parse_args(argv)
    only = args.only.split(",")
    n = args.n
    n3 = n ** 3
    p = default_params(n=n, box=float(n), **BENCH)
    sim = api.Simulation(p)
    sim.run(args.steps)
    st = sim.state()
    gas, s = st["gas"], st["s"].contiguous()
    sch = sim.schedule(args.steps)
    nu = sch["dtau"] * n / p.box
    lam = torch.randn(5, n, n, n, device=gas.device, generator=torch.Generator(gas.device).manual_seed(3))
    delta = (gas[0] / gas[0].mean() - 1).contiguous()
    g = api.gravity(delta, p.box, sch["pref1"])
    gsub = gas.clone()
    gcl = gas.clone()
    clo = api.Closure(np.random.default_rng(0).standard_normal(CLOSURE_NWEIGHTS).astype(np.float32) * 0.05)
    clo.set_norm([0.15, 0, 0, 0, 1e-3], [0.05, 0.01, 0.01, 0.01, 1e-3], [1e-4] * 5)
    grid = torch.zeros(n, n, n, dtype=torch.float32, device=gas.device)
    # one more step, whose reverse pass the step_adjoint entry repeats from fixed adjoints
    sa = None
    if "step_adjoint" in only:
        sa = api.Simulation(p)
        sa.run(args.steps)
        sa.step()
        gen = torch.Generator(gas.device).manual_seed(4)
        lg0 = torch.randn(5, n, n, n, device=gas.device, generator=gen)
        lp0 = torch.randn(6, n ** 3, device=gas.device, generator=gen)
        lg, lp = lg0.clone(), lp0.clone()

        def step_adjoint():
            lg.copy_(lg0)
            lp.copy_(lp0)
            sa.step_adjoint(lg, lp)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=gas.device)

    entries = {
        "sweep": [(f"sweep axis {ax}", (lambda ax=ax: api.sweep(gas, ax, nu, p.gamma, variant=args.variant))) for ax in range(3)],
        "sweep_adjoint": [(f"sweep_adjoint axis {ax}",
                           (lambda ax=ax: api.sweep_adjoint(gas, lam, ax, nu, p.gamma,
                                                             variant=args.variant))) for ax in range(3)],
        "deposit_cic": [("deposit_cic (accumulating)", lambda: api.deposit_cic(s, n, p.box, grid=grid))],
        "interp_cic": [("interp_cic (3 fields)", lambda: api.interp_cic(g, s, n, p.box))],
        "gravity": [("gravity (r2c, Green, 3 c2r)", lambda: api.gravity(delta, p.box, sch["pref1"]))],
        "subgrid": [("subgrid (in place)", lambda: api.subgrid(gsub, sch["a1"], p, args.steps))],
        "closure_apply": [("closure apply (4 tcgen05 convs)", lambda: clo.apply(gcl))],
        "step_adjoint": [("step adjoint (incl. recompute)", lambda: step_adjoint())],
    }
    for key in only:
        for label, fn in entries[key]:
            for _ in range(args.warmup):
                fn()
            ts = []
            for _ in range(args.reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            if BYTES_PER_CELL[key] is None:
                print(f"{label:32s} n={n:4d} {1e3 * ms:9.1f} us", flush=True)
                continue
            gbs = BYTES_PER_CELL[key] * n3 / (ms * 1e-3) / 1e9
            extra = ""
            if key == "closure_apply":
                extra = f" {CLOSURE_FLOPS * n3 / (ms * 1e-3) / 1e12:7.1f} TFLOP/s useful"
            print(f"{label:32s} n={n:4d} {1e3 * ms:9.1f} us {gbs:8.0f} GB/s algorithmic{extra}",
                  flush=True)
    clo.close()
    sim.close()
    if sa is not None:
        sa.close()


if __name__ == "__main__":
    main()
