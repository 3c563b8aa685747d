#!/usr/bin/env python
"""Benchmark of the differentiable hydro step on GB300: cell-steps/s forward + adjoint.

One bench step is one iteration of field-level inference (Sec. 3.2) on a 128^3 grid with
128^3 dark-matter particles: initial conditions from the device-resident white-noise
amplitudes, 100 steps a = 0.05 -> 1.0 (FastPM kick-drift-kick, three relaxing-TVD sweeps,
subgrid with Gumbel-softmax, CIC + spectral Poisson), the posterior against a mock final
density, the checkpointed adjoint (checkpoint every 10 steps) back to the 2,097,152
amplitudes, and an Adam step on them (one sim_fli_step call).

value     cell-steps/s of that iteration = 128^3 * 100 / time, summed over ranks (replicas).
e2e       the same through the C ABI with the amplitudes copied from pinned host memory and
          the updated amplitudes plus the loss copied back inside the timed region.
fli       200 iterations from zero amplitudes: seconds per iteration, the loss, and r_c(k)
          of the recovered amplitudes and final density against the truth.
roofline  the dominant kernel class (hydro sweeps or their adjoints), each launch timed with
          CUDA events on the simulation stream during one eager pass of the same hot path;
          roofline.classes holds that pass's time per stage of the step and adjoint.
cpu_baseline  the FP64 oracle on the host cores on a bounded sample of the same workload.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: launched by torchrun, each rank runs an independent replica (no collective on
the data path); timing is bracketed by barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s fwd & fwd+adjoint at 128^3 FP32; HBM GB/s vs peak; err vs FP64"
WORKLOAD = dict(n=128, box=128.0, n_steps=100, a_start=0.05, a_end=1.0, ckpt_every=10,
                subgrid_on=1, delta_c=100.0, Pi0=0.05, E0=0.03, T_c=3.0e4, w_delta=5.0,
                w_T=1500.0, T0_uv=1.0e4, gamma_uv=1.4, seed=1)
WORKLOAD_NAME = ("128^3 cells + 128^3 DM particles, box 128 Mpc/h, 100 steps a=0.05->1.0, "
                 "subgrid on; one field-level-inference iteration: ICs + forward + posterior "
                 "(mock: seed-7 final density + 10% noise) + checkpointed adjoint (every 10 "
                 "steps) to the 2,097,152 white-noise amplitudes + Adam step")
# field-level inference (Sec. 3.2, the 128^3 / 100-step / checkpoint-10 workload): mock data
# from the held seed's run plus 10% noise, Adam on the amplitudes (learning rate 0.003: 0.01
# oscillates and 0.03 diverges on this workload, measured over 200 iterations)
FLI_TRUTH_SEED = 7
FLI_NOISE_FRAC = 0.1
FLI_LR = 0.003
FLI_ITERS = 200
TAPE_FLOATS_PER_CELL = 46      # floats per cell of one recorded step (six gas states, s0, p0,
                               # g0, s1, g1 and the Gumbel difference)
SWEEP_BYTES_PER_CELL = 40      # sweep: 5 float32 fields read + 5 written
SWEEP_ADJ_BYTES_PER_CELL = 60  # adjoint sweep: state and output adjoint read, input adjoint written
# DRAM bytes per cell of one launch group (dram__bytes_read.sum + dram__bytes_write.sum) from
# the ncu captures summarised in profiles/ (128^3, cold cache): forward sweep, the packed x
# tile (43.9 MB) and the paired y / z forms (44.7, 45.1 MB) averaged; adjoint sweep (x, y, z
# average of the marching pair with fitted segments, x with its input transposes and the
# second pass writing the untransposed result) (374.5 + 253.7 + 254.2) / 3 MB; None where no
# capture of the current kernel exists
TRAFFIC_BYTES_PER_CELL = {"sweep": 21.26, "sweep_adjoint": 140.25}
# the kernel forms (SWEEP_* per axis x, y, z) those captures measured
PROFILED_VARIANTS = {"sweep": [1, 5, 5], "sweep_adjoint": [4, 4, 4]}
# algorithmic bytes per cell of one timed launch group of each class (one particle per cell)
CLASS_BYTES_PER_CELL = {"sweep": SWEEP_BYTES_PER_CELL, "sweep_adjoint": SWEEP_ADJ_BYTES_PER_CELL,
                        "deposit": 28, "poisson": 16, "subgrid": 44, "subgrid_adjoint": 60}


BATCH_SIZES = (32, 48, 64)
BATCH_PER_SIZE = 32
BATCH_RANGES = {"omega_m": (0.25, 0.35), "sigma8": (0.7, 0.9), "delta_c": (50.0, 200.0),
                "Pi0": (0.01, 0.1), "T0_uv": (5.0e3, 2.0e4), "gamma_uv": (1.2, 1.6)}
BATCH_NAME = ("96 instances (32 each at 32^3, 48^3, 64^3; box n Mpc/h), per-instance "
              "Omega_m~U[0.25,0.35], sigma8~U[0.7,0.9], delta_c~U[50,200], Pi0~U[0.01,0.1], "
              "T0~U[5e3,2e4] K, gamma~U[1.2,1.6], own Philox seed; 40 steps a=0.1->1.0, "
              "subgrid on; forward + parameter gradients (checkpoint every 10)")


CLOSURE_NAME = ("learned closure (4 periodic 3x3x3 convs 5-16-16-16-5, GELU, bf16 on tcgen05): "
                "600 pairs from six 64^3 / 128^3 run pairs (100 steps a=0.1->1.0), 600 Adam "
                "iterations; applied every step of 256^3 runs (100 steps), field error against "
                "the 512^3 run restricted to 256^3")


def bench_batched(dh, synth, torch, steps: int, warmup: int):
    """Parameter-sampling form: three batched handles (one per grid size) run as one graph
    group, against the same 96 instances run one handle at a time (graphs on)."""
    draws = synth.uniform_params(2024, len(BATCH_SIZES) * BATCH_PER_SIZE, BATCH_RANGES)
    groups = []
    for k, n in enumerate(BATCH_SIZES):
        ps = []
        for b in range(BATCH_PER_SIZE):
            i = k * BATCH_PER_SIZE + b
            ps.append(dh.default_params(n=n, box=float(n), n_steps=40, a_start=0.1, a_end=1.0,
                                        ckpt_every=10, subgrid_on=1, E0=0.03, seed=1000 + i,
                                        instance=i, **draws[i]))
        groups.append(ps)
    cells = sum(n ** 3 * BATCH_PER_SIZE for n in BATCH_SIZES) * 40
    dev = torch.device("cuda", torch.cuda.current_device())

    def loss_grad(sim):
        st = sim.state()["gas"]
        dL = torch.zeros_like(st)
        dL[:, 0] = st[:, 0] - st[:, 0].mean()
        return dL.contiguous()

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.mean(ts)

    # batched: one handle per size, autotuned sweeps, one graph group
    sims = [dh.Simulation(ps) for ps in groups]
    variants = [sim.autotune(reps=3) for sim in sims]
    for sim in sims:
        sim.run()
    dls = [loss_grad(sim) for sim in sims]
    outs = [torch.zeros(BATCH_PER_SIZE, dh.NPARAMS, dtype=torch.float64, device=dev) for _ in sims]
    cfl = max(sim.cfl() for sim in sims)
    for sim in sims:
        sim.reset()
    grp = dh.Group(sims)

    def batched_pass():
        grp.reset()
        grp.run()
        grp.run_adjoint(dls, out=outs)

    for _ in range(warmup):
        batched_pass()
    ms_b = timed(batched_pass, steps)
    launches0 = dh.lib.sim_kernel_launches()
    batched_pass()
    torch.cuda.synchronize()
    launches_b = dh.lib.sim_kernel_launches() - launches0
    grp.close()
    for sim in sims:
        sim.close()
    # the same instances one handle at a time
    solo = []
    for ps, dl in zip(groups, dls):
        for b, p in enumerate(ps):
            sim = dh.Simulation(p)
            sim.set_graphs(True)
            solo.append((sim, dl[b].contiguous(),
                         torch.zeros(dh.NPARAMS, dtype=torch.float64, device=dev)))

    def solo_pass():
        for sim, dl, out in solo:
            sim.reset()
            sim.run()
            dh._lib.check(dh.lib.sim_run_adjoint(sim.h, dh.api._ptr(dl), None, None,
                                                 dh.api._ptr(out)), "sim_run_adjoint", sim.h)

    for _ in range(warmup):
        solo_pass()
    ms_s = timed(solo_pass, steps)
    # agreement of the parameter gradients of the two forms (same instances, same inputs)
    worst = 0.0
    idx = 0
    for k in range(len(BATCH_SIZES)):
        for b in range(BATCH_PER_SIZE):
            ref = solo[idx][2]
            worst = max(worst, ((outs[k][b] - ref).norm() / ref.norm().clamp_min(1e-300)).item())
            idx += 1
    for sim, _, _ in solo:
        sim.close()
    return {"workload": BATCH_NAME, "value": cells / (ms_b / 1e3), "unit": "cell-steps/s",
            "ms_per_pass": ms_b, "solo_value": cells / (ms_s / 1e3), "solo_ms_per_pass": ms_s,
            "speedup_vs_solo": ms_s / ms_b, "gpu_launches_per_pass": int(launches_b),
            "max_cfl": cfl, "grad_rel_diff_vs_solo": worst,
            "sweep_variants": {str(n): {"fwd": v[0], "adj": v[1]}
                               for n, v in zip(BATCH_SIZES, variants)}}


def bench_256(dh, synth, torch, peak_bw: float, steps: int = 2):
    """The same iteration (ICs, 100-step run, posterior, checkpointed reverse pass, Adam) at
    256^3 cells + 256^3 particles in a 256 Mpc/h box, where the state (335 MB of gas) no
    longer fits in L2: forward and forward + adjoint rates, and the sweep classes of one
    eager pass against the HBM copy peak."""
    n = 256
    p = dh.default_params(**dict(WORKLOAD, n=n, box=float(n)))
    n3 = n ** 3
    dev = torch.device("cuda", torch.cuda.current_device())
    noise = torch.from_numpy(synth.white_noise(n, 100).astype("float32")).to(dev)
    sim = dh.Simulation(p, noise)
    variants = sim.autotune(reps=2)
    sim.set_graphs(True)
    sim.run()
    data = sim.state()["gas"][0].clone()
    sigma_n = FLI_NOISE_FRAC * data.std().item()
    x = noise.clone()
    mom = torch.zeros_like(x)
    vel = torch.zeros_like(x)
    loss = torch.empty(1, dtype=torch.float64, device=dev)

    def it():
        x.copy_(noise)
        sim.fli_step(x, mom, vel, data, sigma_n, FLI_LR, 1, loss=loss)

    def timed(fn):
        ts = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.mean(ts)

    it()
    ms = timed(it)
    sim.set_tape_recording(0)

    def fwd():
        sim.reinit(noise)
        sim.run()

    fwd()
    fwd_ms = timed(fwd)
    sim.set_tape_recording(1)
    sim.kernel_timing(True)
    sim.kernel_times(reset=True)
    it()
    torch.cuda.synchronize()
    kt = sim.kernel_times(reset=True)
    sim.kernel_timing(False)
    sim.close()
    classes = {}
    for name in ("sweep", "sweep_adjoint"):
        tot, cnt = kt[name]
        avg = tot / max(cnt, 1)
        gbs = CLASS_BYTES_PER_CELL[name] * n3 / (avg * 1e-3) / 1e9
        classes[name] = {"launches": cnt, "avg_launch_ms": avg, "achieved_gbs": gbs,
                         "frac_of_peak": gbs / peak_bw}
    return {"workload": "as the headline at 256^3 cells + 256^3 particles, box 256 Mpc/h",
            "value": n3 * p.n_steps / (ms * 1e-3), "ms_per_step": ms,
            "fwd_value": n3 * p.n_steps / (fwd_ms * 1e-3), "fwd_ms_per_step": fwd_ms,
            "unit": "cell-steps/s", "sweep_variants": {"fwd": variants[0], "adj": variants[1]},
            "classes": classes}


def bench_lbfgs(dh, synth, torch, sim, truth, p, iters: int):
    """Sec. 3.2 as the paper runs it: subgrid off, the delta_b T probe (internal energy
    density), pixel noise of variance 1x (S/N = 1) and 5x (S/N = 5) the data variance,
    L-BFGS with M = 8 from zero amplitudes; r_c(k) of the recovered amplitudes."""
    from paper_2502_02294_gb300.inference import fli_lbfgs
    n = p.n
    q = dh.SimParams.from_buffer_copy(p)
    q.subgrid_on = 0
    q.a_end = 0.25          # the paper evolves its field-level-inference box to z = 3
    s2 = dh.Simulation(q, truth)
    s2.set_graphs(True)
    s2.run()
    g = s2.state()["gas"]
    u = (g[4] - 0.5 * (g[1] ** 2 + g[2] ** 2 + g[3] ** 2) / g[0]).contiguous()
    out = {"workload": "128^3, 100 steps a=0.05->0.25 (z = 3), subgrid off; data = internal energy "
                       "density of the seed-%d run + Gaussian pixel noise; L-BFGS M=8 from "
                       "zero amplitudes, at most %d iterations" % (FLI_TRUTH_SEED, iters)}
    nb = n // 2
    for snr in (1.0, 5.0):
        sig = float(snr ** 0.5 * u.std().item())
        data = (u + sig * torch.from_numpy(synth.field(n, 900 + int(snr)).astype("float32")).to(u.device)).contiguous()
        t0 = time.time()
        r = fli_lbfgs(s2, data, sig, torch.zeros_like(truth), dh.OBS_THERMAL, max_iter=iters)
        torch.cuda.synchronize()
        dt = time.time() - t0
        kk, rc, _ = dh.cross_correlation(r.x.contiguous(), truth, p.box, nb)
        pick = [0, 1, 3, 7, 15, 31, nb - 1]
        out[f"snr_{int(snr)}"] = {
            "iterations": r.iterations, "evaluations": r.evaluations, "seconds": dt,
            "seconds_per_evaluation": dt / max(r.evaluations, 1), "converged": r.converged,
            "loss_first": r.history[0][1], "loss_last": r.history[-1][1],
            "k": [float(kk[j]) for j in pick], "r_c": [float(rc[j]) for j in pick]}
    s2.close()
    return out


def _config(ws: int):
    return {"workload": WORKLOAD_NAME, "n": WORKLOAD["n"], "n_steps": WORKLOAD["n_steps"],
            "ckpt_every": WORKLOAD["ckpt_every"], "parallelism": f"replicas x{ws}",
            "l2": "512 MB buffer written between timed iterations"}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(vals, ws):
    """Entry-wise maximum of a tensor over the ranks of the default process group (the
    slowest rank's times); the tensor itself for one rank."""
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(vals, op=dist.ReduceOp.MAX)
    return vals.tolist()


def job_throughput(cells_per_rank, ws, ms):
    """Whole-job cell-steps/s: every rank's cells over the slowest rank's time (weak scaling:
    each rank runs its own replica of the workload)."""
    return cells_per_rank * ws / (ms / 1e3)


def nvsmi_id(dev: int) -> str:
    """nvidia-smi --id of CUDA device `dev`: its UUID (nvidia-smi's own indices need not
    follow CUDA_VISIBLE_DEVICES), else the CUDA ordinal."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(dev).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    return str(dev)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * (max(mx) if mx else 1)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline_sample(steps: int = 1):
    """The oracle (FP64, torch CPU, autograd) on `steps` full steps of the 128^3 workload,
    forward + reverse; returns (cell-steps/s, seconds, threads)."""
    import torch
    from oracle import sim as osim

    prm = dict(osim.Params().as_dict(), **WORKLOAD)
    n = prm["n"]
    noise = torch.randn(n, n, n, dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    st = osim.init_state(noise, prm)
    sched = osim.schedule(prm)
    U = st["U"].detach().clone().requires_grad_(True)
    st["U"] = U
    t0 = time.perf_counter()
    cur = st
    for _ in range(steps):
        cur = osim.step(cur, prm, sched)
    L = (cur["U"][0] ** 2).sum()
    L.backward()
    dt = time.perf_counter() - t0
    return n ** 3 * steps / dt, dt, torch.get_num_threads()


def cpu_forward_sample(steps: int, threads: int | None = None):
    """The oracle's forward alone (no tape) on `steps` steps of the 128^3 workload with
    `threads` host threads (None: torch's default, all cores); returns (cell-steps/s,
    seconds, threads used)."""
    import torch
    from oracle import sim as osim

    prev = torch.get_num_threads()
    if threads:
        torch.set_num_threads(threads)
    try:
        prm = dict(osim.Params().as_dict(), **WORKLOAD)
        n = prm["n"]
        noise = torch.randn(n, n, n, dtype=torch.float64, generator=torch.Generator().manual_seed(1))
        with torch.no_grad():
            st = osim.init_state(noise, prm)
            sched = osim.schedule(prm)
            t0 = time.perf_counter()
            for _ in range(steps):
                st = osim.step(st, prm, sched)
            dt = time.perf_counter() - t0
        return n ** 3 * steps / dt, dt, torch.get_num_threads()
    finally:
        torch.set_num_threads(prev)


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, same metric and unit."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline_sample(1)
    times = []
    for _ in range(args.steps):
        v, dt, threads = cpu_baseline_sample(1)
        times.append(dt)
    ms = 1e3 * statistics.mean(times)
    n3 = WORKLOAD["n"] ** 3
    value = n3 / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": _config(args.gpus),
            "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": threads,
                             "kind": "oracle",
                             "sample": "1 step fwd+reverse at 128^3 per bench step"},
            "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fli", action="store_true",
                    help="skip the field-level-inference record (Adam iterations from zero)")
    ap.add_argument("--fli-iters", type=int, default=FLI_ITERS)
    ap.add_argument("--lbfgs-iters", type=int, default=40)
    ap.add_argument("--no-experiments", action="store_true",
                    help="skip the Sedov, convergence and P(k)-likelihood HMC records")
    ap.add_argument("--cpu-full-forward", action="store_true",
                    help="also time the oracle's whole 128^3 x 100-step forward run (minutes)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched parameter-sampling measurement")
    ap.add_argument("--no-closure", action="store_true",
                    help="skip the learned-closure training and 256^3 application")
    ap.add_argument("--sweep-variants", default=None,
                    help="x,y,z forward and x,y,z adjoint sweep forms (SWEEP_* codes, six "
                         "comma-separated) instead of the autotuner's choice, e.g. for a "
                         "profiler run, under which the autotuner's timings are distorted")
    ap.add_argument("--no-256", action="store_true",
                    help="skip the same iteration at 256^3")
    ap.add_argument("--no-full-tape", action="store_true",
                    help="skip the variant that records every segment's tape during the run")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel eagerly instead of replaying captured graphs")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import __graft_entry__

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    __graft_entry__.build()
    import paper_2502_02294_gb300 as dh
    import synth

    dev = torch.device("cuda", local)
    p = dh.default_params(**WORKLOAD)
    p.seed = WORKLOAD["seed"] + rank
    n = p.n
    n3 = n ** 3
    noise = torch.from_numpy(synth.white_noise(n, 100 + rank).astype("float32")).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # the simulation runs on its own stream so that its runs can be captured as CUDA graphs
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    torch.cuda.set_stream(stream)
    sim = dh.Simulation(p, noise)
    # the library's autotuner picks the sweep kernels for this grid (timed on the ICs)
    if args.sweep_variants:
        v = [int(t) for t in args.sweep_variants.split(",")]
        if len(v) != 6:
            raise SystemExit("--sweep-variants takes six comma-separated codes")
        sim.set_sweep_variants(v[:3], v[3:])
        variants = (v[:3], v[3:])
    else:
        variants = sim.autotune(reps=3)
    if not args.no_graphs:
        dh._lib.check(dh.lib.sim_set_graphs(sim.h, 1), "sim_set_graphs", sim.h)
    # the field-level-inference mock (Sec. 3.2): the final gas density of the run from the
    # held seed's amplitudes plus Gaussian noise at 10% of the field's rms
    truth = torch.from_numpy(synth.white_noise(n, FLI_TRUTH_SEED).astype("float32")).to(dev)
    sim.reinit(truth)
    sim.run()
    rho_true = sim.state()["gas"][0].clone()
    sigma_n = FLI_NOISE_FRAC * rho_true.std().item()
    data = (rho_true + sigma_n * torch.from_numpy(
        synth.field(n, FLI_TRUTH_SEED + 1).astype("float32")).to(dev)).contiguous()
    # one step of the hot path = one inference iteration on the n^3 amplitudes: ICs, the
    # 100-step run, posterior, checkpointed reverse pass, Adam update. Every timed step is
    # the first iteration from the same amplitudes (Adam's moments start from zero), so each
    # times the same work.
    x = noise.clone()
    mom = torch.zeros_like(x)
    vel = torch.zeros_like(x)
    loss = torch.empty(1, dtype=torch.float64, device=dev)

    def hot_path(x_dev):
        # step t = 1: the library starts the moments from zero (their contents are not read)
        sim.fli_step(x_dev, mom, vel, data, sigma_n, FLI_LR, 1, loss=loss)
        return x_dev, loss

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        x.copy_(noise)
        hot_path(x)
    # ---- device-resident timing (value)
    clocks = Clocks(nvsmi_id(torch.cuda.current_device()))
    clocks.start()
    launches0 = dh.lib.sim_kernel_launches()
    times = []
    barrier()
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        flush.zero_()
        x.copy_(noise)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hot_path(x)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = dh.lib.sim_kernel_launches() - launches0
    clk = clocks.stop()
    ms = statistics.mean(times)
    # ---- forward-only timing (runs that record no tape for a reverse pass)
    sim.set_tape_recording(0)
    sim.reinit(noise)
    sim.run()  # untimed: captures this form's graph
    fwd_times = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.reinit(noise)
        sim.run()
        e1.record(stream)
        e1.synchronize()
        fwd_times.append(e0.elapsed_time(e1))
    fwd_ms = statistics.mean(fwd_times)
    sim.set_tape_recording(1)
    # ---- end to end through host buffers
    host_x = noise.cpu().pin_memory()
    host_out = torch.empty_like(host_x).pin_memory()
    host_loss = torch.empty(1, dtype=torch.float64).pin_memory()
    dev_x = torch.empty_like(x)
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dev_x.copy_(host_x, non_blocking=True)
        xo, lo = hot_path(dev_x)
        host_out.copy_(xo, non_blocking=True)
        host_loss.copy_(lo, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = statistics.mean(e2e_times)
    # ---- kernel classes inside one pass: the same hot path run eagerly with every sweep
    # launch bracketed by CUDA events on the simulation's stream
    sim.kernel_timing(True)
    sim.kernel_times(reset=True)
    flush.zero_()
    x.copy_(noise)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hot_path(x)
    e1.record(stream)
    e1.synchronize()
    inst_ms = e0.elapsed_time(e1)
    kt = sim.kernel_times(reset=True)
    sim.kernel_timing(False)
    kclass = {}
    for name, (tot, cnt) in kt.items():
        avg = tot / max(cnt, 1)
        bpc = CLASS_BYTES_PER_CELL.get(name)
        kclass[name] = {"launches": cnt, "total_ms": tot, "share_of_pass": tot / inst_ms,
                        "avg_launch_ms": avg,
                        "achieved_gbs": (bpc * n3 / (avg * 1e-3) / 1e9) if (cnt and bpc) else None}
    dom = max(("sweep", "sweep_adjoint"), key=lambda k: kclass[k]["total_ms"])

    # ---- the same iteration with every checkpoint segment recorded during the run (a tape
    # of all 100 steps, no recompute in the reverse pass): a variant that spends HBM instead
    # of recomputation, reported beside the checkpointed headline
    full_tape = None
    if not args.no_full_tape:
        sim.set_tape_recording(-1)
        for _ in range(2):  # the first one grows the tape
            x.copy_(noise)
            hot_path(x)
        ft = []
        for _ in range(args.steps):
            flush.zero_()
            x.copy_(noise)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hot_path(x)
            e1.record(stream)
            e1.synchronize()
            ft.append(e0.elapsed_time(e1))
        ft_ms = statistics.mean(ft)
        full_tape = {"ms_per_step": ft_ms, "value": n3 * p.n_steps / (ft_ms * 1e-3),
                     "unit": "cell-steps/s",
                     "tape_gb": TAPE_FLOATS_PER_CELL * 4 * n3 * p.n_steps / 1e9,
                     "note": "every segment recorded during the run, no recompute"}
        sim.set_tape_recording(1)

    # ---- field-level inference: FLI_ITERS Adam iterations from zero amplitudes
    fli = None
    if not args.no_fli:
        xs = torch.zeros_like(x)
        fm = torch.zeros_like(x)
        fv = torch.zeros_like(x)
        floss = torch.empty(args.fli_iters, 1, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(1, args.fli_iters + 1):
            sim.fli_step(xs, fm, fv, data, sigma_n, FLI_LR, t, loss=floss[t - 1])
        e1.record(stream)
        e1.synchronize()
        fli_ms = e0.elapsed_time(e1)
        sim.reinit(xs)
        sim.run()
        rho_fit = sim.state()["gas"][0].contiguous()
        nb = n // 2
        kk, rc_ic, _ = dh.cross_correlation(xs, truth, p.box, nb)
        _, rc_fin, _ = dh.cross_correlation(rho_fit, rho_true.contiguous(), p.box, nb)
        fl = floss[:, 0].cpu().numpy()
        pick = [0, 1, 3, 7, 15, 31, nb - 1]
        fli = {"iterations": args.fli_iters, "seconds_per_iteration": fli_ms / 1e3 / args.fli_iters,
               "lr": FLI_LR, "sigma_n": sigma_n, "noise_frac_of_rms": FLI_NOISE_FRAC,
               "loss_first": float(fl[0]), "loss_last": float(fl[-1]),
               "loss_expected_at_truth": 0.5 * 2 * n3,
               "k": [float(kk[j]) for j in pick],
               "r_c_initial_amplitudes": [float(rc_ic[j]) for j in pick],
               "r_c_final_density": [float(rc_fin[j]) for j in pick],
               "workload": "Adam on the 2,097,152 white-noise amplitudes from zero; mock = final "
                           "gas density of seed %d plus N(0, (0.1 rms)^2); 100 steps "
                           "a=0.05->1.0, checkpoint every 10" % FLI_TRUTH_SEED}

    # ---- L-BFGS field-level inference on the delta_b T probe at S/N 1 and 5 (Sec. 3.2)
    lbfgs_rec = None
    if not args.no_fli:
        lbfgs_rec = bench_lbfgs(dh, synth, torch, sim, truth, p, args.lbfgs_iters)
    # ---- Sec. 3.1 parameter inference and Sec. 2.3.4 validation runs
    extra = {}
    if not args.no_experiments:
        from paper_2502_02294_gb300 import inference, validation
        torch.cuda.set_stream(torch.cuda.default_stream())
        extra["sedov"] = validation.sedov(dh, n=128, r_target=20.0)
        extra["convergence"] = validation.convergence(dh, n=64, box=8.0, n_steps=60)
        extra["pk_hmc"] = inference.pk_hmc_experiment(dh)
        torch.cuda.set_stream(stream)

    # ---- the same iteration at 256^3 (state beyond L2)
    run256 = None
    if not args.no_256 and ws == 1:
        pk = _peaks()
        torch.cuda.set_stream(torch.cuda.default_stream())
        run256 = bench_256(dh, synth, torch, pk["hbm_gbs"] if pk else 6800.0)
        torch.cuda.set_stream(stream)

    # ---- batched parameter-sampling form (96 instances on three grid sizes)
    batched = None
    if not args.no_batched:
        torch.cuda.set_stream(torch.cuda.default_stream())
        batched = bench_batched(dh, synth, torch, steps=2, warmup=1)
        torch.cuda.set_stream(stream)

    # ---- learned closure: trained on 64^3 / 128^3 pairs, applied in 256^3 runs
    closure = None
    if not args.no_closure:
        from paper_2502_02294_gb300 import learned
        torch.cuda.set_stream(torch.cuda.default_stream())
        closure = learned.experiment()
        closure["workload"] = CLOSURE_NAME
        torch.cuda.set_stream(stream)

    # ---- max over ranks
    vals = torch.tensor([ms, fwd_ms, e2e_ms], dtype=torch.float64, device=dev)
    ms, fwd_ms, e2e_ms = max_over_ranks(vals, ws)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    peaks = _peaks()
    peak_bw = peaks["hbm_gbs"] if peaks else 6800.0
    line = {
        "metric": METRIC,
        "value": job_throughput(n3 * p.n_steps, ws, ms),
        "unit": "cell-steps/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": _config(ws),
        "cuda_graphs": not args.no_graphs,
        "sweep_variants": {"fwd": variants[0], "adj": variants[1]},
        "fwd_value": job_throughput(n3 * p.n_steps, ws, fwd_ms),
        "fwd_ms_per_step": fwd_ms,
        "e2e": {"value": job_throughput(n3 * p.n_steps, ws, e2e_ms), "unit": "cell-steps/s",
                "h2d_bytes_per_step": n3 * 4, "d2h_bytes_per_step": n3 * 4 + 8},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": kclass[dom]["achieved_gbs"], "peak": peak_bw,
                     "unit": "GB/s", "frac": kclass[dom]["achieved_gbs"] / peak_bw,
                     "traffic": (TRAFFIC_BYTES_PER_CELL[dom] * n3
                                 if TRAFFIC_BYTES_PER_CELL[dom] is not None and
                                 list(variants[0 if dom == "sweep" else 1]) == PROFILED_VARIANTS[dom]
                                 else None),
                     "kernel": {"sweep": "hydro sweep (x, y, z average)",
                                "sweep_adjoint": "adjoint hydro sweep (x, y, z average)"}[dom],
                     "algorithmic_bytes_per_launch":
                         (SWEEP_BYTES_PER_CELL if dom == "sweep" else SWEEP_ADJ_BYTES_PER_CELL) * n3,
                     "launch_ms": kclass[dom]["avg_launch_ms"],
                     "timed_in": "one eager pass of the hot path, CUDA events around every "
                                 "launch on the simulation stream (%.1f ms pass)" % inst_ms,
                     "classes": kclass,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks
                     else "fallback 6.8 TB/s (of fallback)"},
        "clocks": clk,
    }
    if full_tape is not None:
        line["fli_full_tape"] = full_tape
    if run256 is not None:
        line["run_256"] = run256
    if fli is not None:
        line["fli"] = fli
    if lbfgs_rec is not None:
        line["fli_lbfgs"] = lbfgs_rec
    line.update(extra)
    if batched is not None:
        line["batched"] = batched
    if closure is not None:
        line["closure"] = closure
    if not args.no_cpu_baseline:
        v, dt, threads = cpu_baseline_sample(1)
        fa, fdt, fth = cpu_forward_sample(2)
        f1, f1dt, _ = cpu_forward_sample(1, threads=1)
        line["cpu_baseline"] = {"value": v, "unit": "cell-steps/s", "cores": threads,
                                "kind": "oracle",
                                "sample": f"1 full step fwd+reverse at 128^3 ({dt:.1f} s)",
                                "forward_all_cores": {"value": fa, "cores": fth,
                                                      "sample": f"2 steps at 128^3 ({fdt:.1f} s)"},
                                "forward_one_core": {"value": f1, "cores": 1,
                                                     "sample": f"1 step at 128^3 ({f1dt:.1f} s)"}}
        if args.cpu_full_forward:
            ff, ffdt, ffth = cpu_forward_sample(WORKLOAD["n_steps"])
            line["cpu_baseline"]["forward_full_run"] = {
                "value": ff, "cores": ffth, "seconds": ffdt,
                "sample": "the whole 128^3 x 100-step forward run"}
    print(json.dumps(line), flush=True)
    sim.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
