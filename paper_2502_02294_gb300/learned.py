"""Training and evaluation of the learned closure (solver in the loop, Sec. 4) with the
library's own kernels: the solver makes the training pairs, the tensor-core convolutions
and their backward pass train the network, and the trained network runs inside the
solver's step.

Training pairs (one per step of a fine run): the fine run (grid 2n, same box, the coarse
run's linear field -- band-limited noise refinement, spectrum cutoff at the same physical
k) is restricted to the coarse grid at step t (tent-weighted gas, particles of the even
lattice sites), the coarse solver advances that state one step, and the pair is
(coarse result, restricted fine state at step t + 1). The network learns the per-step
correction u <- u + s NN((u - mu) / sigma) with mu, sigma the per-field mean and spread
of the inputs and s the per-field rms of the corrections.

    python -m paper_2502_02294_gb300.learned [--n 64] [--seeds 6] [--run-steps 100]
        [--iters 600] [--eval-n 256]

prints one JSON line: training time and loss, and the field error of the coarse solver
with and without the network against the restricted fine run, with the cost of each.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import api
from ._lib import SimParams, default_params


def fine_params(p: SimParams) -> SimParams:
    """The same run on a grid twice as fine: same box, the spectrum cutoff at the same
    physical wavenumber (kc_frac is relative to the grid's Nyquist frequency)."""
    q = SimParams.from_buffer_copy(p)
    q.n = 2 * p.n
    q.kc_frac = 0.5 * p.kc_frac
    return q


def white_noise(n: int, seed: int, device="cuda"):
    g = torch.Generator(device=device).manual_seed(seed)
    return torch.randn(n, n, n, generator=g, device=device, dtype=torch.float32)


def paired_sims(p: SimParams, noise):
    """(coarse, fine) simulations sharing the linear field of `noise` (coarse grid)."""
    coarse = api.Simulation(p, noise)
    fine = api.Simulation(fine_params(p))
    scale = coarse.ic_amplitude() / fine.ic_amplitude()
    fine.reinit(api.refine_noise(noise, 2 * p.n, scale))
    return coarse, fine


def make_pairs(p: SimParams, seeds, n_steps: int):
    """Training pairs (coarse one-step result, restricted fine target), device tensors."""
    pairs = []
    n = p.n
    for seed in seeds:
        coarse, fine = paired_sims(p, white_noise(n, seed))
        for t in range(n_steps):
            fs = fine.state()
            part = torch.cat([fs["s"], fs["p"]]).contiguous()
            coarse.set_state(api.restrict_gas(fs["gas"]),
                             api.restrict_particles(part, 2 * n).contiguous(), t)
            coarse.step()
            inp = coarse.state()["gas"]
            fine.step()
            pairs.append((inp, api.restrict_gas(fine.state()["gas"])))
        coarse.close()
        fine.close()
    return pairs


def normalisation(pairs):
    """Per-field (mu, sigma) of the inputs and rms s of the corrections."""
    inp = torch.stack([a for a, _ in pairs])
    dif = torch.stack([b - a for a, b in pairs])
    mu = inp.mean(dim=(0, 2, 3, 4))
    sigma = inp.std(dim=(0, 2, 3, 4)).clamp_min(1e-12)
    scale = dif.pow(2).mean(dim=(0, 2, 3, 4)).sqrt().clamp_min(1e-12)
    return mu.tolist(), sigma.tolist(), scale.tolist()


def train(closure, pairs, iters: int, lr: float, batch: int = 1, seed: int = 0,
          lr_final: float | None = None):
    """Adam on random mini-batches of pairs; returns the per-iteration losses (numpy)."""
    rng = np.random.default_rng(seed)
    losses = torch.zeros(iters, dtype=torch.float64, device=pairs[0][0].device)
    n = pairs[0][0].shape[-1]
    xb = torch.empty(batch, 5, n, n, n, device=losses.device)
    tb = torch.empty_like(xb)
    for it in range(iters):
        idx = rng.choice(len(pairs), batch, replace=False)
        for j, k in enumerate(idx):
            xb[j].copy_(pairs[k][0])
            tb[j].copy_(pairs[k][1])
        rate = lr if lr_final is None else lr * (lr_final / lr) ** (it / max(iters - 1, 1))
        closure.train_step(xb, tb, rate, losses[it:it + 1])
    return losses.cpu().numpy()


def pair_loss(closure, pairs):
    """Mean training loss over `pairs` (no update) and the loss of the identity
    correction (the plain solver) in the same units."""
    tot, tot0 = 0.0, 0.0
    for a, b in pairs:
        loss, _ = closure.gradient(a, b)
        tot += loss
    mu, sigma, scale = closure.norm
    s = torch.tensor(scale, device=pairs[0][0].device)[:, None, None, None]
    for a, b in pairs:
        tot0 += (((b - a) / s) ** 2).mean().item()
    return tot / len(pairs), tot0 / len(pairs)


def rel_err(a, b):
    return ((a - b).norm() / b.norm()).item()


def evaluate(p: SimParams, seed: int, closure, n_steps: int | None = None):
    """Field error of the coarse run without and with the closure against the fine run
    restricted to the coarse grid, after n_steps (default: the whole run)."""
    n = p.n
    steps = p.n_steps if n_steps is None else n_steps
    noise = white_noise(n, seed)
    plain, fine = paired_sims(p, noise)
    corr = api.Simulation(p, noise)
    corr.set_closure(closure)
    for s_ in (plain, corr, fine):
        s_.run(steps)
    ref = api.restrict_gas(fine.state()["gas"])
    out = {}
    for name, sim in (("plain", plain), ("closure", corr)):
        g = sim.state()["gas"]
        out[name] = {"rho": rel_err(g[0], ref[0]), "m": rel_err(g[1:4], ref[1:4]),
                     "eps": rel_err(g[4], ref[4])}
    for s_ in (plain, corr, fine):
        s_.close()
    return out


def equal_error(p: SimParams, closure, seed: int = 4000):
    """The closure's run against the plain solver at the error it reaches.

    Runs from one linear field: plain and closure at n, plain at 2n, and a reference at 4n
    (noise refined twice); every field error is taken on the n^3 grid against the reference
    restricted twice (4:1). A power law err(m) = C m^-k through the plain errors at n and 2n
    gives the resolution n_eq at which the plain solver would reach the closure's density
    error, and the measured run times at n and 2n (t ~ m^q) its cost there."""
    n = p.n
    p2 = fine_params(p)
    p4 = fine_params(p2)
    noise = white_noise(n, seed)
    plain = api.Simulation(p, noise)
    corr = api.Simulation(p, noise)
    corr.set_closure(closure)
    mid = api.Simulation(p2)
    w2 = api.refine_noise(noise, 2 * n, plain.ic_amplitude() / mid.ic_amplitude())
    mid.reinit(w2)
    ref = api.Simulation(p4)
    ref.reinit(api.refine_noise(w2, 4 * n, mid.ic_amplitude() / ref.ic_amplitude()))
    for s_ in (plain, corr, mid, ref):
        s_.run()
    truth = api.restrict_gas(api.restrict_gas(ref.state()["gas"]))
    err = {"plain_n": rel_err(plain.state()["gas"][0], truth[0]),
           "closure_n": rel_err(corr.state()["gas"][0], truth[0]),
           "plain_2n": rel_err(api.restrict_gas(mid.state()["gas"])[0], truth[0])}
    for s_ in (plain, corr, mid, ref):
        s_.close()
    ms = {"plain_n": timed_run(p), "closure_n": timed_run(p, closure), "plain_2n": timed_run(p2)}
    out = {"grid": n, "reference_grid": 4 * n, "density_error": err, "ms_per_run": ms}
    if err["plain_2n"] < err["plain_n"] and err["closure_n"] < err["plain_n"]:
        k = np.log(err["plain_n"] / err["plain_2n"]) / np.log(2.0)
        q = np.log(ms["plain_2n"] / ms["plain_n"]) / np.log(2.0)
        n_eq = n * (err["plain_n"] / err["closure_n"]) ** (1.0 / k)
        ms_eq = ms["plain_n"] * (n_eq / n) ** q
        out.update({"error_exponent": k, "cost_exponent": q, "plain_grid_at_closure_error": n_eq,
                    "plain_ms_at_closure_error": ms_eq,
                    "closure_speedup_at_equal_error": ms_eq / ms["closure_n"]})
    return out


def timed_run(p: SimParams, closure=None, reps: int = 2):
    """ms per forward run (all steps) of the solver, with or without the closure."""
    sim = api.Simulation(p, white_noise(p.n, 99))
    if closure is not None:
        sim.set_closure(closure)
    sim.set_graphs(True)
    ts = []
    for _ in range(reps + 1):
        sim.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.run()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    sim.close()
    return float(np.mean(ts[1:]))


def run_params(n: int, n_steps: int):
    """Runs of the pairs and of the evaluation: box n Mpc/h (dx = 1 Mpc/h), a = 0.1 -> 1.0."""
    return default_params(n=n, box=float(n), n_steps=n_steps, a_start=0.1, a_end=1.0,
                          T_init=1e4)


def experiment(n: int = 64, seeds: int = 6, run_steps: int = 100, iters: int = 600,
               batch: int = 2, lr: float = 2e-3, eval_n: int = 256, fine_eval: bool = True):
    """Pairs, training, held-out loss, a-posteriori run error at n, and the trained network
    in eval_n^3 runs (cost with and without it, field error against the 2 eval_n run)."""
    p = run_params(n, run_steps)
    t0 = time.perf_counter()
    pairs = make_pairs(p, range(1, seeds + 1), run_steps)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    mu, sigma, scale = normalisation(pairs)
    clo = api.Closure(_init_weights(0))
    clo.set_norm(mu, sigma, scale)
    held = make_pairs(p, [1000], run_steps)[::10]
    before, plain_loss = pair_loss(clo, held)
    t0 = time.perf_counter()
    losses = train(clo, pairs, iters, lr, batch, lr_final=lr / 10)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    after, _ = pair_loss(clo, held)
    res = {"pairs": len(pairs), "grid": n, "fine_grid": 2 * n,
           "run": f"{run_steps} steps a=0.1->1.0, box n Mpc/h",
           "pair_seconds": t_pairs, "train_seconds": t_train, "iters": iters,
           "batch": batch, "train_loss_first": float(losses[:10].mean()),
           "train_loss_last": float(losses[-10:].mean()),
           "heldout_loss_plain_solver": plain_loss, "heldout_loss_untrained": before,
           "heldout_loss_trained": after,
           "run_error": evaluate(p, 2000, clo),
           "equal_error": equal_error(p, clo)}
    if eval_n:
        pl = run_params(eval_n, run_steps)
        clo_eval = api.Closure(clo.weights())
        clo_eval.set_norm(mu, sigma, scale)
        ms_plain = timed_run(pl)
        ms_clo = timed_run(pl, clo_eval)
        cells = eval_n ** 3 * run_steps
        res["apply"] = {"grid": eval_n, "steps": run_steps,
                        "plain_cell_steps_per_s": cells / (ms_plain / 1e3),
                        "closure_cell_steps_per_s": cells / (ms_clo / 1e3),
                        "plain_ms": ms_plain, "closure_ms": ms_clo}
        if fine_eval:
            res["apply"]["field_error"] = evaluate(pl, 3000, clo_eval)
        clo_eval.close()
    clo.close()
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--seeds", type=int, default=6)
    ap.add_argument("--run-steps", type=int, default=100)
    ap.add_argument("--iters", type=int, default=600)
    ap.add_argument("--batch", type=int, default=2)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--eval-n", type=int, default=256)
    ap.add_argument("--no-fine-eval", action="store_true")
    a = ap.parse_args(argv)
    res = experiment(a.n, a.seeds, a.run_steps, a.iters, a.batch, a.lr, a.eval_n,
                     not a.no_fine_eval)
    print(json.dumps(res), flush=True)
    return res


def _init_weights(seed: int):
    """He-normal weights (last layer scaled by 0.1, zero biases), the layer layout of the
    C ABI."""
    g = np.random.default_rng(seed)
    out = []
    for l, (ci, co) in enumerate(((5, 16), (16, 16), (16, 16), (16, 5))):
        w = g.standard_normal((27, ci, co)) * np.sqrt(2.0 / (27 * ci))
        if l == 3:
            w *= 0.1
        out += [w.reshape(-1), np.zeros(co)]
    return np.concatenate(out).astype(np.float32)


if __name__ == "__main__":
    main()
