"""Physics validation runs of the GPU solver (Sec. 2.3.4 and Fig. 3 of arXiv 2502.02294).

* ``sedov`` -- the Sedov-Taylor point explosion: energy E0 deposited in the central cell of
  a uniform, cold, periodic n^3 gas at rest, evolved with the library's relaxing-TVD sweeps
  in the Strang order (sim_sweep; step length from the largest signal speed at CFL 0.3,
  sim_max_signal_speed) until the self-similar radius r_sh = 1.15 (E0 t^2 / rho1)^(1/5)
  reaches r_target cells. The paper's 128^3 test puts the front within 2 px of r_sh with an
  angular variation below 1 px at r_sh = 20 cells. The front is located along 48 random
  directions as the radius of the density maximum (linear interpolation on the host of the
  final density, which is read back once).
* ``convergence`` -- one linear field run at n and at 2n cells in the same box (the fine
  run's white noise is the band-limited refinement of the coarse one, sim_refine_noise),
  subgrid off; the baryon power spectra of the final gas densities are compared per k bin,
  as the paper's resolution test does (agreement up to k ~ 7 h/Mpc for its 8 Mpc/h box).
"""
from __future__ import annotations

import math

import numpy as np
import torch

STRANG = ("xyz", "zyx", "zxy", "yxz", "yzx", "xzy")


def sedov(dh, n: int = 128, r_target: float = 20.0, E0: float = 1.0e4, rho1: float = 1.0,
          p_bg: float = 1e-6, gamma: float = 5.0 / 3.0, cfl: float = 0.3, seed: int = 0):
    dev = torch.device("cuda", torch.cuda.current_device())
    U = torch.zeros(5, n, n, n, dtype=torch.float32, device=dev)
    U[0] = rho1
    U[4] = p_bg / (gamma - 1)
    c = n // 2
    U[4, c, c, c] += E0
    mass0, energy0 = rho1 * n ** 3, E0 + p_bg / (gamma - 1) * n ** 3
    t_end = math.sqrt((r_target / 1.15) ** 5 * rho1 / E0)
    t, step, max_cfl = 0.0, 0, 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    while t < t_end * (1 - 1e-12):
        vmax = dh.max_signal_speed(U, gamma)
        dt = min(cfl / vmax, t_end - t)
        max_cfl = max(max_cfl, vmax * dt)
        for ax in STRANG[step % 6]:
            U = dh.sweep(U, "xyz".index(ax), dt, gamma)
        t += dt
        step += 1
    e1.record()
    e1.synchronize()
    from scipy.ndimage import map_coordinates
    rho = U[0].double().cpu().numpy()
    rng = np.random.default_rng(seed)
    dirs = rng.normal(size=(48, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = np.arange(2.0, min(1.6 * r_target, n / 2 - 1), 0.05)
    radii = np.array([r[np.argmax(map_coordinates(rho, c + d[:, None] * r[None, :], order=1))]
                      for d in dirs])
    r_exact = 1.15 * (E0 * t_end ** 2 / rho1) ** 0.2
    return {"n": n, "steps": step, "t_end": t_end, "r_exact_cells": r_exact,
            "r_front_mean_cells": float(radii.mean()), "r_front_std_cells": float(radii.std()),
            "max_cfl": max_cfl, "gpu_ms": e0.elapsed_time(e1),
            "mass_rel_change": float(U[0].double().sum().item() / mass0 - 1),
            "energy_rel_change": float(U[4].double().sum().item() / energy0 - 1)}


def convergence(dh, n: int = 64, box: float = 8.0, a_start: float = 0.05, a_end: float = 0.286,
                n_steps: int = 60, seed: int = 5, nbins: int | None = None):
    """Final gas-density P(k) of the same linear field at n and 2n cells (box in Mpc/h;
    a_end 0.286 is z = 2.5)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    import synth
    w = torch.from_numpy(synth.white_noise(n, seed).astype("float32")).to(dev)
    kw = dict(box=box, n_steps=n_steps, ckpt_every=n_steps, a_start=a_start, a_end=a_end,
              subgrid_on=0)
    pc = dh.default_params(n=n, **kw)
    coarse = dh.Simulation(pc, w)
    C_c = coarse.ic_amplitude()
    pf = dh.default_params(n=2 * n, **dict(kw, kc_frac=pc.kc_frac / 2))
    probe = dh.Simulation(pf, torch.zeros(2 * n, 2 * n, 2 * n, device=dev))
    C_f = probe.ic_amplitude()
    probe.close()
    wf = dh.refine_noise(w, 2 * n, C_c / C_f)
    fine = dh.Simulation(pf, wf)
    coarse.run()
    fine.run()
    rc = coarse.state()["gas"][0].contiguous()
    rf = fine.state()["gas"][0].contiguous()
    nb = nbins or n // 2
    k, pkc, _ = dh.power_spectrum(rc, box, nb)
    _, pkf, _ = dh.power_spectrum(rf, box, nb)
    coarse.close()
    fine.close()
    k, pkc, pkf = k.cpu().numpy(), pkc.cpu().numpy(), pkf.cpu().numpy()
    ratio = pkc / pkf
    bad = np.nonzero(np.abs(ratio - 1) > 0.1)[0]
    k_agree = float(k[bad[0] - 1]) if len(bad) and bad[0] > 0 else (float(k[-1]) if not len(bad) else 0.0)
    return {"n": n, "n_fine": 2 * n, "box": box, "a_end": a_end, "k": k.tolist(),
            "pk_ratio_coarse_over_fine": ratio.tolist(), "k_agree_10pct": k_agree,
            "k_nyquist_coarse": math.pi * n / box}
