"""Inference drivers over the library's posterior and gradient entry points (Sec. 3).

* ``lbfgs`` -- limited-memory BFGS (Nocedal & Wright, *Numerical Optimization*, 2nd ed.,
  Algorithm 7.4 two-loop recursion, Algorithm 7.5 outer loop) with an Armijo line search
  (expanding on steepest-descent steps, backtracking otherwise). The paper's field-level
  inference (Sec. 3.2) optimises the white-noise amplitudes with L-BFGS keeping M = 8 pairs
  and a tolerance of 1e-5 (read here as the gradient norm relative to its initial value). The algorithm is written over a small set of vector operations so that
  the same code runs on device vectors (the library's ``sim_dot`` / ``sim_axpby`` kernels:
  the 2,097,152 amplitudes never leave the GPU; only scalars reach the host) and on numpy
  arrays (its CPU tests).
* ``fli_lbfgs`` -- that optimiser on ``Simulation.posterior``.

Scalars (step lengths, curvature pairs' 1/y.s) are host floats; every vector update is a
library kernel launch.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


class NumpyOps:
    """Vector operations on numpy float64 arrays (CPU tests of the algorithm)."""

    @staticmethod
    def dot(a, b):
        return float(np.dot(a.ravel(), b.ravel()))

    @staticmethod
    def axpby(alpha, x, beta, y):
        y *= beta
        y += alpha * x
        return y

    @staticmethod
    def copy(x):
        return x.copy()

    @staticmethod
    def assign(dst, src):
        dst[...] = src
        return dst


class DeviceOps:
    """Vector operations on float32 CUDA tensors through the library's kernels."""

    def __init__(self, dh):
        self.dh = dh

    def dot(self, a, b):
        return self.dh.dot(a, b).item()

    def axpby(self, alpha, x, beta, y):
        return self.dh.axpby(alpha, x, beta, y)

    @staticmethod
    def copy(x):
        return x.clone()

    @staticmethod
    def assign(dst, src):
        dst.copy_(src)
        return dst


@dataclass
class LbfgsResult:
    x: object
    f: float
    iterations: int
    evaluations: int
    converged: bool
    history: list = field(default_factory=list)   # (iteration, f, |g|) per iteration


def lbfgs(fun_grad, x0, ops, m: int = 8, max_iter: int = 100, rtol: float = 1e-5,
          c1: float = 1e-4, max_backtracks: int = 30, max_expand: int = 40, callback=None):
    """Minimise f from x0. fun_grad(x) -> (f, g) with g a new vector; ops: NumpyOps or
    DeviceOps. Stops when |g| <= rtol |g(x0)| (converged), when an iteration no longer lowers
    f or the line search finds no Armijo step, or after max_iter iterations.

    Line search: from the step 1 of the quasi-Newton direction (the first direction is the
    steepest descent, whose scale is unknown: there the step starts at 1 / |g| and is doubled
    while f keeps falling and the Armijo condition holds, so a badly scaled first step does
    not stall the run), halved until the Armijo condition f(x + a d) <= f + c1 a g.d holds."""
    x = ops.copy(x0)
    f, g = fun_grad(x)
    evals = 1
    g0n = math.sqrt(ops.dot(g, g))
    S, Y, R = [], [], []          # curvature pairs s_i, y_i and 1 / (y_i . s_i)
    hist = [(0, f, g0n)]
    converged = g0n == 0.0
    it = 0
    for it in range(1, max_iter + 1):
        if converged:
            it -= 1
            break
        # two-loop recursion: d = -H g with H0 = (s.y / y.y) I from the newest pair
        q = ops.copy(g)
        alpha = []
        for s_i, y_i, r_i in zip(reversed(S), reversed(Y), reversed(R)):
            a_i = r_i * ops.dot(s_i, q)
            alpha.append(a_i)
            ops.axpby(-a_i, y_i, 1.0, q)
        gamma = ops.dot(S[-1], Y[-1]) / ops.dot(Y[-1], Y[-1]) if S else 1.0
        ops.axpby(0.0, q, gamma, q)
        for (s_i, y_i, r_i), a_i in zip(zip(S, Y, R), reversed(alpha)):
            b_i = r_i * ops.dot(y_i, q)
            ops.axpby(a_i - b_i, s_i, 1.0, q)
        d = ops.axpby(0.0, q, -1.0, q)
        gd = ops.dot(g, d)
        steepest = not S
        if not gd < 0:                      # not a descent direction: restart on -g
            S, Y, R = [], [], []
            d = ops.axpby(-1.0, g, 0.0, d)
            gd = ops.dot(g, d)
            steepest = True
        step = 1.0 / max(math.sqrt(-gd), 1e-300) if steepest else 1.0

        def trial(a):
            xt = ops.copy(x)
            ops.axpby(a, d, 1.0, xt)
            ft, gt = fun_grad(xt)
            return xt, ft, gt

        xn, fn, gn = trial(step)
        evals += 1
        ok = math.isfinite(fn) and fn <= f + c1 * step * gd
        if ok and steepest:
            for _ in range(max_expand):       # expand while f keeps falling
                x2, f2, g2 = trial(2.0 * step)
                evals += 1
                if not (math.isfinite(f2) and f2 < fn and f2 <= f + c1 * 2.0 * step * gd):
                    break
                step, xn, fn, gn = 2.0 * step, x2, f2, g2
        else:
            for _ in range(max_backtracks):
                if ok:
                    break
                step *= 0.5
                xn, fn, gn = trial(step)
                evals += 1
                ok = math.isfinite(fn) and fn <= f + c1 * step * gd
        if not ok:
            break
        s_new = ops.axpby(-1.0, x, 1.0, ops.copy(xn))
        y_new = ops.axpby(-1.0, g, 1.0, ops.copy(gn))
        ys = ops.dot(y_new, s_new)
        if ys > 1e-12 * math.sqrt(ops.dot(y_new, y_new) * ops.dot(s_new, s_new)):
            S.append(s_new)
            Y.append(y_new)
            R.append(1.0 / ys)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
                R.pop(0)
        df = f - fn
        x, f, g = xn, fn, gn
        gn2 = math.sqrt(ops.dot(g, g))
        hist.append((it, f, gn2))
        if callback is not None:
            callback(it, x, f, g)
        if gn2 <= rtol * g0n or not df > 0:
            converged = gn2 <= rtol * g0n
            break
    return LbfgsResult(x=x, f=f, iterations=it, evaluations=evals, converged=converged,
                       history=hist)


def fli_lbfgs(sim, data, sigma_n: float, x0, observable: int, m: int = 8, max_iter: int = 50,
              rtol: float = 1e-5, callback=None):
    """Field-level inference (Sec. 3.2) with L-BFGS on the amplitudes: each evaluation is one
    sim_posterior call (ICs, whole run, observable likelihood + prior, checkpointed reverse
    pass)."""
    import paper_2502_02294_gb300 as dh

    def fun_grad(x):
        loss, grad = sim.posterior(x, data, sigma_n, observable=observable)
        return loss.sum().item(), grad

    return lbfgs(fun_grad, x0, DeviceOps(dh), m=m, max_iter=max_iter, rtol=rtol,
                 callback=callback)


# ---------------------------------------------------------------------- Sec. 3.1
PK_PARAMS = ("E0", "delta_c", "sigma8", "omega_m")   # the four parameters the paper samples


def pk_covariance(dh, params, nbins: int):
    """Mean and covariance of the binned gas-density power spectrum over a batch of boxes
    (Sec. 3.1: 100 boxes with independent seeds). `params`: list of SimParams that differ
    only in their seeds; run as one batched handle (every kernel covers all boxes). Returns
    (k, mean, cov, per-box spectra) as numpy float64 arrays (nbins-sized)."""
    import torch
    sim = dh.Simulation(list(params))
    sim.run()
    gas = sim.state()["gas"]
    box = params[0].box
    pks = []
    k = None
    for b in range(len(params)):
        kk, pk, _ = dh.power_spectrum(gas[b, 0].contiguous(), box, nbins)
        pks.append(pk)
        k = kk
    P = torch.stack(pks).cpu().numpy()
    sim.close()
    mean = P.mean(0)
    cov = np.cov(P, rowvar=False)
    return k.cpu().numpy(), mean, cov, P


class PkLikelihood:
    """-log L(theta) = 1/2 (P(theta) - P_obs)^T C^-1 (P(theta) - P_obs) + Gaussian priors, with
    P(theta) the binned gas-density spectrum of one run at the parameters theta from fixed
    white noise, and its gradient through the library's adjoint: dL/dP -> P(k) adjoint ->
    dL/drho -> checkpointed reverse pass -> dL/dtheta. The 64-sized linear algebra of the
    Gaussian (C^-1 by a Cholesky factorisation) is host numpy."""

    def __init__(self, dh, base_params, noise, p_obs, cov, nbins: int, names=PK_PARAMS,
                 prior_mean=None, prior_sigma=None, ridge: float = 1e-12):
        import ctypes
        import torch
        self.dh, self.torch, self.ctypes = dh, torch, ctypes
        self.base = base_params
        self.names = tuple(names)
        self.idx = [dh.PARAM_NAMES.index(nm) for nm in self.names]
        self.nbins = nbins
        self.p_obs = np.asarray(p_obs, dtype=np.float64)
        C = np.asarray(cov, dtype=np.float64)
        C = C + ridge * np.trace(C) / len(C) * np.eye(len(C))
        self.L = np.linalg.cholesky(C)
        self.prior_mean = None if prior_mean is None else np.asarray(prior_mean, dtype=np.float64)
        self.prior_sigma = None if prior_sigma is None else np.asarray(prior_sigma, dtype=np.float64)
        self.sim = dh.Simulation(self._params(self.theta0()), noise)
        n = base_params.n
        self.dL = torch.zeros(5, n, n, n, dtype=torch.float32, device=noise.device)
        self.evals = 0

    def theta0(self):
        return np.array([getattr(self.base, nm) for nm in self.names], dtype=np.float64)

    def _params(self, theta):
        p = self.dh.SimParams.from_buffer_copy(self.base)
        for nm, v in zip(self.names, theta):
            setattr(p, nm, float(v))
        return p

    def spectrum(self, theta):
        self.sim.set_params(self._params(theta))
        self.sim.run()
        rho = self.sim.state()["gas"][0].contiguous()
        _, pk, _ = self.dh.power_spectrum(rho, self.base.box, self.nbins)
        return rho, pk

    def value_and_grad(self, theta):
        """(-log posterior, its gradient with respect to theta)."""
        torch = self.torch
        rho, pk = self.spectrum(theta)
        r = pk.cpu().numpy() - self.p_obs
        w = np.linalg.solve(self.L.T, np.linalg.solve(self.L, r))      # C^-1 r
        val = 0.5 * float(r @ w)
        dL_dpk = torch.from_numpy(w).to(rho.device)
        self.dL[0] = self.dh.power_spectrum_adjoint(rho, self.base.box, self.nbins, dL_dpk)
        _, dpar = self.sim.run_adjoint(self.dL, want_noise=False)
        grad = dpar.cpu().numpy()[self.idx].astype(np.float64)
        if self.prior_mean is not None:
            z = (np.asarray(theta) - self.prior_mean) / self.prior_sigma
            val += 0.5 * float(z @ z)
            grad = grad + z / self.prior_sigma
        self.evals += 1
        return val, grad

    def close(self):
        self.sim.close()


def hmc(value_and_grad, theta0, inv_mass, n_samples: int, n_leapfrog: int = 8,
        step: float = 0.1, n_warmup: int = 50, target_accept: float = 0.75, seed: int = 0):
    """Hamiltonian Monte Carlo (Duane et al. 1987; Neal 2011, Sec. 5.3.2) with a diagonal mass
    matrix (inv_mass: its inverse, e.g. the prior variances), leapfrog integration of
    n_leapfrog steps, a Metropolis accept/reject on the total energy, and during the first
    n_warmup iterations a multiplicative adaptation of the step towards target_accept (the
    step is then frozen). Returns (samples [n_samples, d], accept rate after warm-up, step,
    energies)."""
    rng = np.random.default_rng(seed)
    inv_mass = np.asarray(inv_mass, dtype=np.float64)
    x = np.asarray(theta0, dtype=np.float64).copy()
    U, g = value_and_grad(x)
    out, acc, energies = [], 0, []
    for it in range(n_warmup + n_samples):
        p = rng.normal(size=x.shape) / np.sqrt(inv_mass)
        H0 = U + 0.5 * float(p @ (inv_mass * p))
        xn, pn, gn, Un = x.copy(), p.copy(), g.copy(), U
        pn -= 0.5 * step * gn
        for j in range(n_leapfrog):
            xn += step * inv_mass * pn
            Un, gn = value_and_grad(xn)
            if not np.isfinite(Un):
                break
            if j + 1 < n_leapfrog:
                pn -= step * gn
        pn -= 0.5 * step * gn
        H1 = Un + 0.5 * float(pn @ (inv_mass * pn)) if np.isfinite(Un) else np.inf
        a = math.exp(min(0.0, H0 - H1)) if np.isfinite(H1) else 0.0
        accepted = rng.uniform() < a
        if accepted:
            x, U, g = xn, Un, gn
        if it < n_warmup:
            step *= math.exp(0.5 * (a - target_accept))
        else:
            acc += accepted
            out.append(x.copy())
            energies.append(U)
    return np.array(out), acc / max(n_samples, 1), step, np.array(energies)


def effective_sample_size(chain):
    """N / tau per coordinate, tau = 1 + 2 sum_{t>=1} rho_t evaluated as -1 + 2 sum_k Gamma_k
    with Gamma_k = rho_{2k} + rho_{2k+1}, truncated at the first negative Gamma_k (Geyer's
    initial positive sequence, 1992). Anti-correlated chains give N_eff > N, as the paper
    reports for its sampler."""
    x = np.asarray(chain, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    N = x.shape[0]
    out = []
    for j in range(x.shape[1]):
        y = x[:, j] - x[:, j].mean()
        v = float(y @ y) / N
        if v <= 0:
            out.append(float(N))
            continue
        f = np.fft.rfft(y, 2 * N)
        acf = np.fft.irfft(f * np.conj(f))[:N] / (N * v)
        s = 0.0
        t = 0
        while t + 1 < N:
            pair = acf[t] + acf[t + 1]
            if pair < 0:
                break
            s += pair
            t += 2
        out.append(N / max(-1.0 + 2.0 * s, 1.0 / N))
    return np.array(out)


def pk_hmc_experiment(dh, n: int = 64, box: float = 8.0, a_start: float = 0.05,
                      a_end: float = 0.25, n_steps: int = 20, n_boxes: int = 100,
                      nbins: int | None = None, n_samples: int = 150, n_warmup: int = 30,
                      n_leapfrog: int = 6, seed: int = 0):
    """Sec. 3.1 end to end: the mock spectrum (seed 1 at the fiducial parameters), the
    covariance of the gas spectrum over n_boxes batched boxes with independent seeds, and an
    HMC chain over (E0, delta_c, sigma8, Omega_m) with the paper's Gaussian priors (sigma
    0.002 for E0, 0.02 for the others) centred at the truth. Box to z = 3 (a = 0.25)."""
    import time
    import torch
    nb = nbins or n // 4
    # subgrid thresholds that form stars in this small box (delta_c of order unity, as in
    # the paper's parameter ranges)
    fid = dict(n=n, box=box, n_steps=n_steps, ckpt_every=n_steps, a_start=a_start,
               a_end=a_end, subgrid_on=1, delta_c=1.0, w_delta=0.1, T_c=1e6, w_T=1e5,
               Pi0=0.2, E0=0.03, T0_uv=0.0, rms_ref=0.1)
    t0 = time.time()
    boxes = [dh.default_params(**fid, seed=100 + b, instance=b) for b in range(n_boxes)]
    k, mean, cov, P = pk_covariance(dh, boxes, nb)
    t_cov = time.time() - t0
    base = dh.default_params(**fid, seed=1)
    dev = torch.device("cuda", torch.cuda.current_device())
    import synth
    noise = torch.from_numpy(synth.white_noise(n, 1).astype("float32")).to(dev)
    truth_sim = dh.Simulation(base, noise)
    truth_sim.run()
    rho = truth_sim.state()["gas"][0].contiguous()
    _, p_obs, _ = dh.power_spectrum(rho, box, nb)
    truth_sim.close()
    theta_true = np.array([getattr(base, nm) for nm in PK_PARAMS])
    sig = np.array([0.002, 0.02, 0.02, 0.02])
    like = PkLikelihood(dh, base, noise, p_obs.cpu().numpy(), cov, nb,
                        prior_mean=theta_true, prior_sigma=sig, ridge=1e-6)
    t1 = time.time()
    xs, acc, step, _ = hmc(like.value_and_grad, theta_true, sig ** 2, n_samples,
                           n_leapfrog=n_leapfrog, step=0.3, n_warmup=n_warmup, seed=seed)
    t_hmc = time.time() - t1
    ess = effective_sample_size(xs)
    evals = like.evals
    like.close()
    z = (xs.mean(0) - theta_true) / xs.std(0)
    return {"workload": f"{n}^3 boxes, {box} Mpc/h, {n_steps} steps a={a_start}->{a_end}, "
                        f"subgrid on; covariance from {n_boxes} batched boxes; HMC over "
                        "(E0, delta_c, sigma8, Omega_m) with the paper's priors",
            "nbins": nb, "covariance_seconds": t_cov, "hmc_seconds": t_hmc,
            "gradient_evaluations": evals, "seconds_per_evaluation": t_hmc / max(evals, 1),
            "samples": n_samples, "warmup": n_warmup, "leapfrog": n_leapfrog,
            "step": step, "accept_rate": acc, "ess": ess.tolist(),
            "posterior_mean": xs.mean(0).tolist(), "posterior_std": xs.std(0).tolist(),
            "truth": theta_true.tolist(), "truth_offset_in_std": z.tolist(),
            "params": list(PK_PARAMS)}
