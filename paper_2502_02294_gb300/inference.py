"""Inference drivers over the library's posterior and gradient entry points (Sec. 3).

* ``lbfgs`` -- limited-memory BFGS (Nocedal & Wright, *Numerical Optimization*, 2nd ed.,
  Algorithm 7.4 two-loop recursion, Algorithm 7.5 outer loop) with a backtracking line search
  on the Armijo condition. The paper's field-level inference (Sec. 3.2) optimises the
  white-noise amplitudes with L-BFGS keeping M = 8 pairs and stopping at a relative
  tolerance of 1e-5. The algorithm is written over a small set of vector operations so that
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
          gtol: float = 0.0, c1: float = 1e-4, max_backtracks: int = 20, callback=None):
    """Minimise f from x0. fun_grad(x) -> (f, g) with g a new vector; ops: NumpyOps or
    DeviceOps. Stops when the relative decrease of f over an iteration falls below rtol,
    when |g| <= gtol, or after max_iter iterations."""
    x = ops.copy(x0)
    f, g = fun_grad(x)
    evals = 1
    S, Y, R = [], [], []          # curvature pairs s_i, y_i and 1 / (y_i . s_i)
    hist = [(0, f, math.sqrt(ops.dot(g, g)))]
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        # two-loop recursion: d = -H g with H0 = (s.y / y.y) I from the newest pair
        q = ops.copy(g)
        alpha = []
        for s_i, y_i, r_i in zip(reversed(S), reversed(Y), reversed(R)):
            a_i = r_i * ops.dot(s_i, q)
            alpha.append(a_i)
            ops.axpby(-a_i, y_i, 1.0, q)
        if S:
            gamma = ops.dot(S[-1], Y[-1]) / ops.dot(Y[-1], Y[-1])
        else:
            gamma = 1.0 / max(math.sqrt(ops.dot(g, g)), 1e-300)   # first step of length 1
        ops.axpby(0.0, q, gamma, q)
        for (s_i, y_i, r_i), a_i in zip(zip(S, Y, R), reversed(alpha)):
            b_i = r_i * ops.dot(y_i, q)
            ops.axpby(a_i - b_i, s_i, 1.0, q)
        d = ops.axpby(0.0, q, -1.0, q)
        gd = ops.dot(g, d)
        if not gd < 0:                      # not a descent direction: restart on -g
            S, Y, R = [], [], []
            d = ops.axpby(0.0, g, 0.0, d)
            ops.axpby(-1.0 / max(math.sqrt(ops.dot(g, g)), 1e-300), g, 0.0, d)
            gd = ops.dot(g, d)
        # backtracking line search on the Armijo condition
        step = 1.0
        xn = ops.copy(x)
        accepted = False
        for _ in range(max_backtracks):
            ops.assign(xn, x)
            ops.axpby(step, d, 1.0, xn)
            fn, gn = fun_grad(xn)
            evals += 1
            if math.isfinite(fn) and fn <= f + c1 * step * gd:
                accepted = True
                break
            step *= 0.5
        if not accepted:
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
        if df <= rtol * max(abs(f), 1e-300) or gn2 <= gtol:
            converged = True
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
