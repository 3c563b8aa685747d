"""The L-BFGS optimiser of the inference drivers, run on numpy vectors (no GPU): it is the
algorithm of Nocedal & Wright (two-loop recursion, Algorithm 7.4; outer loop, Algorithm
7.5) with an Armijo backtracking line search, pinned by problems with known minimisers:

* a strictly convex quadratic 1/2 x.Ax - b.x (minimiser A^-1 b, condition number 1e3);
* the Rosenbrock function from (-1.2, 1) (minimiser (1, 1));
* monotone decrease of f (the Armijo condition) and at most M stored pairs.
"""
import importlib.util
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location(
    "dh_inference", os.path.join(ROOT, "paper_2502_02294_gb300", "inference.py"))
inf = importlib.util.module_from_spec(_spec)
sys.modules["dh_inference"] = inf
_spec.loader.exec_module(inf)


def test_quadratic_minimiser():
    rng = np.random.default_rng(0)
    n = 60
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    A = Q @ np.diag(np.logspace(0, 3, n)) @ Q.T
    b = rng.normal(size=n)

    def fg(x):
        return 0.5 * x @ A @ x - b @ x, A @ x - b

    r = inf.lbfgs(fg, np.zeros(n), inf.NumpyOps, m=8, max_iter=500, rtol=1e-12)
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(r.x - xs) < 1e-6 * np.linalg.norm(xs), (r.iterations, np.linalg.norm(r.x - xs))
    fs = [h[1] for h in r.history]
    assert all(f1 <= f0 + 1e-12 for f0, f1 in zip(fs, fs[1:]))


def test_rosenbrock():
    def fg(x):
        a, b = x
        f = (1 - a) ** 2 + 100 * (b - a * a) ** 2
        g = np.array([-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)])
        return f, g

    r = inf.lbfgs(fg, np.array([-1.2, 1.0]), inf.NumpyOps, m=5, max_iter=500, rtol=1e-10)
    assert np.abs(r.x - 1).max() < 1e-5, (r.x, r.iterations)
    assert r.history[-1][1] < 1e-10


def test_first_step_expands_a_badly_scaled_start():
    """f = 1/2 |x|^2 / s^2 with a tiny scale s: the first trial step has length 1 along -g and
    is doubled while f falls, so one iteration already lands near the minimiser."""
    calls = []
    sc = 1e3

    def fg(x):
        calls.append(x.copy())
        return 0.5 * float(x @ x) / sc ** 2, x.copy() / sc ** 2

    x0 = np.full(4, 3.0e3)
    r = inf.lbfgs(fg, x0, inf.NumpyOps, m=2, max_iter=1, rtol=0.0)
    assert np.allclose(calls[1], x0 - x0 / np.linalg.norm(x0))       # unit first trial
    assert np.linalg.norm(calls[2] - x0) > 1.9                       # then doubled
    assert r.f < 0.3 * fg(x0)[0], (r.f, r.evaluations)


def test_hmc_samples_a_correlated_gaussian():
    """Target N(mu, S) with a strong correlation (the sigma8-Omega_m kind of degeneracy):
    the sample mean and covariance match within their sampling errors."""
    mu = np.array([0.3, 0.8])
    S = np.array([[0.02 ** 2, -0.9 * 0.02 * 0.03], [-0.9 * 0.02 * 0.03, 0.03 ** 2]])
    Si = np.linalg.inv(S)

    def vg(x):
        d = x - mu
        return 0.5 * float(d @ Si @ d), Si @ d

    xs, acc, step, _ = inf.hmc(vg, mu + 0.05, np.diag(S), 4000, n_leapfrog=10, step=0.2,
                               n_warmup=300, seed=1)
    assert 0.5 < acc < 0.98, acc
    ess = inf.effective_sample_size(xs)
    se = np.sqrt(np.diag(S) / ess)
    assert np.all(np.abs(xs.mean(0) - mu) < 5 * se), (xs.mean(0), mu, se)
    C = np.cov(xs, rowvar=False)
    assert np.allclose(C, S, rtol=0.15, atol=0.15 * np.abs(S).max()), (C, S)


def test_effective_sample_size_of_ar1():
    """AR(1) with coefficient phi: N_eff = N (1 - phi) / (1 + phi)."""
    rng = np.random.default_rng(3)
    N, phi = 200000, 0.6
    e = rng.normal(size=N)
    x = np.empty(N)
    x[0] = e[0]
    for t in range(1, N):
        x[t] = phi * x[t - 1] + e[t]
    want = N * (1 - phi) / (1 + phi)
    got = inf.effective_sample_size(x)[0]
    assert abs(got / want - 1) < 0.05, (got, want)
    # anti-correlated chain: N_eff above N
    y = np.empty(N)
    y[0] = e[0]
    for t in range(1, N):
        y[t] = -0.5 * y[t - 1] + e[t]
    assert inf.effective_sample_size(y)[0] > N
