"""Torch-facing wrappers of the C ABI (same names as the C entry points, minus ``sim_``).

PyTorch provides device memory and the current CUDA stream; every computation is a call
into libdiffhydro.so. Inputs must be contiguous CUDA tensors of the stated dtype.
"""
from __future__ import annotations

import ctypes

import torch

import numpy as np

from ._lib import (CLOSURE_NWEIGHTS, DG_N, DG_NAMES, KT_N, KT_NAMES, NPARAMS, OBS_DENSITY,
                   OBS_THERMAL, SimParams, check, default_params, lib)

F32, F64, U32 = torch.float32, torch.float64, torch.int32


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _chk(t, dtype, numel, name):
    if t.dtype != dtype or t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements of {dtype}, got {t.numel()} of {t.dtype}")


# ------------------------------------------------------------------ single kernels
def _side(cells: int) -> int:
    n = round(cells ** (1.0 / 3.0))
    if n ** 3 != cells:
        raise ValueError(f"{cells} cells is not a cube")
    return n


def sweep(u_in, axis: int, nu: float, gamma: float = 5.0 / 3.0, limiter_eps: float = 1e-30,
          variant: int = 0):
    """variant: SWEEP_* kernel form (0 = the built-in choice)."""
    n = _side(u_in.numel() // 5)
    _chk(u_in, F32, 5 * n ** 3, "u_in")
    out = torch.empty_like(u_in)
    check(lib.sim_sweep(_ptr(u_in), _ptr(out), n, axis, nu, gamma, limiter_eps, variant,
                        _stream()), "sim_sweep")
    return out


def max_signal_speed(gas, gamma: float = 5.0 / 3.0) -> float:
    """max over cells of max_d |v_d| + c_s (sim_max_signal_speed; synchronises)."""
    n = _side(gas.numel() // 5)
    _chk(gas, F32, 5 * n ** 3, "gas")
    out = torch.empty(1, dtype=F32, device=gas.device)
    check(lib.sim_max_signal_speed(_ptr(gas), n, gamma, _ptr(out), _stream()),
          "sim_max_signal_speed")
    return out.item()


def sweep_adjoint(u_in, lam_out, axis: int, nu: float, gamma: float = 5.0 / 3.0,
                  limiter_eps: float = 1e-30, variant: int = 0):
    n = _side(u_in.numel() // 5)
    _chk(u_in, F32, 5 * n ** 3, "u_in")
    _chk(lam_out, F32, 5 * n ** 3, "lam_out")
    lam_in = torch.empty_like(u_in)
    dnu = torch.zeros(1, dtype=F64, device=u_in.device)
    check(lib.sim_sweep_adjoint(_ptr(u_in), _ptr(lam_out), _ptr(lam_in), n, axis, nu, gamma,
                                limiter_eps, _ptr(dnu), variant, _stream()), "sim_sweep_adjoint")
    return lam_in, dnu


def deposit_cic(s, n: int, box: float, values=None, grid=None):
    _chk(s, F32, 3 * n ** 3, "s")
    if grid is None:
        grid = torch.zeros(n, n, n, dtype=F32, device=s.device)
    check(lib.sim_deposit_cic(_ptr(s), _ptr(values), n, box, _ptr(grid), _stream()), "sim_deposit_cic")
    return grid


def interp_cic(grid, s, n: int, box: float):
    nf = grid.numel() // n ** 3
    _chk(s, F32, 3 * n ** 3, "s")
    out = torch.empty(nf, n ** 3, dtype=F32, device=s.device)
    check(lib.sim_interp_cic(_ptr(grid), nf, n, box, _ptr(s), _ptr(out), _stream()), "sim_interp_cic")
    return out


def gravity(delta, box: float, pref: float):
    n = delta.shape[-1]
    _chk(delta, F32, n ** 3, "delta")
    g = torch.empty(3, n, n, n, dtype=F32, device=delta.device)
    check(lib.sim_gravity(_ptr(delta), n, box, pref, _ptr(g), _stream()), "sim_gravity")
    return g


def gravity_adjoint(lam_g, box: float, pref: float):
    n = lam_g.shape[-1]
    _chk(lam_g, F32, 3 * n ** 3, "lam_g")
    out = torch.empty(n, n, n, dtype=F32, device=lam_g.device)
    check(lib.sim_gravity_adjoint(_ptr(lam_g), n, box, pref, _ptr(out), _stream()), "sim_gravity_adjoint")
    return out


def subgrid(gas, a: float, params: SimParams, step: int, with_outputs: bool = True):
    """In-place subgrid update of gas [5, n, n, n]; returns (zhat, events)."""
    n = gas.shape[-1]
    _chk(gas, F32, 5 * n ** 3, "gas")
    zhat = torch.empty(n, n, n, dtype=F32, device=gas.device) if with_outputs else None
    events = torch.zeros((n ** 3 + 31) // 32, dtype=U32, device=gas.device) if with_outputs else None
    check(lib.sim_subgrid(_ptr(gas), n, a, ctypes.byref(params), step, _ptr(zhat), _ptr(events),
                          _stream()), "sim_subgrid")
    return zhat, events


def subgrid_adjoint(gas_in, lam, a: float, params: SimParams, step: int):
    """lam [5, n, n, n] is overwritten; returns (dparams[NPARAMS], dfb[1])."""
    n = gas_in.shape[-1]
    dpar = torch.zeros(NPARAMS, dtype=F64, device=gas_in.device)
    dfb = torch.zeros(1, dtype=F64, device=gas_in.device)
    check(lib.sim_subgrid_adjoint(_ptr(gas_in), _ptr(lam), n, a, ctypes.byref(params), step,
                                  _ptr(dpar), _ptr(dfb), _stream()), "sim_subgrid_adjoint")
    return dpar, dfb


def philox(seed: int, step: int, instance: int, tag: int, count: int, device="cuda"):
    out = torch.empty(count, 4, dtype=U32, device=device)
    check(lib.sim_philox(seed, step, instance, tag, count, _ptr(out), _stream()), "sim_philox")
    return out


def power_spectrum(a, box: float, nbins: int, b=None):
    n = a.shape[-1]
    k = torch.empty(nbins, dtype=F64, device=a.device)
    pk = torch.empty_like(k)
    nm = torch.empty_like(k)
    check(lib.sim_power_spectrum(_ptr(a), _ptr(b), n, box, nbins, _ptr(k), _ptr(pk), _ptr(nm),
                                 _stream()), "sim_power_spectrum")
    return k, pk, nm


def power_spectrum_adjoint(a, box: float, nbins: int, dL_dpk):
    """dL/da for a loss of the binned auto spectrum of a (sim_power_spectrum_adjoint)."""
    n = a.shape[-1]
    _chk(a, F32, n ** 3, "a")
    _chk(dL_dpk, F64, nbins, "dL_dpk")
    out = torch.empty_like(a)
    check(lib.sim_power_spectrum_adjoint(_ptr(a), n, box, nbins, _ptr(dL_dpk), _ptr(out),
                                         _stream()), "sim_power_spectrum_adjoint")
    return out


def cross_correlation(a, b, box: float, nbins: int):
    """(k, r_c(k), nmodes) of two n^3 fields (sim_cross_correlation)."""
    n = a.shape[-1]
    _chk(a, F32, n ** 3, "a")
    _chk(b, F32, n ** 3, "b")
    k = torch.empty(nbins, dtype=F64, device=a.device)
    rc = torch.empty_like(k)
    nm = torch.empty_like(k)
    check(lib.sim_cross_correlation(_ptr(a), _ptr(b), n, box, nbins, _ptr(k), _ptr(rc), _ptr(nm),
                                    _stream()), "sim_cross_correlation")
    return k, rc, nm


def dot(a, b):
    """sum a_i b_i of two float32 device vectors, as a [1] float64 device tensor (sim_dot)."""
    _chk(b, F32, a.numel(), "b")
    out = torch.empty(1, dtype=F64, device=a.device)
    check(lib.sim_dot(_ptr(a), _ptr(b), a.numel(), _ptr(out), _stream()), "sim_dot")
    return out


def axpby(alpha: float, x, beta: float, y):
    """y = alpha x + beta y in place (sim_axpby)."""
    _chk(x, F32, y.numel(), "x")
    check(lib.sim_axpby(alpha, _ptr(x), beta, _ptr(y), y.numel(), _stream()), "sim_axpby")
    return y


def adam(x, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8, prior_w: float = 0.0, grad_out=None, prior=None):
    """In-place Adam step on x (m, v moments) with gradient g + prior_w x (sim_adam)."""
    cnt = x.numel()
    for t_, nm in ((x, "x"), (g, "g"), (m, "m"), (v, "v")):
        _chk(t_, F32, cnt, nm)
    check(lib.sim_adam(_ptr(x), _ptr(g), _ptr(m), _ptr(v), cnt, lr, beta1, beta2, eps, t,
                       prior_w, _ptr(grad_out), _ptr(prior), _stream()), "sim_adam")
    return x


# ------------------------------------------------------------------ whole path
class Simulation:
    """Owns a sim_t handle. All methods enqueue on torch's current stream at creation.

    `params` is one SimParams, or a list of SimParams for a batch of B instances on grids
    of the same size (sim_init_batch). With B > 1 every array gains a leading instance
    dimension (gas [B, 5, n, n, n], part [B, 6, n^3], noise / target [B, n, n, n],
    parameter derivatives [B, NPARAMS], loss [B]); with B = 1 the shapes have none.
    """

    def __init__(self, params: SimParams | list | None = None, noise=None, **overrides):
        if isinstance(params, (list, tuple)):
            plist = list(params)
            for q in plist:
                for k, v in overrides.items():
                    setattr(q, k, v)
        else:
            q = params if params is not None else default_params(**overrides)
            if params is not None:
                for k, v in overrides.items():
                    setattr(q, k, v)
            plist = [q]
        self.B = len(plist)
        self.params = plist[0]
        self.params_list = plist
        n = self.params.n
        self.n = n
        if noise is not None:
            _chk(noise, F32, self.B * n ** 3, "noise")
        self._stream = torch.cuda.current_stream()
        arr = (SimParams * self.B)(*plist)
        self._arr = arr
        h = ctypes.c_void_p()
        check(lib.sim_init_batch(arr, self.B, _ptr(noise),
                                 ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h)),
              "sim_init_batch")
        self.h = h

    def set_params(self, params):
        """New parameter set(s) for the same grid and schedule (sim_set_params)."""
        plist = list(params) if isinstance(params, (list, tuple)) else [params]
        arr = (SimParams * self.B)(*plist)
        self._check(lib.sim_set_params(self.h, arr), "sim_set_params")
        self.params, self.params_list, self._arr = plist[0], plist, arr

    def _shape(self, *dims):
        return dims if self.B == 1 else (self.B,) + dims

    def close(self):
        if getattr(self, "h", None):
            lib.sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, where):
        check(st, where, self.h)

    def step(self):
        self._check(lib.sim_step(self.h), "sim_step")

    def step_adjoint(self, adj_gas, adj_part, adj_params=None):
        n, B = self.n, self.B
        _chk(adj_gas, F32, 5 * B * n ** 3, "adj_gas")
        _chk(adj_part, F32, 6 * B * n ** 3, "adj_part")
        self._check(lib.sim_step_adjoint(self.h, _ptr(adj_gas), _ptr(adj_part), _ptr(adj_params)),
                    "sim_step_adjoint")

    def run(self, n_steps: int | None = None):
        self._check(lib.sim_run(self.h, self.params.n_steps if n_steps is None else n_steps), "sim_run")

    def run_adjoint(self, dL_dgas=None, dL_dpart=None, want_noise: bool = True):
        n = self.n
        dev = torch.device("cuda", torch.cuda.current_device())
        dnoise = torch.empty(self._shape(n, n, n), dtype=F32, device=dev) if want_noise else None
        dpar = torch.zeros(self._shape(NPARAMS), dtype=F64, device=dev)
        self._check(lib.sim_run_adjoint(self.h, _ptr(dL_dgas), _ptr(dL_dpart), _ptr(dnoise), _ptr(dpar)),
                    "sim_run_adjoint")
        return dnoise, dpar

    def reset(self):
        self._check(lib.sim_reset(self.h), "sim_reset")

    def reinit(self, noise=None):
        if noise is not None:
            _chk(noise, F32, self.B * self.n ** 3, "noise")
        self._check(lib.sim_reinit(self.h, _ptr(noise)), "sim_reinit")

    def loss_density(self, target, c: float, out=None, loss=None):
        """(dL/dgas [5, n, n, n], loss [1] float64) of L = c sum (rho - target)^2
        (per instance with B > 1: [B, 5, n, n, n] and [B])."""
        n, B = self.n, self.B
        _chk(target, F32, B * n ** 3, "target")
        dev = target.device
        out = torch.empty(self._shape(5, n, n, n), dtype=F32, device=dev) if out is None else out
        loss = torch.empty(B, dtype=F64, device=dev) if loss is None else loss
        self._check(lib.sim_loss_density(self.h, _ptr(target), c, _ptr(out), _ptr(loss)),
                    "sim_loss_density")
        return out, loss

    def set_diagnostics(self, on: bool = True):
        self._check(lib.sim_set_diagnostics(self.h, int(on)), "sim_set_diagnostics")

    def diagnostics(self, step: int):
        """Record of the state after `step` (0: initial): {name: value} (a list per name
        with B > 1)."""
        out = (ctypes.c_double * (DG_N * self.B))()
        self._check(lib.sim_diagnostics(self.h, step, out), "sim_diagnostics")
        vals = list(out)
        if self.B == 1:
            return dict(zip(DG_NAMES, vals))
        return {nm: [vals[b * DG_N + j] for b in range(self.B)] for j, nm in enumerate(DG_NAMES)}

    def fli_step(self, noise, m, v, data, sigma_n: float, lr: float, t: int, grad=None,
                 loss=None, observable: int = OBS_DENSITY):
        """One field-level-inference iteration (sim_fli_step): posterior and its gradient at
        `noise`, then an Adam step that updates noise, m, v in place. Returns the loss
        tensor ([1] float64, [B] with B > 1) at the input noise."""
        n, B = self.n, self.B
        for t_, nm in ((noise, "noise"), (m, "m"), (v, "v"), (data, "data")):
            _chk(t_, F32, B * n ** 3, nm)
        if grad is not None:
            _chk(grad, F32, B * n ** 3, "grad")
        loss = torch.empty(B, dtype=F64, device=noise.device) if loss is None else loss
        self._check(lib.sim_fli_step(self.h, observable, _ptr(noise), _ptr(m), _ptr(v), _ptr(data),
                                     sigma_n, lr, t, _ptr(loss), _ptr(grad)), "sim_fli_step")
        return loss

    def posterior(self, noise, data, sigma_n: float, grad=None, loss=None,
                  observable: int = OBS_DENSITY):
        """(loss, dL/dnoise) of the posterior of Sec. 3.2 at `noise` (sim_posterior)."""
        n, B = self.n, self.B
        _chk(noise, F32, B * n ** 3, "noise")
        _chk(data, F32, B * n ** 3, "data")
        grad = torch.empty_like(noise) if grad is None else grad
        loss = torch.empty(B, dtype=F64, device=noise.device) if loss is None else loss
        self._check(lib.sim_posterior(self.h, observable, _ptr(noise), _ptr(data), sigma_n,
                                      _ptr(loss), _ptr(grad)), "sim_posterior")
        return loss, grad

    def loss_field(self, target, c: float, observable: int = OBS_DENSITY, out=None, loss=None):
        """(dL/dgas, loss) of L = c sum (O - target)^2 for an observable O of the state."""
        n, B = self.n, self.B
        _chk(target, F32, B * n ** 3, "target")
        out = torch.empty(self._shape(5, n, n, n), dtype=F32, device=target.device) if out is None else out
        loss = torch.empty(B, dtype=F64, device=target.device) if loss is None else loss
        self._check(lib.sim_loss_field(self.h, observable, _ptr(target), c, _ptr(out), _ptr(loss)),
                    "sim_loss_field")
        return out, loss

    def state(self, gravity: bool = False):
        n = self.n
        sh = self._shape
        dev = torch.device("cuda", torch.cuda.current_device())
        gas = torch.empty(sh(5, n, n, n), dtype=F32, device=dev)
        part = torch.empty(sh(6, n ** 3), dtype=F32, device=dev)
        star = torch.empty(sh(n, n, n), dtype=F32, device=dev)
        aux = torch.empty(sh(n ** 3), dtype=F32, device=dev)
        events = torch.empty(sh((n ** 3 + 31) // 32), dtype=U32, device=dev)
        g = torch.empty(sh(3, n, n, n), dtype=F32, device=dev) if gravity else None
        step = ctypes.c_int32()
        self._check(lib.sim_get_state(self.h, _ptr(gas), _ptr(part), _ptr(star), _ptr(aux),
                                      _ptr(events), _ptr(g), ctypes.byref(step)), "sim_get_state")
        s_, p_ = (part[:3], part[3:]) if self.B == 1 else (part[:, :3], part[:, 3:])
        out = {"gas": gas, "s": s_, "p": p_, "star": star, "aux": aux,
               "events": events, "step": step.value}
        if gravity:
            out["g"] = g
        return out

    def set_state(self, gas, part, step: int):
        n, B = self.n, self.B
        _chk(gas, F32, 5 * B * n ** 3, "gas")
        _chk(part, F32, 6 * B * n ** 3, "part")
        self._check(lib.sim_set_state(self.h, _ptr(gas), _ptr(part), step), "sim_set_state")

    def schedule(self, i: int):
        out = (ctypes.c_double * 6)()
        check(lib.sim_schedule(self.h, i, out), "sim_schedule", self.h)
        return dict(zip(("a0", "a1", "K1", "dtau", "K2", "pref1"), list(out)))

    def cfl(self) -> float:
        c = ctypes.c_double()
        self._check(lib.sim_cfl(self.h, ctypes.byref(c)), "sim_cfl")
        return c.value

    def set_closure(self, closure=None):
        """Apply a learned closure after every step (None: the plain solver)."""
        self._closure = closure
        self._check(lib.sim_set_closure(self.h, closure.h if closure is not None else None),
                    "sim_set_closure")

    def ic_amplitude(self, b: int = 0) -> float:
        c = ctypes.c_double()
        check(lib.sim_ic_amplitude(self.h, b, ctypes.byref(c)), "sim_ic_amplitude", self.h)
        return c.value

    def set_graphs(self, on: bool = True):
        self._check(lib.sim_set_graphs(self.h, int(on)), "sim_set_graphs")

    def set_tape_recording(self, segments: int = 1):
        """Checkpoint segments a run records at its end for the next reverse pass: 1 (the
        default), k, -1 for all (no recompute), 0 for none; see sim_set_tape_recording."""
        self._check(lib.sim_set_tape_recording(self.h, int(segments)), "sim_set_tape_recording")

    def set_sweep_variants(self, fwd=None, adj=None):
        f = (ctypes.c_int32 * 3)(*fwd) if fwd is not None else None
        a = (ctypes.c_int32 * 3)(*adj) if adj is not None else None
        self._check(lib.sim_set_sweep_variants(self.h, f, a), "sim_set_sweep_variants")

    def autotune(self, reps: int = 3):
        """Time the sweep variants on the current state and keep the fastest per axis;
        returns (forward variants, adjoint variants)."""
        f = (ctypes.c_int32 * 3)()
        a = (ctypes.c_int32 * 3)()
        self._check(lib.sim_autotune(self.h, reps, f, a), "sim_autotune")
        return list(f), list(a)

    def kernel_timing(self, on: bool = True):
        self._check(lib.sim_kernel_timing(self.h, int(on)), "sim_kernel_timing")

    def kernel_times(self, reset: bool = True):
        """{class: (total ms, launches)} recorded since the last reset."""
        ms = (ctypes.c_double * KT_N)()
        cnt = (ctypes.c_int64 * KT_N)()
        self._check(lib.sim_kernel_times(self.h, ms, cnt, int(reset)), "sim_kernel_times")
        return {name: (ms[i], cnt[i]) for i, name in enumerate(KT_NAMES)}


def _host_f32(a, count, name):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(-1))
    if a.size != count:
        raise ValueError(f"{name}: expected {count} values, got {a.size}")
    return a


class Closure:
    """Learned per-step correction u <- u + s NN((u - mu) / sigma) (sim_closure_*).
    Weights are a flat float32 vector of CLOSURE_NWEIGHTS values (layout in diffhydro.h)."""

    def __init__(self, weights=None):
        self._stream = torch.cuda.current_stream()
        w = None if weights is None else _host_f32(weights, CLOSURE_NWEIGHTS, "weights")
        h = ctypes.c_void_p()
        check(lib.sim_closure_create(w.ctypes.data if w is not None else None,
                                     ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h)),
              "sim_closure_create")
        self.h = h

    def set_norm(self, mu, sigma, scale):
        m, sg, sc = (_host_f32(v, 5, nm) for v, nm in ((mu, "mu"), (sigma, "sigma"), (scale, "scale")))
        check(lib.sim_closure_set_norm(self.h, m.ctypes.data, sg.ctypes.data, sc.ctypes.data),
              "sim_closure_set_norm")
        self.norm = (m.tolist(), sg.tolist(), sc.tolist())

    def weights(self):
        out = np.empty(CLOSURE_NWEIGHTS, dtype=np.float32)
        check(lib.sim_closure_get_weights(self.h, out.ctypes.data), "sim_closure_get_weights")
        return out

    def set_weights(self, w):
        w = _host_f32(w, CLOSURE_NWEIGHTS, "weights")
        check(lib.sim_closure_set_weights(self.h, w.ctypes.data), "sim_closure_set_weights")

    @staticmethod
    def _dims(gas):
        n = gas.shape[-1]
        B = gas.numel() // (5 * n ** 3)
        _chk(gas, F32, 5 * B * n ** 3, "gas")
        return n, B

    def forward(self, gas):
        n, B = self._dims(gas)
        y = torch.empty_like(gas)
        check(lib.sim_closure_forward(self.h, _ptr(gas), n, B, _ptr(y)), "sim_closure_forward")
        return y

    def apply(self, gas):
        n, B = self._dims(gas)
        check(lib.sim_closure_apply(self.h, _ptr(gas), n, B), "sim_closure_apply")
        return gas

    def gradient(self, gas, target):
        n, B = self._dims(gas)
        _chk(target, F32, 5 * B * n ** 3, "target")
        loss = ctypes.c_double()
        g = np.empty(CLOSURE_NWEIGHTS, dtype=np.float32)
        check(lib.sim_closure_gradient(self.h, _ptr(gas), _ptr(target), n, B, ctypes.byref(loss),
                                       g.ctypes.data), "sim_closure_gradient")
        return loss.value, g

    def train_step(self, gas, target, lr: float, loss_out=None):
        n, B = self._dims(gas)
        _chk(target, F32, 5 * B * n ** 3, "target")
        check(lib.sim_closure_train_step(self.h, _ptr(gas), _ptr(target), n, B, lr,
                                         _ptr(loss_out)), "sim_closure_train_step")

    def status(self):
        check(lib.sim_closure_status(self.h), "sim_closure_status")

    def set_wait_limit(self, ns: int):
        """Time limit of each tensor-core pipeline wait, in nanoseconds (default 1e9)."""
        check(lib.sim_closure_set_wait_limit(self.h, int(ns)), "sim_closure_set_wait_limit")

    def close(self):
        if getattr(self, "h", None):
            lib.sim_closure_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def refine_noise(w_c, n_f: int, scale: float):
    """Band-limited interpolation of coarse white noise onto an n_f^3 grid, times scale."""
    n_c = w_c.shape[-1]
    _chk(w_c, F32, n_c ** 3, "w_c")
    out = torch.empty(n_f, n_f, n_f, dtype=F32, device=w_c.device)
    check(lib.sim_refine_noise(_ptr(w_c), n_c, _ptr(out), n_f, scale, _stream()), "sim_refine_noise")
    return out


def restrict_gas(gas_f):
    """Fine gas [(B,) 5, 2n, 2n, 2n] -> coarse [(B,) 5, n, n, n] (tent weights)."""
    n_f = gas_f.shape[-1]
    B = gas_f.numel() // (5 * n_f ** 3)
    _chk(gas_f, F32, 5 * B * n_f ** 3, "gas_f")
    nc = n_f // 2
    out = torch.empty(gas_f.shape[:-3] + (nc, nc, nc), dtype=F32, device=gas_f.device)
    check(lib.sim_restrict_gas(_ptr(gas_f), n_f, _ptr(out), B, _stream()), "sim_restrict_gas")
    return out


def restrict_particles(part_f, n_f: int):
    """Fine particles [(B,) 6, n_f^3] -> coarse [(B,) 6, (n_f/2)^3] (even lattice sites)."""
    B = part_f.numel() // (6 * n_f ** 3)
    _chk(part_f, F32, 6 * B * n_f ** 3, "part_f")
    out = torch.empty(part_f.shape[:-1] + ((n_f // 2) ** 3,), dtype=F32, device=part_f.device)
    check(lib.sim_restrict_particles(_ptr(part_f), n_f, _ptr(out), B, _stream()),
          "sim_restrict_particles")
    return out


class Group:
    """Member simulations (e.g. one batch per grid size) run as one CUDA graph with a
    concurrent branch per member (sim_group_*). Create the members on the current stream."""

    def __init__(self, sims):
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s_.h.value for s_ in self.sims])
        h = ctypes.c_void_p()
        check(lib.sim_group_create(arr, len(self.sims),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                   ctypes.byref(h)), "sim_group_create")
        self.h = h

    def run(self):
        check(lib.sim_group_run(self.h), "sim_group_run")

    def run_adjoint(self, dL_dgas=None, out=None):
        """dL_dgas: one tensor (or None) per member; returns per-member parameter
        derivatives [B_k, NPARAMS] (or [NPARAMS] for B_k = 1)."""
        K = len(self.sims)
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is None:
            out = [torch.zeros(s_._shape(NPARAMS), dtype=F64, device=dev) for s_ in self.sims]
        g = None
        if dL_dgas is not None:
            for s_, d in zip(self.sims, dL_dgas):
                if d is not None:
                    _chk(d, F32, 5 * s_.B * s_.n ** 3, "dL_dgas")
            g = (ctypes.c_void_p * K)(*[(d.data_ptr() if d is not None else None) for d in dL_dgas])
        o = (ctypes.c_void_p * K)(*[t.data_ptr() for t in out])
        check(lib.sim_group_run_adjoint(self.h, g, o), "sim_group_run_adjoint")
        return out

    def reset(self):
        check(lib.sim_group_reset(self.h), "sim_group_reset")

    def close(self):
        if getattr(self, "h", None):
            lib.sim_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SimRunFunction(torch.autograd.Function):
    """Final gas state [5, n, n, n] of a full run as a differentiable function of the white
    noise [n, n, n] and the parameter vector [NPARAMS] (omega_m, sigma8, delta_c, Pi0, E0,
    T0_uv, gamma_uv). Backward calls sim_run_adjoint (checkpointed recomputation)."""

    @staticmethod
    def forward(ctx, noise, pvec, params: SimParams):
        p = SimParams.from_buffer_copy(params)
        vals = pvec.detach().double().cpu().tolist()
        for name, v in zip(("omega_m", "sigma8", "delta_c", "Pi0", "E0", "T0_uv", "gamma_uv"), vals):
            setattr(p, name, v)
        sim = Simulation(p, noise.detach().float().contiguous())
        sim.run()
        st = sim.state()
        ctx.sim = sim
        ctx.pdev = pvec.device
        return st["gas"]

    @staticmethod
    def backward(ctx, g_gas):
        sim = ctx.sim
        dnoise, dpar = sim.run_adjoint(g_gas.detach().float().contiguous(), None,
                                       want_noise=ctx.needs_input_grad[0])
        sim.close()
        ctx.sim = None
        return dnoise, dpar.to(device=ctx.pdev, dtype=torch.float64), None


def simulate(noise, pvec, params: SimParams):
    return SimRunFunction.apply(noise, pvec, params)


def fli_infer(sim: Simulation, data, sigma_n: float, iters: int, lr: float, noise0=None,
              losses_out=None, observable: int = OBS_DENSITY):
    """Field-level inference (Sec. 3.2): `iters` Adam iterations of sim_fli_step from noise0
    (zeros if None). Returns (amplitudes, per-iteration losses [iters, B] float64 on the
    device). The loop only sequences library calls; no value leaves the device."""
    n, B = sim.n, sim.B
    dev = data.device
    shape = (n, n, n) if B == 1 else (B, n, n, n)
    x = torch.zeros(shape, dtype=F32, device=dev) if noise0 is None else noise0.clone().contiguous()
    m = torch.zeros_like(x)
    v = torch.zeros_like(x)
    losses = torch.empty(iters, B, dtype=F64, device=dev) if losses_out is None else losses_out
    for t in range(1, iters + 1):
        sim.fli_step(x, m, v, data, sigma_n, lr, t, loss=losses[t - 1], observable=observable)
    return x, losses
