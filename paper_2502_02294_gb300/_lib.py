"""ctypes binding of ``libdiffhydro.so`` (C ABI declared in include/diffhydro.h).

Argument marshalling only: every step of the simulation runs in the library's CUDA
kernels. Arrays are torch CUDA tensors (float32 / uint32 / float64, contiguous) whose
device pointers are passed straight through, on torch's current CUDA stream. There is no
CPU fallback: importing this module raises if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdiffhydro.so")

SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_ECFL, SIM_ENAN, SIM_ETIMEOUT, SIM_ENOTIMPL = range(8)
STATUS_NAMES = ["SIM_OK", "SIM_EINVAL", "SIM_ENOMEM", "SIM_ECUDA", "SIM_ECFL", "SIM_ENAN",
                "SIM_ETIMEOUT", "SIM_ENOTIMPL"]
P_OMEGA_M, P_SIGMA8, P_DELTA_C, P_PI0, P_E0, P_T0_UV, P_GAMMA_UV, NPARAMS = range(8)
KT_NAMES = ("sweep", "sweep_adjoint", "kick", "kick_adjoint", "deposit", "deposit_adjoint",
            "poisson", "poisson_adjoint", "subgrid", "subgrid_adjoint")
KT_N = len(KT_NAMES)
KT_SWEEP, KT_SWEEP_ADJOINT = 0, 1
SWEEP_DEFAULT, SWEEP_TILE, SWEEP_MARCH32, SWEEP_MARCH16, SWEEP_MARCH_FIT = range(5)
CLOSURE_NWEIGHTS = 18197
PARAM_NAMES = ["omega_m", "sigma8", "delta_c", "Pi0", "E0", "T0_uv", "gamma_uv"]
DG_NAMES = ("a", "mass", "mx", "my", "mz", "energy", "px", "py", "pz", "stars", "events",
            "nonfinite", "rho_min", "p_min")
DG_N = len(DG_NAMES)
OBS_DENSITY, OBS_THERMAL = 0, 1


class SimParams(ctypes.Structure):
    """Mirror of the C struct sim_params (field order and types must match the header)."""
    _fields_ = [
        ("n", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("ckpt_every", ctypes.c_int32),
        ("subgrid_on", ctypes.c_int32), ("gravity_on", ctypes.c_int32),
        ("hydro_on", ctypes.c_int32), ("kdk_mode", ctypes.c_int32), ("instance", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("box", ctypes.c_double), ("omega_m", ctypes.c_double), ("omega_b", ctypes.c_double),
        ("h", ctypes.c_double), ("sigma8", ctypes.c_double), ("gamma", ctypes.c_double),
        ("mu", ctypes.c_double), ("T_init", ctypes.c_double), ("a_start", ctypes.c_double),
        ("a_end", ctypes.c_double), ("delta_c", ctypes.c_double), ("Pi0", ctypes.c_double),
        ("E0", ctypes.c_double), ("T_c", ctypes.c_double), ("w_delta", ctypes.c_double),
        ("w_T", ctypes.c_double), ("tau", ctypes.c_double), ("T0_uv", ctypes.c_double),
        ("gamma_uv", ctypes.c_double), ("rms_ref", ctypes.c_double), ("a_ref", ctypes.c_double),
        ("sigma8_ref", ctypes.c_double), ("omega_m_ref", ctypes.c_double),
        ("kc_frac", ctypes.c_double), ("limiter_eps", ctypes.c_double),
        ("cfl_max", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_P = ctypes.c_void_p
_I32, _I64, _U32, _U64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
_PP = ctypes.POINTER(SimParams)

# name -> (restype, argtypes)
SIGNATURES = {
    "sim_params_default": (ctypes.c_int, [_PP]),
    "sim_last_error": (ctypes.c_char_p, [_P]),
    "sim_kernel_launches": (ctypes.c_int64, []),
    "sim_init": (ctypes.c_int, [_PP, _P, _P, ctypes.POINTER(_P)]),
    "sim_init_batch": (ctypes.c_int, [_PP, _I32, _P, _P, ctypes.POINTER(_P)]),
    "sim_batch_size": (ctypes.c_int32, [_P]),
    "sim_set_params": (ctypes.c_int, [_P, _PP]),
    "sim_set_sweep_variants": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "sim_autotune": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "sim_destroy": (None, [_P]),
    "sim_closure_create": (ctypes.c_int, [_P, _P, ctypes.POINTER(_P)]),
    "sim_closure_destroy": (None, [_P]),
    "sim_closure_set_norm": (ctypes.c_int, [_P, _P, _P, _P]),
    "sim_closure_get_weights": (ctypes.c_int, [_P, _P]),
    "sim_closure_set_weights": (ctypes.c_int, [_P, _P]),
    "sim_closure_forward": (ctypes.c_int, [_P, _P, _I32, _I32, _P]),
    "sim_closure_apply": (ctypes.c_int, [_P, _P, _I32, _I32]),
    "sim_closure_gradient": (ctypes.c_int, [_P, _P, _P, _I32, _I32, _P, _P]),
    "sim_closure_train_step": (ctypes.c_int, [_P, _P, _P, _I32, _I32, _D, _P]),
    "sim_closure_status": (ctypes.c_int, [_P]),
    "sim_closure_set_wait_limit": (ctypes.c_int, [_P, _I64]),
    "sim_set_closure": (ctypes.c_int, [_P, _P]),
    "sim_refine_noise": (ctypes.c_int, [_P, _I32, _P, _I32, _D, _P]),
    "sim_restrict_gas": (ctypes.c_int, [_P, _I32, _P, _I32, _P]),
    "sim_restrict_particles": (ctypes.c_int, [_P, _I32, _P, _I32, _P]),
    "sim_ic_amplitude": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_D)]),
    "sim_group_create": (ctypes.c_int, [ctypes.POINTER(_P), _I32, _P, ctypes.POINTER(_P)]),
    "sim_group_run": (ctypes.c_int, [_P]),
    "sim_group_run_adjoint": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "sim_group_reset": (ctypes.c_int, [_P]),
    "sim_group_destroy": (None, [_P]),
    "sim_set_graphs": (ctypes.c_int, [_P, _I32]),
    "sim_set_tape_recording": (ctypes.c_int, [_P, _I32]),
    "sim_kernel_timing": (ctypes.c_int, [_P, _I32]),
    "sim_kernel_times": (ctypes.c_int, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I64), _I32]),
    "sim_step": (ctypes.c_int, [_P]),
    "sim_step_adjoint": (ctypes.c_int, [_P, _P, _P, _P]),
    "sim_run": (ctypes.c_int, [_P, _I32]),
    "sim_run_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "sim_reset": (ctypes.c_int, [_P]),
    "sim_reinit": (ctypes.c_int, [_P, _P]),
    "sim_loss_density": (ctypes.c_int, [_P, _P, _D, _P, _P]),
    "sim_get_state": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_I32)]),
    "sim_set_state": (ctypes.c_int, [_P, _P, _P, _I32]),
    "sim_schedule": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_D)]),
    "sim_cfl": (ctypes.c_int, [_P, ctypes.POINTER(_D)]),
    "sim_sweep": (ctypes.c_int, [_P, _P, _I32, _I32, _D, _D, _D, _I32, _P]),
    "sim_sweep_adjoint": (ctypes.c_int, [_P, _P, _P, _I32, _I32, _D, _D, _D, _P, _I32, _P]),
    "sim_max_signal_speed": (ctypes.c_int, [_P, _I32, _D, _P, _P]),
    "sim_deposit_cic": (ctypes.c_int, [_P, _P, _I32, _D, _P, _P]),
    "sim_deposit_cic_static": (ctypes.c_int, [_P, _P, _I32, _D, _P, _P]),
    "sim_interp_cic": (ctypes.c_int, [_P, _I32, _I32, _D, _P, _P, _P]),
    "sim_gravity": (ctypes.c_int, [_P, _I32, _D, _D, _P, _P]),
    "sim_gravity_adjoint": (ctypes.c_int, [_P, _I32, _D, _D, _P, _P]),
    "sim_subgrid": (ctypes.c_int, [_P, _I32, _D, _PP, _I32, _P, _P, _P]),
    "sim_subgrid_adjoint": (ctypes.c_int, [_P, _P, _I32, _D, _PP, _I32, _P, _P, _P]),
    "sim_philox": (ctypes.c_int, [_U64, _U32, _U32, _U32, _I64, _P, _P]),
    "sim_power_spectrum": (ctypes.c_int, [_P, _P, _I32, _D, _I32, _P, _P, _P, _P]),
    "sim_set_diagnostics": (ctypes.c_int, [_P, _I32]),
    "sim_diagnostics": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_D)]),
    "sim_fli_step": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P, _D, _D, _I32, _P, _P]),
    "sim_posterior": (ctypes.c_int, [_P, _I32, _P, _P, _D, _P, _P]),
    "sim_loss_field": (ctypes.c_int, [_P, _I32, _P, _D, _P, _P]),
    "sim_dot": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "sim_axpby": (ctypes.c_int, [_D, _P, _D, _P, _I64, _P]),
    "sim_adam": (ctypes.c_int, [_P, _P, _P, _P, _I64, _D, _D, _D, _D, _I32, _D, _P, _P, _P]),
    "sim_power_spectrum_adjoint": (ctypes.c_int, [_P, _I32, _D, _I32, _P, _P, _P]),
    "sim_cross_correlation": (ctypes.c_int, [_P, _P, _I32, _D, _I32, _P, _P, _P, _P]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python paper_2502_02294_gb300/build.py or __graft_entry__.build()). "
            "There is no CPU fallback.")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


class SimError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")


def check(status: int, where: str, handle=None):
    if status != SIM_OK:
        msg = lib.sim_last_error(handle)
        raise SimError(status, where, msg.decode() if msg else "")


def default_params(**overrides) -> SimParams:
    p = SimParams()
    check(lib.sim_params_default(ctypes.byref(p)), "sim_params_default")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p
