"""The C-ABI library loads and exports every entry point declared in include/diffhydro.h;
the ctypes mirror of sim_params matches the C layout; argument checks that run before any
device call reject bad input. No GPU is needed (no compute call is made)."""
import ctypes
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "diffhydro.h")


@pytest.fixture(scope="module")
def dh():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2502_02294_gb300 as m
    return m


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(dh):
    names = _declared()
    assert len(names) >= 20
    lib = ctypes.CDLL(dh._lib.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a signature for every entry point
    assert sorted(dh._lib.SIGNATURES) == names


def test_params_struct_layout_matches_c(dh):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    fields = [f for f, _ in dh.SimParams._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "diffhydro.h"', "int main(void){",
           'printf("%zu\\n", sizeof(sim_params));']
    src += [f'printf("%zu\\n", offsetof(sim_params, {f}));' for f in fields]
    src += ["return 0;}"]
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write("\n".join(src))
        subprocess.run([gcc, "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                              check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(dh.SimParams)
    assert out[1:] == [getattr(dh.SimParams, f).offset for f in fields]


def test_defaults(dh):
    p = dh.default_params()
    assert (p.n, p.n_steps, p.ckpt_every, p.gravity_on, p.hydro_on) == (32, 20, 6, 1, 1)
    assert p.box == 32.0 and p.omega_m == 0.3 and abs(p.gamma - 5 / 3) < 1e-15
    assert p.tau == 0.1 and p.kc_frac == 0.5 and p.rms_ref == 0.05


@pytest.mark.parametrize("field,value", [("n", 2), ("n_steps", 0), ("box", -1.0),
                                         ("omega_b", 0.5), ("a_end", 0.05), ("kdk_mode", 7)])
def test_invalid_params_rejected_before_device_work(dh, field, value):
    p = dh.default_params(**{field: value})
    h = ctypes.c_void_p()
    st = dh.lib.sim_init(ctypes.byref(p), None, None, ctypes.byref(h))
    assert st == dh._lib.SIM_EINVAL
    assert h.value is None
    assert dh.lib.sim_last_error(None)


def test_null_arguments_rejected(dh):
    L = dh.lib
    assert L.sim_sweep(None, None, 8, 0, 0.1, 5 / 3, 1e-30, 0, None) == dh._lib.SIM_EINVAL
    assert L.sim_deposit_cic(None, None, 8, 8.0, None, None) == dh._lib.SIM_EINVAL
    assert L.sim_power_spectrum(None, None, 8, 8.0, 4, None, None, None, None) == dh._lib.SIM_EINVAL
    assert L.sim_step(None) == dh._lib.SIM_EINVAL
    assert L.sim_kernel_timing(None, 1) == dh._lib.SIM_EINVAL
    assert L.sim_kernel_times(None, None, None, 0) == dh._lib.SIM_EINVAL
    L.sim_destroy(None)  # ignored
    E = dh._lib.SIM_EINVAL
    # the entry points of field-level inference, diagnostics and validation runs
    assert L.sim_fli_step(None, 0, None, None, None, None, 0.1, 0.01, 1, None, None) == E
    assert L.sim_posterior(None, 0, None, None, 0.1, None, None) == E
    assert L.sim_loss_field(None, 0, None, 1.0, None, None) == E
    assert L.sim_adam(None, None, None, None, 8, 0.1, 0.9, 0.999, 1e-8, 1, 0.0, None, None, None) == E
    assert L.sim_dot(None, None, 8, None, None) == E
    assert L.sim_axpby(1.0, None, 1.0, None, 8, None) == E
    assert L.sim_cross_correlation(None, None, 8, 8.0, 4, None, None, None, None) == E
    assert L.sim_power_spectrum_adjoint(None, 8, 8.0, 4, None, None, None) == E
    assert L.sim_max_signal_speed(None, 8, 5 / 3, None, None) == E
    assert L.sim_set_params(None, None) == E
    assert L.sim_set_diagnostics(None, 1) == E
    assert L.sim_diagnostics(None, 0, None) == E
    assert L.sim_closure_set_wait_limit(None, 0) == E
    assert L.sim_deposit_cic_static(None, None, 8, 8.0, None, None) == E
    assert L.sim_set_tape_recording(None, 1) == E


def test_no_unresolved_library_symbols(dh):
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--undefined-only", dh._lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    ours = [ln for ln in out.splitlines() if "_ZN2dh" in ln or " sim_" in ln]
    assert not ours, ours
