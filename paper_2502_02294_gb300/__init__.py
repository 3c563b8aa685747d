"""GB300-native differentiable cosmological hydro step (arXiv 2502.02294, diffHydro).

The computation lives in libdiffhydro.so (hand-written sm_103a CUDA behind a C ABI,
include/diffhydro.h); this package is its Python binding. Importing it raises ImportError
when the library has not been built: there is no CPU fallback.
"""
from ._lib import (NPARAMS, PARAM_NAMES, SimError, SimParams, default_params, lib)  # noqa: F401
from ._lib import (SIM_ECFL, SIM_EINVAL, SIM_ENAN, SIM_ENOTIMPL, SIM_ETIMEOUT,  # noqa: F401
                   SIM_OK)
from .api import (adam, axpby, cross_correlation, dot, fli_infer, max_signal_speed,  # noqa: F401
                  power_spectrum_adjoint)  # noqa: F401
from ._lib import (OBS_DENSITY, OBS_THERMAL)  # noqa: F401
from .api import (Closure, Group, Simulation, SimRunFunction, refine_noise,  # noqa: F401
                  restrict_gas, restrict_particles, deposit_cic, gravity, gravity_adjoint,  # noqa: F401
                  interp_cic, philox, power_spectrum, simulate, subgrid, subgrid_adjoint,
                  sweep, sweep_adjoint)
