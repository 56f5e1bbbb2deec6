"""GB300-native electrostatic particle-particle (PP) electron-bunch expansion.

Direct O(N^2) Coulomb sum with the Velocity-Verlet push (arXiv 2502.10640, Sec. 2.1),
as hand-written sm_103a CUDA kernels behind the C ABI of include/pp.h.  The ctypes
binding (module ``capi``) re-exports that ABI under the same names; they are loaded on
first use so that importing the package (for example for ``workloads``) needs no GPU.
"""
from __future__ import annotations

import importlib

_CAPI_NAMES = {
    "pp_create", "pp_set_option", "pp_load_particles", "pp_compute_fields", "pp_step",
    "pp_diagnostics", "pp_get_particles", "pp_get_state", "pp_set_state", "pp_get_n",
    "pp_destroy", "pp_last_error", "pp_version", "pp_pairs_per_step", "PPError",
    "Simulation",
}


def __getattr__(name):
    if name in _CAPI_NAMES or name.startswith("PP_"):
        capi = importlib.import_module(".capi", __name__)
        return getattr(capi, name)
    raise AttributeError(name)
