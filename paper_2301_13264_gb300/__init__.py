"""GB300 library for biorthonormal CCSD non-adiabatic derivative couplings.

The computation lives in the CUDA library libccsd_gb300.so (C ABI declared in
include/ccsd.h); :mod:`.binding` loads it with ctypes.  :mod:`.synth` draws
seeded synthetic Hamiltonians.  The binding is imported on first use of one of
its names, so that importing :mod:`.synth` alone loads nothing of the library.
"""
import importlib

_BINDING_NAMES = (
    "CCSDError", "ccsd_coupling_densities", "ccsd_create", "ccsd_default_options", "ccsd_derivative_coupling",
    "ccsd_describe_program", "ccsd_destroy", "ccsd_get_amplitudes", "ccsd_get_states", "ccsd_guess_features",
    "ccsd_jacobian_transform", "ccsd_mlp_gradient", "ccsd_mlp_predict", "ccsd_mlp_train", "ccsd_residual",
    "ccsd_set_amplitudes", "ccsd_set_guess_model", "ccsd_solve_ground", "ccsd_stats", "eom_solve_left",
    "eom_solve_right", "vector_dim",
)
__all__ = list(_BINDING_NAMES)


def __getattr__(name):
    if name in _BINDING_NAMES:
        return getattr(importlib.import_module(".binding", __name__), name)
    if name in ("binding", "synth", "learned_guess", "build"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
