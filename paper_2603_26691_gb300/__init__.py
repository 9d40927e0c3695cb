"""GB300-native per-particle Lagrangian step of a two-way coupled Euler-Lagrange method
(SCALE-TRACK, arXiv 2603.26691): trilinear gather, Stokes drag + gravity by the exponential
integrator, relocation, deterministic per-cell momentum deposit, and a stable counting sort,
as hand-written CUDA for sm_103a behind a C ABI (include/scaletrack.h).

The CUDA library must be built (``__graft_entry__.build()``); importing ``Sim`` loads it and
raises if it is missing.
"""
from . import inputs  # noqa: F401  (numpy-only input generators)

__all__ = ["Sim", "StError", "inputs"]


def __getattr__(name):
    if name in ("Sim", "StError"):
        from .sim import Sim, StError
        return {"Sim": Sim, "StError": StError}[name]
    raise AttributeError(name)
