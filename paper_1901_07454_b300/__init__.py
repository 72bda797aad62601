"""B300-native batched cable-equation stepper (the hot path of arXiv 1901.07454's method).

The CUDA library libarb_b300.so (sm_103a) does all the work; this package is its binding.
Importing it fails when the library has not been built: there is no CPU fallback.
"""
from . import _lib
from ._lib import ArbError, load, EXPORTED, kernel_variants
from .sim import Plan, Simulation, default_params

load()

from .adjoint import AdjointLoss, adjoint_loss, spread_params  # noqa: E402  (needs the library)
from .autotune import autotune_packing, autotune_streamed  # noqa: E402

__all__ = ["ArbError", "Plan", "Simulation", "default_params", "load", "EXPORTED", "AdjointLoss", "adjoint_loss",
           "spread_params", "autotune_packing", "autotune_streamed", "kernel_variants"]
