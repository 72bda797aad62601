"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only draws random morphologies, mechanism placements, connectivity and
Poisson event trains, and returns them as plain NumPy arrays. It holds none of the
method's arithmetic: no discretisation, no conductances, no time stepping.
"""
from .model import Model, SimSpec
from .configs import make_config, config_names, small_tree_model, uniform_cable_model

__all__ = ["Model", "SimSpec", "make_config", "config_names", "small_tree_model", "uniform_cable_model"]
