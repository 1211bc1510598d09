"""GB300 (sm_103a) implementation of the well-balanced phase-field lattice
Boltzmann model for incompressible binary fluids (arXiv:2311.10827).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lbm.h``); ``capi`` binds it with the same function names and ``sim``
wraps one context.  ``workloads`` holds seeded initial conditions only.
"""
from . import build, workloads  # noqa: F401

__all__ = ["build", "workloads", "capi", "sim"]
