"""GB300-native D2Q9 MRT lattice Boltzmann solver for nonlinear anisotropic
convection-diffusion equations (arXiv:1603.09577).

The compute path is liblbm.so (hand-written sm_103a CUDA kernels behind a C
ABI, include/lbm.h); this package marshals arguments and lends torch's device
memory and streams.
"""
from . import adjoint, ensemble, tune  # noqa: F401
from ._lib import LBMError, lib  # noqa: F401
from .ensemble import Ensemble  # noqa: F401
from .solver import Solver  # noqa: F401
from .solver3 import Solver3  # noqa: F401

__all__ = ["Solver", "Solver3", "Ensemble", "LBMError", "lib", "adjoint", "ensemble", "tune"]
