"""GB300-native MRT lattice Boltzmann solver for nonlinear anisotropic
convection-diffusion equations (arXiv:1603.09577).

The compute path is liblbm.so: hand-written sm_103a CUDA kernels behind a C ABI
(include/lbm.h for D2Q9, include/lbm3.h for D3Q19). This package marshals
arguments and lends torch's device memory and streams:

  Solver    one D2Q9 lattice: Scheme B or A, periodic / anti-bounce-back /
            extrapolated walls, FP64 / FP32 / BF16-shifted storage, one or two
            steps per sweep, CUDA-graph capture and replay
  Solver3   one periodic D3Q19 lattice
  Ensemble  hundreds of independent D2Q9 lattices in one launch per step
  adjoint   the discrete adjoint behind torch.autograd (gradients in K(x), u, phi0)
  tune      the launch-configuration autotuner
"""
from . import adjoint, ensemble, tune  # noqa: F401
from ._lib import LBMError, lib  # noqa: F401
from .ensemble import Ensemble  # noqa: F401
from .solver import Solver  # noqa: F401
from .solver3 import Solver3  # noqa: F401

__all__ = ["Solver", "Solver3", "Ensemble", "LBMError", "lib", "adjoint", "ensemble", "tune"]
