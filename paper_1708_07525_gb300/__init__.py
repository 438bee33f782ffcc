"""GB300-native implementation of the fused three-lattice step of the REV-scale
MRT lattice Boltzmann model for double-diffusive convection in porous media
(Liu & He, arXiv:1708.07525).  The compute path is liblbm.so (CUDA, sm_103a);
this package holds its ctypes binding, its build script and the workload
generators."""
from . import build  # noqa: F401
