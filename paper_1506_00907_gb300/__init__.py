"""GB300 (sm_103a) nodal discontinuous-Galerkin RTM library: CUDA kernels behind a C ABI
(``include/ridg.h``), with this thin ctypes binding.  See ``ridg.Solver``."""

from . import ridg  # noqa: F401
from .ridg import Mesh, Solver, RidgError, reference_operators  # noqa: F401
