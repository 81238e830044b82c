"""GB300-native generalized-Poisson solver with a dry/wet (FFT / multigrid) split.

Hot path of Sanchez, Sued & Scherlis, arXiv:0904.4887: eps(R) from atoms
(Sec. II.B), div(eps grad phi) = -4 pi rho (Eq. 3) by FP32 multigrid inside
FP64 defect correction, the FFT dry region (Eq. 15, Scheme 1), energy (Eq. 4)
and forces (Eq. 11). The compute runs in ``libgp_gb300.so`` (CUDA, sm_103a);
this package only binds it.
"""
from . import _build  # noqa: F401
from .gp import Context, GPError, default_params, load  # noqa: F401
from .solver import GPSolver, PoissonEnergy, poisson_energy  # noqa: F401

__all__ = ["Context", "GPError", "GPSolver", "PoissonEnergy", "default_params", "load", "poisson_energy"]
