"""GB300-native hot path of a p-adaptive implicit flux-reconstruction solver.

The FR residual of the compressible Euler/Navier-Stokes equations on elements
of mixed polynomial degree, its exact JVP and VJP, the finite-difference Jv,
restarted GMRES, ESDIRK stages by pseudo-transient continuation, and the
spectral-decay p-adaptation with on-device rebucketing (arXiv:1910.03693,
Secs. 2-3), as hand-written CUDA kernels for sm_103a behind a C ABI
(``include/fr.h``).  This Python layer only marshals arguments.
"""
from .api import FRContext, FRError, autograd_residual, dfloat_eval, esdirk_tableau, fma_rate  # noqa: F401
