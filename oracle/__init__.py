"""Plain FP64 CPU oracle of the p-adaptive implicit flux-reconstruction hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call or
execute anything here; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` do.  The oracle shares no code with the CUDA
library: it takes its inputs from ``cases`` (seeded generators) and follows the
paper step by step in plain PyTorch CPU float64 operations, vectorised over the
elements of equal polynomial degree but otherwise without blocking, fusion or
reordering.

Modules
  basis      Gauss-Legendre points, Lagrange operators, DG (Radau) correction
             derivatives, Legendre Vandermonde matrices (Sec. 2.2).
  geometry   element maps, metric terms |J| grad(xi_d) at solution and flux
             points (cross-product form from the interpolated map).
  physics    Euler / Navier-Stokes fluxes (Sec. 2.1), Rusanov common flux,
             scalar linear advection (for the FR = DG check).
  fr         the FR residual R(q) = -div f with common fluxes, BR2 common
             gradient, mortars between elements of different degree, wall and
             far-field boundaries (Sec. 2.2, Eq. FR_diff, Eqs. com_q, com_grad_q).
  linearize  finite-difference Jv (Sec. 2.3), exact JVP and VJP (definition:
             directional derivative / transpose, by automatic differentiation
             of ``fr``).
  krylov     restarted GMRES(m) with modified Gram-Schmidt and Givens
             rotations (Sec. 2.3).
  esdirk     ESDIRK tableaus, stage residual F (Eq. ESDIRK_conservative),
             pseudo-transient continuation with SER (Eqs. pseudo_transient,
             linearized_pseudo_transient_final, ser).
  adapt      spectral-decay indicator (Sec. 3.1), p decision, neighbour
             smoothing, prolongation / projection, bucket order.
  dg         direct nodal DG discretisations (linear advection; scalar
             diffusion with the BR2 lifting) used only to check FR with the DG
             correction against DG.

Readings where the paper is silent are listed in the repository's design notes
and repeated in each function's docstring.
"""
import torch

torch.set_default_dtype(torch.float64)
