"""Element-Jacobi preconditioner, FP64, test infrastructure only (Sec. 2.3).

The paper preconditions GMRES from the left with the inverse of the diagonal
blocks of (1/(w dt) + 1/dtau_max) I - dR/dq: one dense block per element (all
of the element's DOFs), evaluated once at the start of every physical time
step.  Here the blocks are read off the exact Jacobian by its definition,
J[:, k] = dR(q)[e_k] (``linearize.dense_jacobian``), so only tiny meshes are
practical; the canonical layout keeps each element's DOFs contiguous
(``FR.offsets``).  Left preconditioning is the composition z = M^-1 (A v),
b' = M^-1 b in any GMRES (``krylov.gmres``), with its convergence test on the
preconditioned residual.
"""
import torch

from .linearize import dense_jacobian, jvp


def element_blocks(fr, q, sigma, J=None, elements=None):
    """[(lo, hi, B_e)] with B_e = sigma I - J[lo:hi, lo:hi] for every element
    (J, the dense Jacobian at q, is computed when not given).  With
    ``elements``, only those blocks are formed, column by column from the
    products J e_k with the unit vectors of the element's own DOFs (B_e is
    None for the others)."""
    off = fr.offsets
    out = []
    if elements is not None and J is None:
        keep = set(int(e) for e in elements)
        for e in range(len(off) - 1):
            lo, hi = int(off[e]), int(off[e + 1])
            if e not in keep:
                out.append((lo, hi, None))
                continue
            B = torch.zeros(hi - lo, hi - lo, dtype=q.dtype)
            for k in range(lo, hi):
                u = torch.zeros_like(q)
                u[k] = 1.0
                B[:, k - lo] = -jvp(fr, q, u)[lo:hi]
                B[k - lo, k - lo] += sigma
            out.append((lo, hi, B))
        return out
    if J is None:
        J = dense_jacobian(fr, q)
    for e in range(len(off) - 1):
        lo, hi = int(off[e]), int(off[e + 1])
        out.append((lo, hi, sigma * torch.eye(hi - lo, dtype=J.dtype) - J[lo:hi, lo:hi]))
    return out


def apply_inverse(blocks, w):
    """z = M^-1 w, M the block-diagonal matrix of ``blocks`` (dense solves; NaN
    on elements whose block was not formed)."""
    z = torch.full_like(w, float("nan"))
    for lo, hi, B in blocks:
        if B is not None:
            z[lo:hi] = torch.linalg.solve(B, w[lo:hi])
    return z
