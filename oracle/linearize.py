"""Linearisations of the FR residual, FP64, test infrastructure only.

* ``fd_jv``: the paper's matrix-free product (Sec. 2.3, unnumbered equation
  after Eq. ser): J v ~ (R(q + eps v) - R(q)) / eps with eps = 1e-6 and no
  scaling of v.
* ``jvp`` / ``vjp``: the exact directional derivative dR(q)[v] and its
  transpose dR(q)^T[w] by their definitions, evaluated with PyTorch's
  automatic differentiation of the oracle residual (a library primitive).
"""
import torch
from torch.func import jvp as _jvp


def fd_jv(fr, q, v, eps=1e-6, R0=None):
    if R0 is None:
        R0 = fr.residual(q)
    return (fr.residual(q + eps * v) - R0) / eps


def jvp(fr, q, v):
    return _jvp(fr.residual, (q,), (v,))[1]


def vjp(fr, q, w):
    q = q.detach().clone().requires_grad_(True)
    R = fr.residual(q)
    (g,) = torch.autograd.grad(R, q, w)
    return g


def dense_jacobian(fr, q):
    """J[:, k] = dR(q)[e_k]; only for tiny systems."""
    n = q.numel()
    cols = []
    for k in range(n):
        e = torch.zeros(n)
        e[k] = 1.0
        cols.append(jvp(fr, q, e))
    return torch.stack(cols, dim=1)
