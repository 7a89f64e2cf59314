"""Element maps and metric terms, FP64, test infrastructure only.

Tensors of one degree-p element group are laid out ``[E, ..., (P,)*nd]`` with
the spatial axes ordered (zeta, eta, xi): reference direction d lives on tensor
axis ``-1-d``.  The metric terms are S[d][j] = |J| d(xi_d)/d(x_j) (the
contravariant vectors scaled by |J|), in cross-product form from the
derivatives of the degree-p interpolant X of the element map: in 2D
S_xi = (y_eta, -x_eta), S_eta = (-y_xi, x_xi); in 3D S_i = dX/dxi_j x dX/dxi_k
for (i, j, k) cyclic.  The discrete metric identities sum_d D_d S_d = 0, and
with them free-stream preservation, hold in 2D and for affine and extruded
hexahedra (every 3D mesh here); general curved hexahedra would need Kopriva's
(2006) conservative curl form instead.
"""
import torch

from .basis import basis, lagrange


def apply1d(M: torch.Tensor, t: torch.Tensor, d: int) -> torch.Tensor:
    """Apply the 1D operator M [n_out, P] along reference direction d of ``t``."""
    ax = t.dim() - 1 - d
    t2 = torch.movedim(t, ax, -1)
    return torch.movedim(t2 @ M.T, -1, ax)


def face_trace(t: torch.Tensor, b, d: int, s: int, nd: int) -> torch.Tensor:
    """Value at face (d, s) of the polynomial through the solution points along d.

    Returns ``[..., nfp]`` with face points in face-local order (first
    tangential direction fastest)."""
    out = apply1d(b.ext[s:s + 1], t, d)
    out = out.squeeze(t.dim() - 1 - d)
    return out.reshape(out.shape[: out.dim() - (nd - 1)] + (-1,))


def node_map(nodes: torch.Tensor, geom_order: int, p: int, nd: int) -> torch.Tensor:
    """Physical coordinates of the solution points: [E, nd(component), (P,)*nd]."""
    nn = geom_order + 1
    b = basis(p)
    equi = torch.linspace(-1.0, 1.0, nn, dtype=torch.float64)
    N1 = lagrange(equi, b.x)                            # [P, nn]
    E = nodes.shape[0]
    X = nodes.permute(0, 2, 1).reshape((E, nd) + (nn,) * nd)
    for d in range(nd):
        X = apply1d(N1, X, d)
    return X


class ElementGeometry:
    """Metric terms of one group of elements sharing the degree p."""

    def __init__(self, nodes: torch.Tensor, geom_order: int, p: int, nd: int):
        self.p, self.nd = p, nd
        b = self.b = basis(p)
        X = self.X = node_map(nodes, geom_order, p, nd)          # [E, nd, sp]
        dX = [apply1d(b.D, X, d) for d in range(nd)]             # dX[d][:, comp] = dX_comp/dxi_d
        if nd == 2:
            x_xi, y_xi = dX[0][:, 0], dX[0][:, 1]
            x_et, y_et = dX[1][:, 0], dX[1][:, 1]
            S0 = torch.stack([y_et, -x_et], dim=1)
            S1 = torch.stack([-y_xi, x_xi], dim=1)
            self.S = torch.stack([S0, S1], dim=1)                # [E, d, j, sp]
            self.J = x_xi * y_et - x_et * y_xi
        else:
            # S_i = dX/dxi_j x dX/dxi_k, (i, j, k) cyclic
            rows = []
            for i in range(3):
                j, k = (i + 1) % 3, (i + 2) % 3
                A, B = dX[j], dX[k]
                rows.append(torch.stack([A[:, 1] * B[:, 2] - A[:, 2] * B[:, 1],
                                         A[:, 2] * B[:, 0] - A[:, 0] * B[:, 2],
                                         A[:, 0] * B[:, 1] - A[:, 1] * B[:, 0]], dim=1))
            self.S = torch.stack(rows, dim=1)
            a = [[dX[d][:, c] for d in range(3)] for c in range(3)]  # a[comp][d]
            self.J = (a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1])
                      - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
                      + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]))
        # metric terms and |J| at every face: Sf [E, 2nd, d, j, nfp], Jf [E, 2nd, nfp]
        Sf, Jf = [], []
        for d in range(nd):
            for s in (0, 1):
                Sf.append(face_trace(self.S, b, d, s, nd))
                Jf.append(face_trace(self.J, b, d, s, nd))
        self.Sf = torch.stack(Sf, dim=1)
        self.Jf = torch.stack(Jf, dim=1)
