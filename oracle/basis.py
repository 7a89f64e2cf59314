"""One-dimensional FR building blocks (Sec. 2.2), FP64, test infrastructure only.

Solution points are the P = p+1 Gauss-Legendre points of [-1, 1]; the flux is
interpolated by the Lagrange polynomial through them; the correction functions
are the left and right Radau polynomials of degree p+1 ("g_DG"), for which FR
reproduces nodal DG with Gauss collocation.
"""
import math

import torch


def legendre(n: int, x: torch.Tensor):
    """Legendre polynomial P_n(x) and its derivative by the three-term recurrence."""
    x = torch.as_tensor(x, dtype=torch.float64)
    p0 = torch.ones_like(x)
    d0 = torch.zeros_like(x)
    if n == 0:
        return p0, d0
    p1 = x.clone()
    d1 = torch.ones_like(x)
    for k in range(1, n):
        # (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};  P'_{k+1} = P'_{k-1} + (2k+1) P_k
        p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        d2 = d0 + (2 * k + 1) * p1
        p0, p1 = p1, p2
        d0, d1 = d1, d2
    return p1, d1


def gauss_points(P: int):
    """Gauss-Legendre points (ascending) and weights on [-1, 1] by Newton on P_P."""
    i = torch.arange(1, P + 1, dtype=torch.float64)
    x = torch.cos(math.pi * (4 * i - 1) / (4 * P + 2))
    for _ in range(100):
        pn, dn = legendre(P, x)
        dx = pn / dn
        x = x - dx
        if float(dx.abs().max()) < 1e-16:
            break
    pn, dn = legendre(P, x)
    w = 2.0 / ((1.0 - x * x) * dn * dn)
    order = torch.argsort(x)
    return x[order].contiguous(), w[order].contiguous()


def lagrange(xs: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """Matrix L[i, k] = l_k(x_i) of the Lagrange basis through the nodes ``xs``."""
    xs = torch.as_tensor(xs, dtype=torch.float64)
    x = torch.as_tensor(x, dtype=torch.float64).reshape(-1)
    n = len(xs)
    L = torch.ones(len(x), n, dtype=torch.float64)
    for k in range(n):
        for m in range(n):
            if m != k:
                L[:, k] = L[:, k] * (x - xs[m]) / (xs[k] - xs[m])
    return L


def lagrange_deriv(xs: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """Matrix D[i, k] = l_k'(x_i) (product rule over the factors of l_k)."""
    xs = torch.as_tensor(xs, dtype=torch.float64)
    x = torch.as_tensor(x, dtype=torch.float64).reshape(-1)
    n = len(xs)
    D = torch.zeros(len(x), n, dtype=torch.float64)
    for k in range(n):
        for j in range(n):
            if j == k:
                continue
            term = torch.full_like(x, 1.0 / (xs[k] - xs[j]))
            for m in range(n):
                if m != k and m != j:
                    term = term * (x - xs[m]) / (xs[k] - xs[m])
            D[:, k] = D[:, k] + term
    return D


def radau_dg(p: int, x: torch.Tensor):
    """Left/right DG correction functions and derivatives at ``x``.

    g_L = (-1)^p/2 (P_p - P_{p+1}) (g_L(-1) = 1, g_L(1) = 0) and
    g_R = (P_p + P_{p+1})/2 (g_R(-1) = 0, g_R(1) = 1).
    Returns (gL, gR, dgL, dgR).
    """
    Pp, dPp = legendre(p, x)
    Pq, dPq = legendre(p + 1, x)
    sgn = (-1.0) ** p
    gL = 0.5 * sgn * (Pp - Pq)
    gR = 0.5 * (Pp + Pq)
    return gL, gR, 0.5 * sgn * (dPp - dPq), 0.5 * (dPp + dPq)


def legendre_vandermonde(xs: torch.Tensor, n: int) -> torch.Tensor:
    """V[i, m] = P_m(x_i) for m < n."""
    cols = [legendre(m, xs)[0] for m in range(n)]
    return torch.stack(cols, dim=1)


class Basis1D:
    """All 1D operators for polynomial degree p (P = p+1 Gauss points)."""

    def __init__(self, p: int):
        self.p = p
        self.P = P = p + 1
        self.x, self.w = gauss_points(P)
        self.D = lagrange_deriv(self.x, self.x)                 # [P, P]
        ends = torch.tensor([-1.0, 1.0], dtype=torch.float64)
        self.ext = lagrange(self.x, ends)                       # [2, P]: row 0 -> xi=-1, row 1 -> xi=+1
        self.dext = lagrange_deriv(self.x, ends)                # [2, P]: derivative at the ends
        gL, gR, dgL, dgR = radau_dg(p, self.x)
        self.dg = torch.stack([dgL, dgR])                      # [2, P]: g_L', g_R' at solution points
        _, _, dgLe, dgRe = radau_dg(p, ends)
        # g_s' evaluated at its own face: g_L'(-1) and g_R'(+1)
        self.dg_face = torch.tensor([float(dgLe[0]), float(dgRe[1])])
        # modal transform: nodal -> Legendre coefficients (exact by Gauss quadrature)
        V = legendre_vandermonde(self.x, P)                     # [P, P]
        norm = torch.tensor([2.0 / (2 * m + 1) for m in range(P)])
        self.to_modal = (V * self.w[:, None]).T / norm[:, None]  # c_m = sum_i w_i P_m(x_i) s_i / ||P_m||^2
        self.to_nodal = V                                        # s_i = sum_m c_m P_m(x_i)


_CACHE = {}


def basis(p: int) -> Basis1D:
    if p not in _CACHE:
        _CACHE[p] = Basis1D(p)
    return _CACHE[p]


def mortar_ops(ps: int, pm: int):
    """Interpolation from degree-ps face points to degree-pm mortar points and the
    L2 projection back: I [Pm, Ps], Pi [Ps, Pm] with Pi[a, m] = w_m l_a(x_m) / w_a."""
    bs, bm = basis(ps), basis(pm)
    I = lagrange(bs.x, bm.x)
    Pi = (bm.w[None, :] * I.T) / bs.w[:, None]
    return I, Pi
