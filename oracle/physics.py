"""Pointwise physics (Sec. 2.1), FP64, test infrastructure only.

Layout: the variable axis is dim 1 of every state tensor ``q [N, nv, ...]``;
fluxes are ``[N, nd(j), nv, ...]`` with j the physical direction.
"""
import torch


class Euler:
    """Compressible Euler / Navier-Stokes with constant mu and Pr.

    q = (rho, rho u_i, rho E); E = (p/rho)/(gamma-1) + u.u/2; f_j inviscid =
    (rho u_j, rho u_i u_j + p delta_ij, (rho E + p) u_j).  Viscous flux
    (tau_ij, u_i tau_ij - K_j) with tau = 2 mu (S - div(u)/3 I) and
    K = -mu C_p/Pr grad T = -mu gamma/((gamma-1) Pr) grad(p/rho).
    """

    def __init__(self, nd, gamma=1.4, mu=0.0, Pr=0.72, q_inf=None):
        self.nd, self.nv = nd, nd + 2
        self.gamma, self.mu, self.Pr = float(gamma), float(mu), float(Pr)
        self.viscous = self.mu > 0.0
        self.q_inf = None if q_inf is None else torch.as_tensor(q_inf, dtype=torch.float64)

    # -- inviscid -------------------------------------------------------------
    def primitives(self, q):
        nd, g = self.nd, self.gamma
        rho = q[:, 0]
        vel = q[:, 1:1 + nd] / rho[:, None]
        pres = (g - 1.0) * (q[:, nd + 1] - 0.5 * rho * (vel * vel).sum(1))
        return rho, vel, pres

    def flux(self, q):
        nd = self.nd
        rho, vel, pres = self.primitives(q)
        rows = []
        for j in range(nd):
            comps = [q[:, 1 + j]]
            for i in range(nd):
                fij = q[:, 1 + i] * vel[:, j]
                if i == j:
                    fij = fij + pres
                comps.append(fij)
            comps.append((q[:, nd + 1] + pres) * vel[:, j])
            rows.append(torch.stack(comps, dim=1))
        return torch.stack(rows, dim=1)

    def wave_speed(self, q, n):
        """|u.n| + c for unit normals ``n [N, nd, ...]``.  |x| is written as the
        branch x < 0 ? -x : x, so its derivative at x = 0 is +1 (reading)."""
        rho, vel, pres = self.primitives(q)
        c = torch.sqrt(self.gamma * pres / rho)
        un = (vel * n).sum(1)
        return torch.where(un < 0, -un, un) + c

    def rusanov(self, qL, qR, n):
        """Rusanov (local Lax-Friedrichs) normal flux: average of the two normal
        fluxes minus half the largest |u.n|+c times the jump qR - qL.  The
        maximum is the branch lamR > lamL ? lamR : lamL, so at a tie the
        derivative follows the "-" side (reading)."""
        fL = (self.flux(qL) * n[:, :, None]).sum(1)
        fR = (self.flux(qR) * n[:, :, None]).sum(1)
        lamL, lamR = self.wave_speed(qL, n), self.wave_speed(qR, n)
        lam = torch.where(lamR > lamL, lamR, lamL)
        return 0.5 * (fL + fR) - 0.5 * lam[:, None] * (qR - qL)

    # -- viscous --------------------------------------------------------------
    def viscous_flux(self, q, G):
        """Viscous flux from the state and its physical gradient G [N, nd(j), nv, ...]."""
        nd, g, mu = self.nd, self.gamma, self.mu
        kappa = mu * g / ((g - 1.0) * self.Pr)
        rho = q[:, 0]
        vel = [q[:, 1 + i] / rho for i in range(nd)]
        Es = q[:, nd + 1] / rho
        du = [[(G[:, j, 1 + i] - vel[i] * G[:, j, 0]) / rho for j in range(nd)] for i in range(nd)]
        dT = []
        for j in range(nd):
            dE = (G[:, j, nd + 1] - Es * G[:, j, 0]) / rho
            dT.append((g - 1.0) * (dE - sum(vel[k] * du[k][j] for k in range(nd))))
        div = sum(du[k][k] for k in range(nd))
        tau = [[mu * (du[i][j] + du[j][i]) - (2.0 / 3.0 * mu * div if i == j else 0.0)
                for j in range(nd)] for i in range(nd)]
        rows = []
        for j in range(nd):
            comps = [torch.zeros_like(rho)]
            comps += [tau[i][j] for i in range(nd)]
            comps.append(sum(vel[i] * tau[i][j] for i in range(nd)) + kappa * dT[j])
            rows.append(torch.stack(comps, dim=1))
        return torch.stack(rows, dim=1)

    # -- boundary ghost states ------------------------------------------------
    def ghost(self, q, kind):
        """Ghost state: wall (-1) keeps rho, rho E and reverses momentum; far
        field (-2) is the free stream."""
        nd = self.nd
        if kind == -1:
            return torch.cat([q[:, :1], -q[:, 1:1 + nd], q[:, nd + 1:]], dim=1)
        if kind == -2:
            shape = (q.shape[0], self.nv) + (1,) * (q.dim() - 2)
            return self.q_inf.reshape((1, self.nv) + (1,) * (q.dim() - 2)).expand(shape) + 0.0 * q
        raise ValueError(kind)


class Advection:
    """Scalar linear advection f_j = a_j q; Rusanov with |a.n| is the upwind flux."""

    def __init__(self, nd, a):
        self.nd, self.nv = nd, 1
        self.a = torch.as_tensor(a, dtype=torch.float64)
        self.viscous = False

    def flux(self, q):
        shape = (1, self.nd, 1) + (1,) * (q.dim() - 2)
        return self.a.reshape(shape) * q[:, None]

    def rusanov(self, qL, qR, n):
        an = (self.a.reshape((1, self.nd) + (1,) * (n.dim() - 2)) * n).sum(1)
        return 0.5 * an[:, None] * (qL + qR) - 0.5 * torch.abs(an)[:, None] * (qR - qL)
