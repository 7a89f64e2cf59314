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

    def __init__(self, nd, gamma=1.4, mu=0.0, Pr=0.72, q_inf=None, flux="rusanov"):
        self.nd, self.nv = nd, nd + 2
        self.gamma, self.mu, self.Pr = float(gamma), float(mu), float(Pr)
        self.viscous = self.mu > 0.0
        self.q_inf = None if q_inf is None else torch.as_tensor(q_inf, dtype=torch.float64)
        if flux not in ("rusanov", "roe"):
            raise ValueError(flux)
        self.flux_kind = flux

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

    def common_flux(self, qL, qR, n):
        """The common inviscid normal flux of the face: Rusanov or Roe."""
        return self.roe(qL, qR, n) if self.flux_kind == "roe" else self.rusanov(qL, qR, n)

    def roe_average(self, qL, qR):
        """Roe's averages (Roe 1981): sqrt(rho)-weighted velocity and total
        enthalpy H = (rho E + p) / rho, and the sound speed from them."""
        g = self.gamma
        rL, vL, pL = self.primitives(qL)
        rR, vR, pR = self.primitives(qR)
        sL, sR = torch.sqrt(rL), torch.sqrt(rR)
        HL = (qL[:, self.nd + 1] + pL) / rL
        HR = (qR[:, self.nd + 1] + pR) / rR
        w = sL + sR
        u = (sL[:, None] * vL + sR[:, None] * vR) / w[:, None]
        H = (sL * HL + sR * HR) / w
        c = torch.sqrt((g - 1.0) * (H - 0.5 * (u * u).sum(1)))
        return u, H, c

    def roe_eigensystem(self, u, H, c, n):
        """Eigenvalues and right eigenvectors of the normal flux Jacobian
        d(f.n)/dq at the averaged state (velocity u, enthalpy H, sound speed c):
        u.n - c, u.n (entropy and nd - 1 shear waves along tangents of n),
        u.n + c.  Points are moved to the leading axes: lam [..., nv],
        R [..., nv, nv] with the eigenvectors as columns."""
        nd, nv = self.nd, self.nv
        # points first: [N, nd, *pts] -> [N, *pts, nd]
        perm = (0,) + tuple(range(2, u.dim())) + (1,)
        u, n = u.permute(perm), n.permute(perm)
        H, c = H, c
        un = (u * n).sum(-1)
        # tangents: e_i minus its normal part for the axis least aligned with n,
        # then (3D) the cross product completes the frame
        ai = torch.argmin(torch.abs(n), dim=-1)
        e = torch.nn.functional.one_hot(ai, nd).to(n.dtype)
        t1 = e - (e * n).sum(-1, keepdim=True) * n
        t1 = t1 / torch.sqrt((t1 * t1).sum(-1, keepdim=True))
        tans = [t1]
        if nd == 3:
            tans.append(torch.linalg.cross(n, t1, dim=-1))
        one = torch.ones_like(un)
        zero = torch.zeros_like(un)
        cols = [torch.cat([one[..., None], u - c[..., None] * n, (H - c * un)[..., None]], -1),
                torch.cat([one[..., None], u, (0.5 * (u * u).sum(-1))[..., None]], -1)]
        for t in tans:
            cols.append(torch.cat([zero[..., None], t, (u * t).sum(-1)[..., None]], -1))
        cols.append(torch.cat([one[..., None], u + c[..., None] * n, (H + c * un)[..., None]], -1))
        R = torch.stack(cols, dim=-1)
        lam = torch.stack([un - c] + [un] * nd + [un + c], dim=-1)
        return lam, R

    def roe(self, qL, qR, n):
        """Roe's common normal flux (the paper's Sec. 2.2 formula): average of
        the two normal fluxes minus half of R |Lambda| R^-1 (qR - qL), the
        eigensystem of the normal flux Jacobian at Roe's averaged state.  No
        entropy fix (the paper names none); |x| is the branch x < 0 ? -x : x
        (derivative +1 at 0, as in the wave speed)."""
        fL = (self.flux(qL) * n[:, :, None]).sum(1)
        fR = (self.flux(qR) * n[:, :, None]).sum(1)
        u, H, c = self.roe_average(qL, qR)
        lam, R = self.roe_eigensystem(u, H, c, n)
        perm = (0,) + tuple(range(2, qL.dim())) + (1,)
        dq = (qR - qL).permute(perm)
        alpha = torch.linalg.solve(R, dq[..., None])[..., 0]        # wave strengths R^-1 dq
        diss = (R @ (torch.where(lam < 0, -lam, lam) * alpha)[..., None])[..., 0]
        inv = [0, qL.dim() - 1] + list(range(1, qL.dim() - 1))
        return 0.5 * (fL + fR) - 0.5 * diss.permute(inv)

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

    def common_flux(self, qL, qR, n):
        """The upwind flux (for a scalar the Roe and Rusanov fluxes coincide)."""
        return self.rusanov(qL, qR, n)


class Diffusion:
    """Scalar diffusion dq/dt = mu Lap q (no inviscid flux; viscous flux mu grad q),
    used only to check the BR2 common gradient against a direct DG-BR2 weak form."""

    def __init__(self, nd, mu):
        self.nd, self.nv = nd, 1
        self.mu = float(mu)
        self.viscous = True

    def flux(self, q):
        return torch.zeros((q.shape[0], self.nd) + tuple(q.shape[1:]), dtype=q.dtype)

    def common_flux(self, qL, qR, n):
        return torch.zeros_like(qL)

    def viscous_flux(self, q, G):
        return self.mu * G
