"""FR residual R(q) = -div f on hexahedra / quadrilaterals of mixed degree p.

FP64, test infrastructure only.  Follows Sec. 2.2 of the paper:

* differential FR form dq/dt + P(div f) + delta = 0 (Eq. FR_diff), with the
  flux interpolated at the solution points ("P") and the correction field
  delta built dimension by dimension from the 1D DG correction functions;
  in reference space, per direction d and face side s,
      dF_d/dxi_d  ->  D F_d + g_s'(xi_d) (F^com_(d,s) - F_d(xi_d = +-1)),
  R = -(1/|J|) sum_d [...]  (R = -div f, Eq. ESDIRK_ns);
* the common inviscid normal flux is Rusanov (the paper uses Roe, Eq.
  invis_com; the hot path is specified with Rusanov);
* common solution q^com = (q- + q+)/2 (Eq. com_q) and common gradient
  grad q^com = (grad q- + r- + grad q+ + r+)/2 (Eq. com_grad_q) with the
  BR2-type lifting r = g_s'(face) (S_d/|J|) (q^com - q) of the face jump
  (reading: the paper gives no BR2 details);
* the viscous flux inside an element uses the corrected gradient
  d_xi_d q^C = D_d q + sum_s g_s'(xi_d) (q^com - q)_(d,s);
* between elements of different degree the face is a mortar with the Gauss
  points of the higher degree ("master" side); the lower-degree side
  interpolates its traces up and receives the L2 projection of the common
  flux (reading: the paper only limits the jump to one degree, Sec. 3.1);
* walls: ghost state with reversed momentum, zero energy viscous flux
  (adiabatic); far field: free-stream ghost state (readings).
"""
import numpy as np
import torch

from .basis import basis, mortar_ops
from .geometry import ElementGeometry, apply1d, face_trace

WALL, FARFIELD = -1, -2


def face_apply(M: torch.Tensor, t: torch.Tensor, nd: int) -> torch.Tensor:
    """Apply the 1D operator M along every face-local axis of ``t [..., nfp]``."""
    if nd == 2:
        return t @ M.T
    Pin = M.shape[1]
    t = t.reshape(t.shape[:-1] + (Pin, Pin))
    t = t @ M.T
    t = (t.transpose(-1, -2) @ M.T).transpose(-1, -2)
    return t.reshape(t.shape[:-2] + (-1,))


def orientation_map(code: int, P: int, nd: int) -> np.ndarray:
    """Face-local index of the neighbour for each face-local index of this side.

    Bit 0 swaps the two axes, bit 1 flips the first, bit 2 the second."""
    n = P ** (nd - 1)
    out = np.empty(n, dtype=np.int64)
    for t in range(n):
        if nd == 2:
            u, v = t, 0
        else:
            ia, ib = t % P, t // P
            u, v = (ib, ia) if code & 1 else (ia, ib)
        if code & 2:
            u = P - 1 - u
        if code & 4 and nd == 3:
            v = P - 1 - v
        out[t] = u + P * v
    return out


def lift(vec: torch.Tensor, face_vals: torch.Tensor, d: int, nd: int, P: int) -> torch.Tensor:
    """vec(xi_d) times the face values, spread along the lines of direction d."""
    lead = face_vals.shape[:-1]
    J = face_vals.reshape(lead + (P,) * (nd - 1))
    ax = len(lead) + (nd - 1 - d)
    J = J.unsqueeze(ax)
    shape = [1] * J.dim()
    shape[ax] = P
    return J * vec.reshape(shape)


def _sign(s):
    return 2.0 * s - 1.0


class FR:
    """Discretisation of one mesh with fixed per-element degrees."""

    def __init__(self, mesh, physics):
        self.mesh, self.phys = mesh, physics
        nd = self.nd = mesh.nd
        self.nv = physics.nv
        self.nf = 2 * nd
        E = mesh.n_elem
        p = mesh.p.astype(np.int64)
        self.n_dof = int(((p + 1) ** nd).sum()) * self.nv
        off = np.zeros(E + 1, dtype=np.int64)
        np.cumsum((p + 1) ** nd * self.nv, out=off[1:])
        self.offsets = off
        self.pos = np.zeros(E, dtype=np.int64)
        self.groups = {}
        nodes = torch.from_numpy(np.ascontiguousarray(mesh.nodes))
        for pg in sorted(set(p.tolist())):
            elems = np.nonzero(p == pg)[0]
            self.pos[elems] = np.arange(len(elems))
            P = pg + 1
            nsp = P ** nd
            idx = torch.from_numpy(off[elems][:, None] + np.arange(nsp * self.nv)[None, :])
            geom = ElementGeometry(nodes[elems], mesh.geom_order, pg, nd)
            self.groups[pg] = dict(elems=elems, idx=idx, geom=geom, P=P, nsp=nsp,
                                   nfp=P ** (nd - 1))
        self._build_faces()

    # ------------------------------------------------------------------ faces
    def _build_faces(self):
        m, nd = self.mesh, self.nd
        p = m.p.astype(np.int64)
        inter, bnd = {}, {}
        for e in range(m.n_elem):
            for f in range(self.nf):
                n = int(m.nbr[e, f])
                if n < 0:
                    bnd.setdefault((int(p[e]), n), []).append((self.pos[e], f))
                    continue
                g = int(m.nbr_face[e, f])
                master = (p[e] > p[n]) or (p[e] == p[n] and (e < n or (e == n and f < g)))
                if master:
                    inter.setdefault((int(p[e]), int(p[n])), []).append(
                        (self.pos[e], f, self.pos[n], g, int(m.orient[e, f])))
        self.inter = {}
        for (pm, ps), lst in inter.items():
            a = np.array(lst, dtype=np.int64)
            Pm = pm + 1
            perm = np.stack([orientation_map(int(c), Pm, nd) for c in a[:, 4]])
            inv = np.argsort(perm, axis=1)
            self.inter[(pm, ps)] = dict(mE=torch.from_numpy(a[:, 0]), mF=torch.from_numpy(a[:, 1]),
                                        sE=torch.from_numpy(a[:, 2]), sF=torch.from_numpy(a[:, 3]),
                                        perm=torch.from_numpy(perm), inv=torch.from_numpy(inv))
        self.bnd = {}
        for (pg, kind), lst in bnd.items():
            a = np.array(lst, dtype=np.int64)
            self.bnd[(pg, kind)] = dict(E=torch.from_numpy(a[:, 0]), F=torch.from_numpy(a[:, 1]))

    # ----------------------------------------------------------- layout helpers
    def to_groups(self, q: torch.Tensor) -> dict:
        """Canonical vector -> {p: [E_p, nv, (P,)*nd]}."""
        out = {}
        for pg, G in self.groups.items():
            P, nd = G["P"], self.nd
            t = q[G["idx"]].reshape((-1,) + (P,) * nd + (self.nv,))
            out[pg] = torch.movedim(t, -1, 1)
        return out

    def from_groups(self, parts: dict) -> torch.Tensor:
        """{p: [E_p, nv, (P,)*nd]} -> canonical vector."""
        idx, vals = [], []
        for pg, G in self.groups.items():
            t = torch.movedim(parts[pg], 1, -1).reshape(len(G["elems"]), -1)
            idx.append(G["idx"].reshape(-1))
            vals.append(t.reshape(-1))
        idx = torch.cat(idx)
        vals = torch.cat(vals)
        ref = vals if vals.numel() else torch.zeros(0)
        return torch.zeros(self.n_dof, dtype=ref.dtype).index_put((idx,), vals)

    # --------------------------------------------------------------- residual
    def residual(self, q: torch.Tensor) -> torch.Tensor:
        nd, nv, nf, ph = self.nd, self.nv, self.nf, self.phys
        visc = getattr(ph, "viscous", False)
        Q = self.to_groups(q)
        qf, gf, dq = {}, {}, {}
        for pg, G in self.groups.items():
            b = basis(pg)
            qf[pg] = torch.stack([face_trace(Q[pg], b, d, s, nd) for d in range(nd) for s in (0, 1)], dim=1)
            if visc:
                geom = G["geom"]
                dq[pg] = torch.stack([apply1d(b.D, Q[pg], d) for d in range(nd)], dim=1)
                faces = []
                for d in range(nd):
                    for s in (0, 1):
                        f = 2 * d + s
                        dqf = face_trace(dq[pg], b, d, s, nd)              # [E, d', nv, nfp]
                        Gp = torch.einsum("edjn,edvn->ejvn", geom.Sf[:, f], dqf)
                        faces.append(Gp / geom.Jf[:, f][:, None, None])
                gf[pg] = torch.stack(faces, dim=1)                          # [E, nf, j, nv, nfp]

        slots = {pg: ([], [], []) for pg in self.groups}   # linear slot, Fcom, dq

        def put(pg, E_idx, F_idx, Fv, Dv):
            slots[pg][0].append(E_idx * nf + F_idx)
            slots[pg][1].append(Fv)
            slots[pg][2].append(Dv)

        # interior faces (mortars when the degrees differ)
        for (pm, ps), fg in self.inter.items():
            GM, GS = self.groups[pm], self.groups[ps]
            bM, bS = basis(pm), basis(ps)
            I, Pi = mortar_ops(ps, pm)
            mE, mF, sE, sF = fg["mE"], fg["mF"], fg["sE"], fg["sF"]
            perm, inv = fg["perm"], fg["inv"]

            def to_master(t):
                t = face_apply(I, t, nd)
                return torch.gather(t, -1, perm.reshape(perm.shape[:1] + (1,) * (t.dim() - 2) + perm.shape[1:]).expand(t.shape))

            def to_slave(t):
                t = torch.gather(t, -1, inv.reshape(inv.shape[:1] + (1,) * (t.dim() - 2) + inv.shape[1:]).expand(t.shape))
                return face_apply(Pi, t, nd)

            dm, sm = mF // 2, mF % 2
            ds, ss = sF // 2, sF % 2
            qM = qf[pm][mE, mF]
            qS_own = qf[ps][sE, sF]
            qS = to_master(qS_own)
            A = _sign(sm)[:, None, None] * GM["geom"].Sf[mE, mF, dm]        # [F, j, nfp]
            absA = torch.sqrt((A * A).sum(1))
            n = A / absA[:, None]
            Fn = ph.common_flux(qM, qS, n) * absA[:, None]
            qc = None
            if visc:
                qc = 0.5 * (qM + qS)
                cM = bM.dg_face[sm][:, None, None] * GM["geom"].Sf[mE, mF, dm] / GM["geom"].Jf[mE, mF][:, None]
                cS_own = bS.dg_face[ss][:, None, None] * GS["geom"].Sf[sE, sF, ds] / GS["geom"].Jf[sE, sF][:, None]
                cS = to_master(cS_own)
                GMf = gf[pm][mE, mF]
                GSf = to_master(gf[ps][sE, sF])
                Gc = 0.5 * (GMf + cM[:, :, None] * (qc - qM)[:, None]
                            + GSf + cS[:, :, None] * (qc - qS)[:, None])
                Fv = (ph.viscous_flux(qc, Gc) * A[:, :, None]).sum(1)
                Fn = Fn - Fv
            put(pm, mE, mF, _sign(sm)[:, None, None] * Fn, (qc - qM) if visc else None)
            FS = _sign(ss)[:, None, None] * to_slave(-Fn)
            put(ps, sE, sF, FS, (to_slave(qc) - qS_own) if visc else None)

        # boundary faces
        for (pg, kind), bg in self.bnd.items():
            Gg = self.groups[pg]
            b = basis(pg)
            Ei, Fi = bg["E"], bg["F"]
            d, s = Fi // 2, Fi % 2
            qM = qf[pg][Ei, Fi]
            qG = ph.ghost(qM, kind)
            A = _sign(s)[:, None, None] * Gg["geom"].Sf[Ei, Fi, d]
            absA = torch.sqrt((A * A).sum(1))
            n = A / absA[:, None]
            Fn = ph.common_flux(qM, qG, n) * absA[:, None]
            qc = None
            if visc:
                qc = 0.5 * (qM + qG)
                cM = b.dg_face[s][:, None, None] * Gg["geom"].Sf[Ei, Fi, d] / Gg["geom"].Jf[Ei, Fi][:, None]
                Gc = gf[pg][Ei, Fi] + cM[:, :, None] * (qc - qM)[:, None]
                Fv = (ph.viscous_flux(qc, Gc) * A[:, :, None]).sum(1)
                if kind == WALL:   # adiabatic wall: no energy flux through the wall
                    Fv = torch.cat([Fv[:, :nv - 1], torch.zeros_like(Fv[:, nv - 1:])], dim=1)
                Fn = Fn - Fv
            put(pg, Ei, Fi, _sign(s)[:, None, None] * Fn, (qc - qM) if visc else None)

        # volume: corrected gradient, flux, divergence and correction
        R = {}
        for pg, G in self.groups.items():
            b, P, geom = basis(pg), G["P"], G["geom"]
            Eg, nfp = len(G["elems"]), G["nfp"]
            lin = torch.cat(slots[pg][0])
            FC = torch.zeros(Eg * nf, nv, nfp).index_put((lin,), torch.cat(slots[pg][1])).reshape(Eg, nf, nv, nfp)
            q = Q[pg]
            f = ph.flux(q)                                                   # [E, j, nv, sp]
            if visc:
                DQ = torch.zeros(Eg * nf, nv, nfp).index_put((lin,), torch.cat(slots[pg][2])).reshape(Eg, nf, nv, nfp)
                dqc = []
                for d in range(nd):
                    t = dq[pg][:, d]
                    for s in (0, 1):
                        t = t + lift(b.dg[s], DQ[:, 2 * d + s], d, nd, P)
                    dqc.append(t)
                dqc = torch.stack(dqc, dim=1)                                 # [E, d, nv, sp]
                Gp = torch.einsum("edjx,edvx->ejvx", geom.S.flatten(3), dqc.flatten(3))
                Gp = Gp.reshape(dqc.shape) / geom.J[:, None, None]
                f = f - ph.viscous_flux(q, Gp)
            Ft = torch.einsum("edjx,ejvx->edvx", geom.S.flatten(3), f.flatten(3)).reshape(f.shape)
            div = 0.0
            for d in range(nd):
                div = div + apply1d(b.D, Ft[:, d], d)
                for s in (0, 1):
                    jump = FC[:, 2 * d + s] - face_trace(Ft[:, d], b, d, s, nd)
                    div = div + lift(b.dg[s], jump, d, nd, P)
            R[pg] = -div / geom.J[:, None]
        return self.from_groups(R)

    # ----------------------------------------------------------- diagnostics
    def quadrature_weights(self) -> torch.Tensor:
        """w_xi w_eta (w_zeta) |J| at every DOF (canonical layout)."""
        parts = {}
        for pg, G in self.groups.items():
            w = basis(pg).w
            if self.nd == 2:
                W = w[:, None] * w[None, :]
            else:
                W = w[:, None, None] * w[None, :, None] * w[None, None, :]
            wj = G["geom"].J * W
            parts[pg] = wj[:, None].expand((-1, self.nv) + wj.shape[1:])
        return self.from_groups(parts)

    def sp_coordinates(self) -> dict:
        return {pg: G["geom"].X for pg, G in self.groups.items()}
