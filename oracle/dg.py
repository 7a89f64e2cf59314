"""Direct nodal DG for 2D scalar linear advection, FP64, test infrastructure only.

Used only to check that FR with the DG (Radau) correction functions and Gauss
solution points reproduces nodal DG with Gauss quadrature (Huynh 2007).  This
routine is a weak form, written independently of ``fr``:

  w_i |J| dq_i/dt = sum_k w_k |J| f(q_k) . grad(phi_i)(x_k)
                    - sum_faces sum_fp w_fp |dx/ds| phi_i(x_fp) f^com(x_fp) . n_out

on parallelogram elements (constant Jacobian) with the upwind flux.  Returns
R = dq/dt in the canonical layout.
"""
import numpy as np

from .basis import basis


def dg_advection_residual(mesh, q, a):
    assert mesh.nd == 2 and mesh.geom_order == 1
    a = np.asarray(a, dtype=np.float64)
    E = mesh.n_elem
    p = int(mesh.p[0])
    assert np.all(mesh.p == p)
    b = basis(p)
    P = p + 1
    x = b.x.numpy()
    w = b.w.numpy()
    L = np.eye(P)                                                    # l_k(x_i) at the Gauss points
    D = b.D.numpy()                                                  # D[i, k] = l_k'(x_i)
    ends = b.ext.numpy()                                             # [2, P]
    q = np.asarray(q, dtype=np.float64).reshape(E, P, P)            # [e, j(eta), i(xi)]
    R = np.zeros_like(q)
    # element Jacobian from the vertices (nodes 0: (-1,-1), 1: (1,-1), 2: (-1,1))
    X = mesh.nodes
    e1 = 0.5 * (X[:, 1] - X[:, 0])
    e2 = 0.5 * (X[:, 2] - X[:, 0])
    Jm = np.stack([e1, e2], axis=-1)                                 # [E, comp, ref]
    detJ = np.linalg.det(Jm)
    Jinv = np.linalg.inv(Jm)                                         # [E, ref, comp]

    def trace(e, f):
        d, s = f // 2, f % 2
        if d == 0:
            return q[e] @ ends[s]                                    # along xi: [eta]
        return ends[s] @ q[e]                                        # along eta: [xi]

    for e in range(E):
        # volume term: sum_k w_k |J| f(q_k) . grad phi_i(x_k)
        for jj in range(P):
            for ii in range(P):
                acc = 0.0
                for kj in range(P):
                    for ki in range(P):
                        # grad_xi phi_(ii,jj) at (ki, kj)
                        gx = D[ki, ii] * L[kj, jj]
                        gy = L[ki, ii] * D[kj, jj]
                        grad = Jinv[e].T @ np.array([gx, gy])
                        acc += w[ki] * w[kj] * detJ[e] * q[e, kj, ki] * (a @ grad)
                R[e, jj, ii] += acc
        # surface term
        for f in range(4):
            d, s = f // 2, f % 2
            nb, g = int(mesh.nbr[e, f]), int(mesh.nbr_face[e, f])
            tang = e2 if d == 0 else e1                               # dx/ds along the face
            ds = np.linalg.norm(tang[e])
            nvec = Jinv[e][d] * (1.0 if s == 1 else -1.0)
            nvec = nvec / np.linalg.norm(nvec)
            an = float(a @ nvec)
            qin = trace(e, f)
            qout = trace(nb, g)
            if mesh.orient[e, f] & 2:
                qout = qout[::-1]
            fcom = an * (qin if an >= 0 else qout)
            # phi_(i,j) at face point t is ends[s, i] delta_(j,t) on xi-faces and
            # ends[s, j] delta_(i,t) on eta-faces
            if d == 0:
                for t in range(P):
                    R[e, t, :] -= w[t] * ds * ends[s, :] * fcom[t]
            else:
                for t in range(P):
                    R[e, :, t] -= w[t] * ds * ends[s, :] * fcom[t]
        for jj in range(P):
            for ii in range(P):
                R[e, jj, ii] /= w[ii] * w[jj] * detJ[e]
    return R.reshape(-1)
