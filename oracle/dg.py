"""Direct nodal DG discretisations in 2D, FP64, test infrastructure only.

Used only to check that FR with the DG (Radau) correction functions and Gauss
solution points reproduces DG (Huynh 2007), for the two parts of the FR
residual that such a check can fix:

* ``dg_advection_residual``: scalar linear advection with the upwind flux
  (the divergence, the correction and the common inviscid flux);
* ``dg_br2_diffusion_residual``: scalar diffusion with the BR2 common gradient
  of Bassi and Rebay (the corrected gradient and the face-local lifting of the
  paper's common gradient, Sec. 2.2, Eq. com_grad_q).

The advection routine is a weak form, written independently of ``fr``:

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


def _lagrange_1d(nodes, x):
    """L[a, k] = l_k(x_a) and dL[a, k] = l_k'(x_a) of the Lagrange basis through
    ``nodes``, by the product formula and its product rule."""
    n, m = len(nodes), len(x)
    L = np.ones((m, n))
    dL = np.zeros((m, n))
    for k in range(n):
        for j in range(n):
            if j != k:
                L[:, k] *= (x - nodes[j]) / (nodes[k] - nodes[j])
        for j in range(n):
            if j == k:
                continue
            t = np.full(m, 1.0 / (nodes[k] - nodes[j]))
            for i in range(n):
                if i != k and i != j:
                    t *= (x - nodes[i]) / (nodes[k] - nodes[i])
            dL[:, k] += t
    return L, dL


def dg_br2_diffusion_residual(mesh, q, mu):
    """DG for dq/dt = mu Lap q on parallelograms with the BR2 common gradient.

    Written as the weak form of Bassi and Rebay's second scheme, independently
    of ``fr`` and of its basis module: nodal basis phi_k = l_i(xi) l_j(eta) at
    the Gauss points (k = i + P j), every integral by a Gauss rule with P + 2
    points per direction (numpy's ``leggauss``), dense mass matrices.

    * common value on a face: q^ = (q- + q+)/2;
    * face-local lifting of side K on face f: r_f in [Q_p]^2 with
      int_K r_f . tau = int_f (q^ - q_K) tau . n_K  for every tau in [Q_p]^2;
    * element gradient: sigma_K = grad q_K + sum_f r_f (the global lifting);
    * face gradient: sigma^_f = {grad q + r_f}, the mean of both sides;
    * weak form: int_K phi R = -int_K mu sigma_K . grad phi + sum_f int_f phi mu sigma^_f . n_K.

    With the penalty factor 1, this is the reading of the paper's common
    gradient (Eq. com_grad_q) that the FR oracle implements.  Returns R in the
    canonical layout."""
    assert mesh.nd == 2 and mesh.geom_order == 1
    E = mesh.n_elem
    p = int(mesh.p[0])
    assert np.all(mesh.p == p)
    P = p + 1
    xs, _ = np.polynomial.legendre.leggauss(P)                       # solution points
    xq, wq = np.polynomial.legendre.leggauss(P + 2)                  # integration rule
    Lq, dLq = _lagrange_1d(xs, xq)                                   # [Q, P]
    Le, dLe = _lagrange_1d(xs, np.array([-1.0, 1.0]))                # [2, P]
    nq = len(xq)
    # volume: phi and its reference gradient at the tensor rule, point (a, b) -> a + Q b
    Phi = np.einsum("ai,bj->abji", Lq, Lq).reshape(nq * nq, P * P)
    Dxi = np.einsum("ai,bj->abji", dLq, Lq).reshape(nq * nq, P * P)
    Deta = np.einsum("ai,bj->abji", Lq, dLq).reshape(nq * nq, P * P)
    Wv = np.einsum("a,b->ab", wq, wq).reshape(-1)

    def face_ops(f):
        """phi, d/dxi phi, d/deta phi at the Q points of face f (f = 2d + s)."""
        d, s = f // 2, f % 2
        if d == 0:      # xi = -1 / +1, tangential parameter eta
            ph = np.einsum("i,cj->cji", Le[s], Lq)
            dx = np.einsum("i,cj->cji", dLe[s], Lq)
            de = np.einsum("i,cj->cji", Le[s], dLq)
        else:           # eta = -1 / +1, tangential parameter xi
            ph = np.einsum("ci,j->cji", Lq, Le[s])
            dx = np.einsum("ci,j->cji", dLq, Le[s])
            de = np.einsum("ci,j->cji", Lq, dLe[s])
        return ph.reshape(nq, P * P), dx.reshape(nq, P * P), de.reshape(nq, P * P)

    F = [face_ops(f) for f in range(4)]
    X = mesh.nodes
    e1 = 0.5 * (X[:, 1] - X[:, 0])
    e2 = 0.5 * (X[:, 2] - X[:, 0])
    Jm = np.stack([e1, e2], axis=-1)                                 # [E, comp, ref]
    detJ = np.linalg.det(Jm)
    Jinv = np.linalg.inv(Jm)                                         # row d = grad(xi_d)
    q = np.asarray(q, dtype=np.float64).reshape(E, P * P)

    def grad(e, Dx, De):
        """Physical gradient operators [.., 2(j), P^2] from the reference ones."""
        return np.stack([Jinv[e, 0, j] * Dx + Jinv[e, 1, j] * De for j in range(2)], axis=-2)

    M = [Phi.T @ (Wv[:, None] * detJ[e] * Phi) for e in range(E)]
    # face data of every side: normal, area weights, trace and gradient trace
    nrm, wS, u, gu = {}, {}, {}, {}
    for e in range(E):
        for f in range(4):
            d, s = f // 2, f % 2
            tang = e2[e] if d == 0 else e1[e]
            wS[e, f] = wq * np.linalg.norm(tang)
            nv = Jinv[e, d] * (1.0 if s == 1 else -1.0)
            nrm[e, f] = nv / np.linalg.norm(nv)
            ph, dx, de = F[f]
            u[e, f] = ph @ q[e]
            gu[e, f] = grad(e, dx, de) @ q[e]                          # [Q, 2]

    def other(e, f):
        nb, g = int(mesh.nbr[e, f]), int(mesh.nbr_face[e, f])
        rev = bool(mesh.orient[e, f] & 2)
        return nb, g, (slice(None, None, -1) if rev else slice(None))

    # face-local liftings r[e, f] as coefficient vectors [2, P^2]
    r = {}
    for e in range(E):
        for f in range(4):
            nb, g, sl = other(e, f)
            qhat = 0.5 * (u[e, f] + u[nb, g][sl])
            ph = F[f][0]
            rhs = np.stack([ph.T @ (wS[e, f] * (qhat - u[e, f]) * nrm[e, f][j]) for j in range(2)])
            r[e, f] = np.linalg.solve(M[e], rhs.T).T
    R = np.zeros((E, P * P))
    for e in range(E):
        G = grad(e, Dxi, Deta)                                         # [Q^2, 2, P^2]
        sigma = G @ q[e] + sum(Phi @ r[e, f].T for f in range(4))      # [Q^2, 2]
        rhs = -np.einsum("a,aj,ajk->k", Wv * detJ[e] * mu, sigma, G)
        for f in range(4):
            nb, g, sl = other(e, f)
            ph = F[f][0]
            mine = gu[e, f] + ph @ r[e, f].T
            theirs = (gu[nb, g] + F[g][0] @ r[nb, g].T)[sl]
            shat = 0.5 * (mine + theirs)
            rhs += ph.T @ (wS[e, f] * mu * (shat @ nrm[e, f]))
        R[e] = np.linalg.solve(M[e], rhs)
    return R.reshape(-1)
