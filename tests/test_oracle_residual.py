"""Pins of the oracle FR residual: invariants, closed forms, an independent DG
discretisation, and the convergence order on the isentropic vortex."""
import math

import numpy as np
import pytest
import torch

import cases
from oracle.dg import dg_advection_residual
from oracle.fr import FR
from oracle.physics import Advection, Euler


def _euler(m, mu=0.0, Pr=0.72, q_inf=None):
    return FR(m, Euler(m.nd, 1.4, mu, Pr, q_inf))


def _qinf(nd, vel=(0.3, 0.2, 0.1)):
    return cases.free_stream_q(nd, vel=vel, mach=0.3)


def _free_stream_residual(m, mu):
    fr = _euler(m, mu, 0.7, _qinf(m.nd))
    q = torch.from_numpy(cases.freestream_state(m, vel=(0.3, 0.2, 0.1), mach=0.3))
    return float(fr.residual(q).abs().max())


def _no_walls(m):
    m.nbr = m.nbr.copy()
    m.nbr[m.nbr == cases.WALL] = cases.FARFIELD
    return m


@pytest.mark.parametrize("name,builder", [
    ("jittered quads p2", lambda: cases.workload_vortex2d(6, 2)[0]),
    ("jittered quads mixed p", lambda: cases.workload_vortex2d(6, 2)[0].with_p(
        (cases.uniform(5, 36) * 4 + 1).astype(np.int8))),
    ("box p3", lambda: cases.periodic_box(3, 3, 0.0, 2 * math.pi, 3)),
    ("box mixed p", lambda: cases.periodic_box(3, 3, 0.0, 1.0, 1).with_p(
        (cases.uniform(6, 27) * 3 + 1).astype(np.int8))),
    ("cylinder quadratic p2", lambda: _no_walls(cases.cylinder_ogrid(3, 8, 2, g=2, p=2))),
    ("cylinder quadratic p2/p3", lambda: _no_walls(cases.cylinder_ogrid(3, 8, 2, g=2, p=2)).with_p(
        (cases.uniform(7, 48) * 2 + 2).astype(np.int8))),
    ("naca mixed p, wake cut", lambda: _no_walls(cases.naca_cgrid(24, 4, 2, n_wake=6)).with_p(
        (cases.uniform(8, 192) * 3 + 1).astype(np.int8))),
])
@pytest.mark.parametrize("mu", [0.0, 1e-2])
def test_free_stream_preservation(name, builder, mu):
    m = builder()
    flux_scale = (1.0 / (1.4 * 0.09)) / 0.005   # pressure over the smallest element size
    assert _free_stream_residual(m, mu) <= 1e-12 * flux_scale, name


def test_free_stream_not_preserved_when_geometry_underresolved():
    """p = 1 cannot represent the quadratic cylinder map: the check above is not vacuous."""
    m = _no_walls(cases.cylinder_ogrid(3, 8, 2, g=2, p=1))
    assert _free_stream_residual(m, 0.0) > 1e-3


@pytest.mark.parametrize("mesh_p", ["uniform", "mixed"])
@pytest.mark.parametrize("mu", [0.0, 0.05])
@pytest.mark.parametrize("nd", [2, 3])
def test_conservation_periodic(mesh_p, mu, nd):
    if nd == 2:
        m = cases.workload_vortex2d(5, 2)[0]
    else:
        m = cases.periodic_box(3, 3, 0.0, 1.0, 2)
        m.nodes = m.nodes + 0.03 * np.sin(7 * m.nodes[..., ::-1])  # non-affine but watertight
    if mesh_p == "mixed":
        m = m.with_p((cases.uniform(11, m.n_elem) * 3 + 1).astype(np.int8))
    fr = _euler(m, mu, 0.71)
    q = torch.from_numpy(cases.random_state(m, 3))
    R = fr.residual(q)
    W = fr.quadrature_weights()
    # per variable: sum over every solution point of w |J| R
    parts = fr.to_groups(W * R)
    tot = sum(t.flatten(2).sum(dim=(0, 2)) for t in parts.values())
    scale = sum(t.abs().flatten(2).sum(dim=(0, 2)) for t in parts.values())
    assert torch.all(tot.abs() <= 1e-13 * scale), (tot, scale)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fr_dg_equals_nodal_dg_linear_advection(p):
    m = cases.periodic_box(2, 4, 0.0, 1.0, p)
    m.nodes = m.nodes.copy()
    m.nodes[..., 0] += 0.3 * m.nodes[..., 1]          # parallelograms
    a = (1.0, 0.7)
    fr = FR(m, Advection(2, a))
    q = torch.from_numpy(cases.uniform(3, int(m.n_sp().sum())) - 0.5)
    R1 = fr.residual(q).numpy()
    R2 = dg_advection_residual(m, q.numpy(), a)
    assert np.abs(R1 - R2).max() <= 1e-13 * np.abs(R1).max()


def _rot2(th):
    c, s = math.cos(th), math.sin(th)
    return np.array([[c, -s], [s, c]])


@pytest.mark.parametrize("nd", [2, 3])
@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_rotation_equivariance(nd, mu):
    """Rotating mesh and velocity rotates the momentum residual and leaves the rest."""
    if nd == 2:
        m = cases.workload_vortex2d(4, 2)[0]
        Rm = _rot2(0.7)
    else:
        m = cases.periodic_box(3, 2, 0.0, 1.0, 2)
        a = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
        K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
        Rm = np.eye(3) + math.sin(0.9) * K + (1 - math.cos(0.9)) * K @ K
    q = cases.random_state(m, 5).reshape(-1, nd + 2)
    R0 = _euler(m, mu, 0.71).residual(torch.from_numpy(q.reshape(-1))).numpy().reshape(-1, nd + 2)
    mr = cases.Mesh(m.nd, m.geom_order, m.nodes @ Rm.T, m.nbr, m.nbr_face, m.orient, m.p)
    qr = q.copy()
    qr[:, 1:1 + nd] = q[:, 1:1 + nd] @ Rm.T
    R1 = _euler(mr, mu, 0.71).residual(torch.from_numpy(qr.reshape(-1))).numpy().reshape(-1, nd + 2)
    Rexp = R0.copy()
    Rexp[:, 1:1 + nd] = R0[:, 1:1 + nd] @ Rm.T
    assert np.abs(R1 - Rexp).max() <= 1e-11 * np.abs(R0).max()


def _tg_mesh(nd, n, p):
    return cases.periodic_box(nd, n, 0.0, 2 * math.pi, p)


@pytest.mark.parametrize("nd", [2, 3])
def test_viscous_operator_taylor_green_closed_form(nd):
    """R(mu) - R(0) = div f_v; for the Taylor-Green velocity field at constant
    density and pressure, div tau = mu Lap u = -nd mu u, and in 2D the energy
    term is 2 mu (cos^2 y cos 2x + cos^2 x cos 2y).  The pointwise error of the
    discrete second-derivative operator must fall with h (order >= 2 at p = 4)."""
    mu, p = 0.01, 4
    errs = []
    for n in (4, 8):
        m = _tg_mesh(nd, n, p)
        qs, exact = [], []
        for x in cases.solution_point_positions(m):
            u = np.sin(x[:, 0]) * np.cos(x[:, 1])
            v = -np.cos(x[:, 0]) * np.sin(x[:, 1])
            if nd == 3:
                u = u * np.cos(x[:, 2])
                v = v * np.cos(x[:, 2])
            vel = np.stack([u, v] + ([np.zeros_like(u)] if nd == 3 else []), -1)
            qs.append(cases.prim_to_cons(np.ones_like(u), vel, np.full_like(u, 10.0)))
            ex = np.zeros((len(x), nd + 2))
            ex[:, 1] = -nd * mu * u
            ex[:, 2] = -nd * mu * v
            if nd == 2:
                cx, cy = np.cos(x[:, 0]), np.cos(x[:, 1])
                ex[:, 3] = 2 * mu * (cy ** 2 * np.cos(2 * x[:, 0]) + cx ** 2 * np.cos(2 * x[:, 1]))
            exact.append(ex)
        q = torch.from_numpy(np.concatenate([a.reshape(-1) for a in qs]))
        Rv = (_euler(m, mu, 0.71).residual(q) - _euler(m, 0.0).residual(q)).numpy().reshape(-1, nd + 2)
        ex = np.concatenate(exact)
        cols = [0, 1, 2, 3]
        errs.append(np.array([np.abs(Rv[:, c] - ex[:, c]).max() / (nd * mu) for c in cols]))
    assert errs[1][0] == 0.0                      # no viscous mass flux
    assert np.all(errs[1][1:] < errs[0][1:] / 4), errs
    assert errs[1][1] < 3e-3 and errs[1][2] < 3e-3, errs


def test_heat_flux_closed_form():
    """Fluid at rest, rho = 1, p/rho = T0 + a sin x: the viscous energy residual is
    kappa d2(p/rho)/dx2 = -kappa a sin x, kappa = mu gamma / ((gamma-1) Pr)."""
    mu, Pr, g, a = 0.02, 0.7, 1.4, 0.3
    kappa = mu * g / ((g - 1) * Pr)
    m = _tg_mesh(2, 8, 4)
    X = cases.solution_point_positions(m)
    qs, ex = [], []
    for x in X:
        T = 5.0 + a * np.sin(x[:, 0])
        qs.append(cases.prim_to_cons(np.ones_like(T), np.zeros((len(T), 2)), T))
        e = np.zeros((len(T), 4))
        e[:, 3] = -kappa * a * np.sin(x[:, 0])
        ex.append(e)
    q = torch.from_numpy(np.concatenate([t.reshape(-1) for t in qs]))
    Rv = (_euler(m, mu, Pr).residual(q) - _euler(m, 0.0).residual(q)).numpy().reshape(-1, 4)
    assert np.abs(Rv - np.concatenate(ex)).max() < 2e-3 * kappa * a


def _vortex_error(n, p, T=0.5):
    m = cases.periodic_box(2, n, -10.0, 10.0, p)
    fr = _euler(m)
    q = torch.from_numpy(cases.vortex_state(m))
    h = 20.0 / n
    nsteps = int(math.ceil(T / (0.3 * h / (4.0 * (2 * p + 1)))))
    dt = T / nsteps
    for _ in range(nsteps):   # classical RK4, a test-only integrator
        k1 = fr.residual(q)
        k2 = fr.residual(q + 0.5 * dt * k1)
        k3 = fr.residual(q + 0.5 * dt * k2)
        k4 = fr.residual(q + dt * k3)
        q = q + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    qe = torch.from_numpy(cases.vortex_exact(m, T))
    W = fr.quadrature_weights()
    return float(torch.sqrt((W * (q - qe) ** 2).sum() / W.sum()))


@pytest.mark.parametrize("p,ns", [(1, (20, 40)), (2, (20, 40)), (3, (10, 20))])
def test_isentropic_vortex_convergence_order(p, ns):
    """The vortex of Sec. 3.3 is an exact Euler solution advected with the free
    stream; the FR error must fall at least like h^(p+1/2) (DG theory)."""
    e0, e1 = (_vortex_error(n, p) for n in ns)
    order = math.log2(e0 / e1)
    assert order >= p + 0.2, (e0, e1, order)
