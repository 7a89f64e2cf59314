"""Pins of the oracle's Roe flux (Sec. 2.2, Roe 1981) by what fixes it
independently of its own formulas: Roe's property of the averaged Jacobian
(taken by automatic differentiation of the flux), the eigenvectors against
that Jacobian, |A| against a numerical eigendecomposition, consistency,
upwinding in supersonic flow, the FR residual's invariants with Roe, and
its linearisation (central-difference step sweep, adjoint identity)."""
import math

import numpy as np
import pytest
import torch

import cases
from oracle.fr import FR
from oracle.physics import Euler

G = 1.4


def _cons(rho, u, p):
    E = p / ((G - 1.0) * rho) + 0.5 * (u * u).sum(1)
    return torch.cat([rho[:, None], rho[:, None] * u, (rho * E)[:, None]], 1)


def _states(nd, seed, n=40, mach=0.5):
    g = torch.Generator().manual_seed(seed)
    r = lambda *s: torch.rand(*s, generator=g, dtype=torch.float64)
    rho = 0.5 + r(n)
    p = 1.0 / G * (0.5 + r(n))
    u = (2 * r(n, nd) - 1) * mach
    qL = _cons(rho, u, p)
    qR = _cons(rho * (0.7 + 0.6 * r(n)), u + (2 * r(n, nd) - 1) * 0.3 * mach, p * (0.7 + 0.6 * r(n)))
    nrm = torch.randn(n, nd, generator=g, dtype=torch.float64)
    nrm = nrm / nrm.norm(dim=1, keepdim=True)
    return qL, qR, nrm


def _jacobian_at(ph, u, H, n):
    """d(f.n)/dq at a conservative state with velocity u and total enthalpy H
    (the Euler flux Jacobian depends on u and H only), by autograd."""
    nd = ph.nd
    E = (H + 0.5 * (G - 1.0) * (u * u).sum(-1)) / G
    A = []
    for i in range(u.shape[0]):
        q0 = torch.cat([torch.ones(1, dtype=torch.float64), u[i], E[i:i + 1]])
        fn = lambda q: (ph.flux(q[None])[0] * n[i][:, None]).sum(0)
        A.append(torch.autograd.functional.jacobian(fn, q0))
    return torch.stack(A)


def _fn(ph, q, n):
    return (ph.flux(q) * n[:, :, None]).sum(1)


@pytest.mark.parametrize("nd", [2, 3])
def test_roe_property_of_the_averaged_jacobian(nd):
    """f.n(qR) - f.n(qL) = A(Roe average) (qR - qL) exactly (Roe 1981): a wrong
    average (arithmetic instead of sqrt(rho) weights, static instead of total
    enthalpy) fails it."""
    ph = Euler(nd, G, flux="roe")
    qL, qR, n = _states(nd, 1)
    u, H, c = ph.roe_average(qL, qR)
    A = _jacobian_at(ph, u, H, n)
    lhs = _fn(ph, qR, n) - _fn(ph, qL, n)
    rhs = (A @ (qR - qL)[:, :, None])[:, :, 0]
    assert torch.allclose(lhs, rhs, rtol=0, atol=1e-13 * float(lhs.abs().max()))


@pytest.mark.parametrize("nd", [2, 3])
def test_eigenvectors_diagonalise_the_averaged_jacobian(nd):
    ph = Euler(nd, G, flux="roe")
    qL, qR, n = _states(nd, 2)
    u, H, c = ph.roe_average(qL, qR)
    A = _jacobian_at(ph, u, H, n)
    lam, R = ph.roe_eigensystem(u, H, c, n)
    assert torch.allclose(A @ R, R * lam[:, None, :], rtol=0, atol=1e-12 * float(A.abs().max()))
    assert float(torch.linalg.det(R).abs().min()) > 1e-6


@pytest.mark.parametrize("nd", [2, 3])
def test_dissipation_equals_absolute_jacobian_from_a_numerical_eigendecomposition(nd):
    """R |Lambda| R^-1 (qR - qL) against V |D| V^-1 (qR - qL) with (D, V) from
    torch.linalg.eig of the autograd Jacobian."""
    ph = Euler(nd, G, flux="roe")
    qL, qR, n = _states(nd, 3)
    u, H, c = ph.roe_average(qL, qR)
    A = _jacobian_at(ph, u, H, n)
    D, V = torch.linalg.eig(A)
    absA = (V @ torch.diag_embed(D.real.abs().to(V.dtype)) @ torch.linalg.inv(V)).real
    F = ph.roe(qL, qR, n)
    Fref = 0.5 * (_fn(ph, qL, n) + _fn(ph, qR, n)) - 0.5 * (absA @ (qR - qL)[:, :, None])[:, :, 0]
    assert torch.allclose(F, Fref, rtol=0, atol=1e-10 * float(Fref.abs().max()))


@pytest.mark.parametrize("nd", [2, 3])
def test_consistency_and_supersonic_upwinding(nd):
    ph = Euler(nd, G, flux="roe")
    qL, qR, n = _states(nd, 4)
    assert torch.allclose(ph.roe(qL, qL, n), _fn(ph, qL, n), rtol=0, atol=1e-14 * float(qL.abs().max()) * 10)
    # Mach ~2.5 along n on both sides: every eigenvalue of the average has one sign
    g = torch.Generator().manual_seed(5)
    rho = 1.0 + torch.rand(30, generator=g, dtype=torch.float64)
    p = torch.full((30,), 1.0 / G, dtype=torch.float64)
    nn = torch.randn(30, nd, generator=g, dtype=torch.float64)
    nn = nn / nn.norm(dim=1, keepdim=True)
    u = 2.5 * nn + 0.1 * torch.randn(30, nd, generator=g, dtype=torch.float64)
    a = _cons(rho, u, p)
    b = _cons(rho * 1.2, u * 1.05, p * 0.9)
    ua, Ha, ca = ph.roe_average(a, b)
    assert bool(((ua * nn).sum(1) - ca > 0).all())
    assert torch.allclose(ph.roe(a, b, nn), _fn(ph, a, nn), rtol=0, atol=1e-12 * float(_fn(ph, a, nn).abs().max()))
    assert torch.allclose(ph.roe(a, b, -nn), _fn(ph, b, -nn), rtol=0, atol=1e-12 * float(_fn(ph, b, nn).abs().max()))


@pytest.mark.parametrize("nd", [2, 3])
def test_roe_is_antisymmetric_under_exchange_of_sides(nd):
    ph = Euler(nd, G, flux="roe")
    qL, qR, n = _states(nd, 6)
    assert torch.allclose(ph.roe(qL, qR, n), -ph.roe(qR, qL, -n), rtol=0,
                          atol=1e-13 * float(ph.roe(qL, qR, n).abs().max()))


def _fr(m, mu=0.0, q_inf=None):
    return FR(m, Euler(m.nd, G, mu, 0.71, q_inf, flux="roe"))


@pytest.mark.parametrize("builder", [
    lambda: cases.workload_vortex2d(6, 2)[0].with_p((cases.uniform(5, 36) * 4 + 1).astype(np.int8)),
    lambda: cases.periodic_box(3, 3, 0.0, 1.0, 1).with_p((cases.uniform(6, 27) * 3 + 1).astype(np.int8)),
])
def test_free_stream_preservation_with_roe(builder):
    m = builder()
    fr = _fr(m, 1e-2, cases.free_stream_q(m.nd, vel=(0.3, 0.2, 0.1), mach=0.3))
    q = torch.from_numpy(cases.freestream_state(m, vel=(0.3, 0.2, 0.1), mach=0.3))
    assert float(fr.residual(q).abs().max()) <= 1e-12 * (1.0 / (1.4 * 0.09)) / 0.005


@pytest.mark.parametrize("nd", [2, 3])
def test_conservation_periodic_with_roe(nd):
    if nd == 2:
        m = cases.workload_vortex2d(5, 2)[0]
    else:
        m = cases.periodic_box(3, 3, 0.0, 1.0, 2)
        m.nodes = m.nodes + 0.03 * np.sin(7 * m.nodes[..., ::-1])
    m = m.with_p((cases.uniform(11, m.n_elem) * 3 + 1).astype(np.int8))
    fr = _fr(m, 0.05)
    R = fr.residual(torch.from_numpy(cases.random_state(m, 3)))
    parts = fr.to_groups(fr.quadrature_weights() * R)
    tot = sum(t.flatten(2).sum(dim=(0, 2)) for t in parts.values())
    scale = sum(t.abs().flatten(2).sum(dim=(0, 2)) for t in parts.values())
    assert torch.all(tot.abs() <= 1e-13 * scale), (tot, scale)


def test_rotation_equivariance_with_roe():
    """The tangent frame of the shear waves is chosen per face from the normal
    alone; R |Lambda| R^-1 must not depend on it, so rotating mesh and
    velocity rotates the momentum residual."""
    m = cases.periodic_box(3, 2, 0.0, 1.0, 2)
    a = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    Rm = np.eye(3) + math.sin(0.9) * K + (1 - math.cos(0.9)) * K @ K
    q = cases.random_state(m, 5).reshape(-1, 5)
    R0 = _fr(m, 0.05).residual(torch.from_numpy(q.reshape(-1))).numpy().reshape(-1, 5)
    mr = cases.Mesh(m.nd, m.geom_order, m.nodes @ Rm.T, m.nbr, m.nbr_face, m.orient, m.p)
    qr = q.copy()
    qr[:, 1:4] = q[:, 1:4] @ Rm.T
    R1 = _fr(mr, 0.05).residual(torch.from_numpy(qr.reshape(-1))).numpy().reshape(-1, 5)
    Rexp = R0.copy()
    Rexp[:, 1:4] = R0[:, 1:4] @ Rm.T
    assert np.abs(R1 - Rexp).max() <= 1e-11 * np.abs(R0).max()


def test_roe_differs_from_rusanov():
    """The two fluxes are different operators (the flux selection is live)."""
    m = cases.workload_vortex2d(4, 2)[0]
    q = torch.from_numpy(cases.random_state(m, 8))
    Rr = FR(m, Euler(2, G, flux="rusanov")).residual(q)
    Ro = FR(m, Euler(2, G, flux="roe")).residual(q)
    assert float((Rr - Ro).abs().max()) > 1e-3 * float(Rr.abs().max())


def _small_roe(nd, mu):
    if nd == 2:
        m, q, _ = cases.workload_vortex2d(3, 2)
        m = m.with_p(np.array([1, 2, 3, 2, 1, 2, 3, 2, 1], dtype=np.int8))
        q = cases.random_state(m, 2)
    else:
        m, q, _ = cases.workload_diff(2, 2)
    return FR(m, Euler(nd, G, mu, 0.71, flux="roe")), torch.from_numpy(q)


@pytest.mark.parametrize("nd,mu", [(2, 0.0), (3, 0.05)])
def test_roe_jvp_matches_finite_difference_sweep(nd, mu):
    """The oracle's linearisation of the Roe residual (automatic
    differentiation through the eigenvector solve) against central
    differences of the residual itself over a step sweep: the V-curve's
    minimum below 1e-8."""
    from oracle import linearize as L
    fr, q = _small_roe(nd, mu)
    g = torch.Generator().manual_seed(12)
    q = q + 1e-3 * q.abs().mean() * (2 * torch.rand(q.numel(), generator=g, dtype=torch.float64) - 1)
    v = torch.from_numpy(cases.uniform(19, q.numel()) - 0.5) * q.abs().mean()
    Jv = L.jvp(fr, q, v)
    errs = {}
    for k in range(2, 9):
        eps = 10.0 ** -k
        fd = (fr.residual(q + eps * v) - fr.residual(q - eps * v)) / (2 * eps)
        errs[k] = float((fd - Jv).abs().max() / Jv.abs().max())
    best = min(errs.values())
    assert best < 1e-8, errs
    assert errs[2] > 10 * best and errs[8] > 10 * best, errs


@pytest.mark.parametrize("nd", [2, 3])
def test_roe_vjp_dot_product(nd):
    from oracle import linearize as L
    fr, q = _small_roe(nd, 0.05)
    v = torch.from_numpy(cases.uniform(21, q.numel()) - 0.5)
    w = torch.from_numpy(cases.uniform(22, q.numel()) - 0.5)
    lhs = float(torch.dot(w, L.jvp(fr, q, v)))
    rhs = float(torch.dot(L.vjp(fr, q, w), v))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1.0)
