"""Pins of the oracle's linearisations, GMRES, ESDIRK and pseudo-transient solver."""
import math

import numpy as np
import pytest
import torch

import cases
from oracle import esdirk, krylov
from oracle import linearize as L
from oracle.fr import FR
from oracle.physics import Euler


def _small(nd, mu):
    if nd == 2:
        m, q, _ = cases.workload_vortex2d(3, 2)
        m = m.with_p(np.array([1, 2, 3, 2, 1, 2, 3, 2, 1], dtype=np.int8))
        q = cases.random_state(m, 2)
    else:
        m, q, _ = cases.workload_diff(2, 2)
    return FR(m, Euler(nd, 1.4, mu, 0.71)), torch.from_numpy(q)


@pytest.mark.parametrize("nd,mu", [(2, 0.0), (2, 0.05), (3, 0.05)])
def test_jvp_matches_finite_difference_sweep(nd, mu):
    fr, q = _small(nd, mu)
    v = torch.from_numpy(cases.uniform(9, q.numel()) - 0.5) * q.abs().mean()
    Jv = L.jvp(fr, q, v)
    errs = {}
    for k in range(2, 9):
        eps = 10.0 ** -k
        fd = (fr.residual(q + eps * v) - fr.residual(q - eps * v)) / (2 * eps)
        errs[k] = float((fd - Jv).abs().max() / Jv.abs().max())
    best = min(errs.values())
    assert best < 1e-8, errs
    # V-curve: truncation error on the left, rounding on the right
    kbest = min(errs, key=errs.get)
    assert errs[2] > 10 * best and errs[8] > 10 * best, errs
    # the paper's one-sided form with eps = 1e-6 is first order accurate
    fd1 = L.fd_jv(fr, q, v, 1e-6)
    assert float((fd1 - Jv).abs().max() / Jv.abs().max()) < 1e-4


@pytest.mark.parametrize("nd,mu", [(2, 0.05), (3, 0.05)])
def test_vjp_dot_product_and_dense_transpose(nd, mu):
    fr, q = _small(nd, mu)
    v = torch.from_numpy(cases.uniform(9, q.numel()) - 0.5)
    w = torch.from_numpy(cases.uniform(10, q.numel()) - 0.5)
    lhs = float(torch.dot(w, L.jvp(fr, q, v)))
    rhs = float(torch.dot(L.vjp(fr, q, w), v))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0) * 100
    if nd == 2:
        J = L.dense_jacobian(fr, q)
        assert torch.allclose(L.vjp(fr, q, w), J.T @ w, atol=1e-10 * float(J.abs().max()))


def test_gmres_matches_dense_solve():
    fr, q = _small(2, 0.0)
    J = L.dense_jacobian(fr, q)
    n = J.shape[0]
    A = 20.0 * torch.eye(n) - J
    b = torch.from_numpy(cases.uniform(4, n) - 0.5)
    x, st = krylov.gmres(lambda v: A @ v, b, m=30, rtol=1e-13, max_it=5000)
    assert st["converged"] and st["restarts"] > 1
    xd = torch.linalg.solve(A, b)
    assert float((x - xd).abs().max() / xd.abs().max()) < 1e-11


def test_gmres_stops_at_tolerance_and_iteration_cap():
    n = 50
    A = torch.diag(torch.linspace(1.0, 100.0, n))
    b = torch.ones(n)
    x, st = krylov.gmres(lambda v: A @ v, b, m=10, rtol=1e-1, max_it=100)
    r = float(torch.linalg.vector_norm(b - A @ x) / torch.linalg.vector_norm(b))
    assert st["converged"] and r <= 1e-1 + 1e-12
    x, st = krylov.gmres(lambda v: A @ v, b, m=5, rtol=1e-14, max_it=7)
    assert not st["converged"] and st["iterations"] == 7


@pytest.mark.parametrize("tab", [esdirk.esdirk2(), esdirk.esdirk3()])
def test_tableau_order_conditions_and_l_stability(tab):
    for k, r in esdirk.order_condition_residuals(tab).items():
        assert abs(r) < 1e-15, k
    assert tab.A[0][0] == 0.0 and all(tab.A[i][i] == tab.A[1][1] for i in range(1, tab.s))
    assert tab.A[-1] == tab.b                        # stiffly accurate
    assert abs(esdirk.stability_function(tab, -1e9)) < 1e-6
    for y in np.linspace(0.0, 200.0, 401):
        assert abs(esdirk.stability_function(tab, 1j * y)) <= 1.0 + 1e-12
    for x in np.linspace(-50.0, 0.0, 51):
        assert abs(esdirk.stability_function(tab, x)) <= 1.0 + 1e-12


def test_esdirk3_gamma_root():
    g = esdirk.esdirk3_gamma()
    assert abs(6 * g ** 3 - 18 * g ** 2 + 9 * g - 1) < 1e-15 and 0.43 < g < 0.44


def _prothero_robinson(lam, tab, dt, T=1.0):
    """y' = lam (y - cos t) - sin t, y(0) = 1 (exact y = cos t), written
    autonomously as (y, t)' = (lam (y - cos t) - sin t, 1)."""
    def R(q):
        y, t = q[0], q[1]
        return torch.stack([lam * (y - torch.cos(t)) - torch.sin(t), torch.ones_like(t)])

    def jv(q, v, Rq):
        return torch.func.jvp(R, (q,), (v,))[1]

    opts = esdirk.NewtonOpts(tol=1e-13, dtau_init=1e3, dtau_max=1e6, gmres_rtol=1e-12)
    q = torch.tensor([1.0, 0.0])
    for _ in range(int(round(T / dt))):
        q, _ = esdirk.esdirk_step(R, jv, q, tab, dt, opts)
    return abs(float(q[0]) - math.cos(T))


@pytest.mark.parametrize("tab,order", [(esdirk.esdirk2(), 2), (esdirk.esdirk3(), 3)])
def test_esdirk_order_on_prothero_robinson(tab, order):
    e = [_prothero_robinson(-1.0, tab, dt) for dt in (0.1, 0.05, 0.025)]
    slopes = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(slopes) > order - 0.2, (e, slopes)
    # stiff case: stays accurate (stiffly accurate, L-stable)
    assert _prothero_robinson(-1e5, tab, 0.1) < 1e-3


def test_pseudo_transient_stage_reaches_tolerance():
    """One ESDIRK3 stage of the 2D vortex by pseudo-transient continuation with
    the paper's FD Jv: the stage residual F falls by 1e-8 and q solves F(q) = 0."""
    m, q, _ = cases.workload_vortex2d(4, 2)
    fr = FR(m, Euler(2, 1.4, 0.0, 0.72))
    qn = torch.from_numpy(q)
    tab = esdirk.esdirk3()
    Rn = fr.residual(qn)
    opts = esdirk.NewtonOpts(tol=1e-8, dtau_init=0.05, dtau_max=10.0, gmres_m=30)
    jv = lambda qq, v, Rq: L.fd_jv(fr, qq, v, 1e-6, Rq)
    q2, R2, st = esdirk.solve_stage(fr.residual, jv, qn, [Rn], 1, tab, 0.05, qn, opts)
    assert st["converged"] and st["final_norm"] <= 1e-8 * st["norms"][0]
    w = tab.A[1][1]
    F = -q2 / (w * 0.05) + fr.residual(q2) + (qn + 0.05 * tab.A[1][0] * Rn) / (w * 0.05)
    assert float(torch.linalg.vector_norm(F)) <= 1.01e-8 * st["norms"][0]


def test_symmetric_taylor_green_sits_on_rusanov_ties():
    """The Taylor-Green state (rho w = 0) puts faces exactly on the kinks of
    |u.n| and max(lam-, lam+): central differences of R do not converge to the
    JVP there, while a seeded additive perturbation restores the V-curve."""
    import cases as C
    m, q, ph = C.workload_tgv(3, 2)
    fr = FR(m, Euler(3, ph["gamma"], ph["mu"], ph["Pr"]))

    def best_fd_error(qq):
        qt = torch.from_numpy(qq)
        v = torch.from_numpy((C.uniform(901, qq.size) - 0.5) * np.abs(qq).mean())
        J = L.jvp(fr, qt, v)
        errs = []
        for k in range(4, 9):
            eps = 10.0 ** -k
            fd = (fr.residual(qt + eps * v) - fr.residual(qt - eps * v)) / (2 * eps)
            errs.append(float((fd - J).abs().max() / J.abs().max()))
        return min(errs)

    assert best_fd_error(q) > 1e-6
    qg = q + 1e-3 * np.abs(q).mean() * (2.0 * C.uniform(77, q.size) - 1.0)
    assert best_fd_error(qg) < 1e-7
