"""Pins of the oracle's p-adaptation: indicator closed forms, decisions, the
jump-limiting fixed point (brute force), state transfer, bucket order."""
import itertools
import math

import numpy as np
import pytest
import torch

import cases
from oracle import adapt
from oracle.basis import legendre
from oracle.fr import FR
from oracle.physics import Euler


def _fr(m):
    return FR(m, Euler(m.nd, 1.4, 0.0, 0.72))


def _state_from_rhou(m, fn):
    """rho = 1, rho*u = fn(xi coordinates of the reference element), rest constant."""
    out = []
    for e, X in enumerate(cases.solution_point_positions(m)):
        q = np.zeros((len(X), m.nv))
        q[:, 0] = 1.0
        q[:, m.nv - 1] = 10.0
        q[:, 1] = fn(X)
        out.append(q.reshape(-1))
    return np.concatenate(out)


@pytest.mark.parametrize("nd,p", [(2, 1), (2, 3), (3, 2)])
def test_indicator_closed_forms(nd, p):
    # unit box elements [0,1]^nd -> xi = 2x - 1 within element 0 of a 1-element mesh
    m = cases.periodic_box(nd, 1, 0.0, 1.0, p)
    fr = _fr(m)
    # polynomial of degree p-1 per direction: eta = 0
    q = _state_from_rhou(m, lambda X: 1.0 + 0.5 * (2 * X[:, 0] - 1) ** (p - 1))
    assert adapt.indicator(fr, torch.from_numpy(q))[0] == pytest.approx(0.0, abs=1e-26)
    # a L_0 + b L_p(xi): eta = b^2 |L_p|^2 / (a^2 |L_0|^2 + b^2 |L_p|^2), |L_m|^2 = 2/(2m+1)
    a, b = 0.7, 0.4
    q = _state_from_rhou(m, lambda X: a + b * legendre(p, torch.from_numpy(2 * X[:, 0] - 1))[0].numpy())
    expect = b * b * 2 / (2 * p + 1) / (a * a * 2 + b * b * 2 / (2 * p + 1))
    assert adapt.indicator(fr, torch.from_numpy(q))[0] == pytest.approx(expect, rel=1e-12)
    # pure top mode in the last direction: eta = 1
    q = _state_from_rhou(m, lambda X: legendre(p, torch.from_numpy(2 * X[:, nd - 1] - 1))[0].numpy())
    assert adapt.indicator(fr, torch.from_numpy(q))[0] == pytest.approx(1.0, rel=1e-12)
    # zero variable: eta = 0 by definition
    q = _state_from_rhou(m, lambda X: 0.0 * X[:, 0])
    assert adapt.indicator(fr, torch.from_numpy(q))[0] == 0.0


def test_indicator_weighting_uses_jacobian():
    """On a stretched element the weights w|J| matter only through ratios: the
    indicator of a mapped polynomial is invariant under uniform scaling."""
    m = cases.workload_vortex2d(3, 3)[0]
    q = cases.random_state(m, 4)
    e1 = adapt.indicator(_fr(m), torch.from_numpy(q))
    m2 = cases.Mesh(2, 1, m.nodes * 3.0, m.nbr, m.nbr_face, m.orient, m.p)
    e2 = adapt.indicator(_fr(m2), torch.from_numpy(q))
    assert np.allclose(e1, e2, rtol=1e-12)


def test_decide_rules():
    eta = np.array([1.0, 0.2, 0.05, 0.0005, 0.002, 0.1])
    p = np.array([2, 2, 2, 2, 1, 3])
    out = adapt.decide(eta, p, 0.1, 0.001, 1, 3)
    # thresholds 0.1 and 0.001 of eta_max = 1: strict comparisons
    assert out.tolist() == [3, 3, 2, 1, 1, 3]
    assert adapt.decide(np.zeros(3), np.array([1, 2, 3]), p_max=3).tolist() == [1, 2, 3]


def _brute_min_limited(mesh, p0, p_max):
    best = None
    E = mesh.n_elem
    for cand in itertools.product(*[range(int(p0[e]), p_max + 1) for e in range(E)]):
        c = np.array(cand)
        ok = all(abs(c[e] - c[n]) <= 1 for e in range(E) for n in mesh.nbr[e] if n >= 0)
        if ok and (best is None or np.all(c <= best) or c.sum() < best.sum()):
            best = c
    return best


@pytest.mark.parametrize("seed", range(5))
def test_limit_jumps_is_minimal_fixed_point(seed):
    m = cases.periodic_box(2, 3, 0.0, 1.0, 1)
    p0 = 1 + np.floor(cases.uniform(100 + seed, m.n_elem) * 4).astype(np.int64)
    p0 = np.where(cases.uniform(200 + seed, m.n_elem) < 0.7, 1, p0)
    got = adapt.limit_jumps(m, p0)
    ref = _brute_min_limited(m, p0, 4)
    assert np.array_equal(got, ref)
    assert np.all(got >= p0)


@pytest.mark.parametrize("po,pn", [(2, 3), (3, 2), (1, 4), (4, 1)])
def test_transfer_prolong_exact_and_project_is_l2(po, pn):
    nd = 2
    m = cases.periodic_box(nd, 1, 0.0, 1.0, po)
    X = cases.solution_point_positions(m)[0]
    xi = 2 * X - 1
    deg = min(po, pn)
    f = lambda x: 0.3 + x[:, 0] ** deg - 0.4 * x[:, 1] ** max(deg - 1, 0) * x[:, 0]
    s = torch.from_numpy(f(xi).reshape(po + 1, po + 1))
    out = adapt.transfer_element(s, po, pn, nd)
    m2 = m.with_p(pn)
    xi2 = 2 * cases.solution_point_positions(m2)[0] - 1
    # a polynomial of degree <= min(po, pn) is reproduced exactly
    assert np.allclose(out.numpy().reshape(-1), f(xi2), atol=1e-13)
    if pn < po:
        # projecting a top-degree mode removes it: the residual is orthogonal to Q_pn
        g = torch.from_numpy((legendre(po, torch.from_numpy(xi[:, 0]))[0]).numpy().reshape(po + 1, po + 1))
        assert float(adapt.transfer_element(g, po, pn, nd).abs().max()) < 1e-13


def test_bucket_order_is_stable_sort_and_bijection():
    p = np.array([3, 1, 2, 1, 3, 2, 1])
    order = adapt.bucket_order(p)
    assert order.tolist() == [1, 3, 6, 2, 5, 0, 4]
    assert sorted(order.tolist()) == list(range(len(p)))


def test_adapt_state_round_trip_on_vortex():
    """Raise every element then lower it back: the state returns exactly
    (prolongation is exact, projection of the prolonged field recovers it)."""
    m, q, _ = cases.workload_vortex2d(4, 2)
    fr2 = _fr(m)
    fr3 = _fr(m.with_p(3))
    q = torch.from_numpy(q)
    back = adapt.transfer(fr3, adapt.transfer(fr2, q, fr3), fr2)
    assert torch.allclose(back, q, atol=1e-12)


def _filter_mesh():
    """Affine 3D box (|J| constant per element) with degrees 1..4."""
    m = cases.periodic_box(3, 3, 0.0, 1.0, 2)
    m = m.with_p(np.array([1, 2, 3, 4, 3, 2, 1, 4, 3] * 3, dtype=np.int8))
    return m


def test_nodal_filter_pins():
    """Elements of degree <= 2 are untouched; a state of degree p - 1 in every
    element is a fixed point; the element integrals (weights w |J|) of every
    variable are kept (the dropped Legendre modes integrate to zero on affine
    elements); a single top mode is scaled by 1 - alpha."""
    m = _filter_mesh()
    fr = _fr(m)
    q = torch.from_numpy(cases.random_state(m, 61))
    qf = adapt.nodal_filter(fr, q, alpha=0.2, p_above=2)
    parts, fparts = fr.to_groups(q), fr.to_groups(qf)
    for p in parts:
        if p <= 2:
            assert torch.equal(parts[p], fparts[p])
        else:
            assert float((parts[p] - fparts[p]).abs().max()) > 0
    W = fr.quadrature_weights()
    Q, QF, WW = (t.reshape(-1, fr.nv) for t in (q, qf, W))
    off = fr.offsets // fr.nv
    for e in range(m.n_elem):
        a, b = int(off[e]), int(off[e + 1])
        assert torch.allclose((WW[a:b] * QF[a:b]).sum(0), (WW[a:b] * Q[a:b]).sum(0), rtol=0, atol=1e-13)
    # degree p - 1 polynomials: the truncation of any state, filtered again, stays put
    low = {p: (adapt.truncate(s, p, 3) if p > 2 else s) for p, s in parts.items()}
    ql = fr.from_groups(low)
    assert torch.allclose(adapt.nodal_filter(fr, ql, 0.2, 2), ql, rtol=0, atol=1e-13 * float(ql.abs().max()))
    # a pure top mode P_p(xi) P_0(eta) P_p(zeta) is scaled by 1 - alpha
    from oracle.basis import basis as B1
    for p in (3, 4):
        x = B1(p).x
        lp = legendre(p, x)[0]
        mode = lp[:, None, None] * lp[None, None, :] * torch.ones(1, p + 1, 1, dtype=torch.float64)
        s = mode.expand(2, fr.nv, p + 1, p + 1, p + 1).clone()
        f = (1.0 - 0.3) * s + 0.3 * adapt.truncate(s, p, 3)
        assert torch.allclose(f, 0.7 * s, rtol=0, atol=1e-13)
