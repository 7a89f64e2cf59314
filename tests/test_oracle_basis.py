"""Pins of the oracle's 1D FR building blocks against closed forms and numpy."""
import math

import numpy as np
import pytest
import torch

from oracle import basis as B


def test_gauss_textbook_values():
    x, w = B.gauss_points(2)
    assert np.allclose(x.numpy(), [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-16)
    assert np.allclose(w.numpy(), [1.0, 1.0], atol=1e-15)
    x, w = B.gauss_points(3)
    assert np.allclose(x.numpy(), [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], atol=1e-16)
    assert np.allclose(w.numpy(), [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


@pytest.mark.parametrize("P", range(1, 8))
def test_gauss_matches_numpy_and_is_exact(P):
    x, w = B.gauss_points(P)
    xr, wr = np.polynomial.legendre.leggauss(P)
    assert np.allclose(x.numpy(), xr, atol=2e-16 * P) and np.allclose(w.numpy(), wr, atol=4e-16 * P)
    for k in range(2 * P):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert float((w * x ** k).sum()) == pytest.approx(exact, abs=1e-14)


@pytest.mark.parametrize("p", range(1, 6))
def test_lagrange_derivative_exact_on_polynomials(p):
    b = B.basis(p)
    rng = np.random.default_rng(p)
    c = rng.standard_normal(p + 1)
    f = sum(c[k] * b.x ** k for k in range(p + 1))
    df = sum(k * c[k] * b.x ** (k - 1) for k in range(1, p + 1))
    assert torch.allclose(b.D @ f, df, atol=1e-12)
    ends = torch.tensor([-1.0, 1.0])
    fe = sum(c[k] * ends ** k for k in range(p + 1))
    dfe = sum(k * c[k] * ends ** (k - 1) for k in range(1, p + 1))
    assert torch.allclose(b.ext @ f, fe, atol=1e-12)
    assert torch.allclose(b.dext @ f, dfe, atol=1e-11)


@pytest.mark.parametrize("p", range(1, 6))
def test_radau_correction_closed_forms(p):
    ends = torch.tensor([-1.0, 1.0])
    gL, gR, dgL, dgR = B.radau_dg(p, ends)
    assert float(gL[0]) == pytest.approx(1.0) and abs(float(gL[1])) < 1e-15
    assert abs(float(gR[0])) < 1e-15 and float(gR[1]) == pytest.approx(1.0)
    assert float(dgR[1]) == pytest.approx((p + 1) ** 2 / 2)
    assert float(dgL[0]) == pytest.approx(-(p + 1) ** 2 / 2)
    b = B.basis(p)
    # g_R' is a degree-p polynomial: its Gauss integral is g_R(1) - g_R(-1) = 1
    assert float((b.w * b.dg[1]).sum()) == pytest.approx(1.0, abs=1e-14)
    assert float((b.w * b.dg[0]).sum()) == pytest.approx(-1.0, abs=1e-14)
    # g_R is orthogonal to P_{p-1}: Radau polynomial property
    xs, ws = B.gauss_points(p + 3)
    _, gRq, _, _ = B.radau_dg(p, xs)
    for m in range(p):
        Pm, _ = B.legendre(m, xs)
        assert abs(float((ws * gRq * Pm).sum())) < 1e-14


@pytest.mark.parametrize("p", range(1, 5))
def test_modal_roundtrip_and_mortar_projection(p):
    b = B.basis(p)
    s = torch.linspace(-1, 2, p + 1) ** 2
    assert torch.allclose(b.to_nodal @ (b.to_modal @ s), s, atol=1e-13)
    I, Pi = B.mortar_ops(p, p + 1)
    assert torch.allclose(Pi @ I, torch.eye(p + 1), atol=1e-13)   # projection of an interpolant returns it
    bm = B.basis(p + 1)
    # the projection keeps the face integral of any mortar function
    f = torch.cos(3 * bm.x)
    assert float((b.w * (Pi @ f)).sum()) == pytest.approx(float((bm.w * f).sum()), abs=1e-14)
