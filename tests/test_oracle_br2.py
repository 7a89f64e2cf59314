"""Pin of the oracle's BR2 common gradient (Sec. 2.2, Eq. com_grad_q, with the
face-local lifting r = g_s'(face) (S_d/|J|) (q^com - q) of the design's
reading): FR with the DG correction functions must reproduce, to round-off,
an independent DG discretisation of scalar diffusion with Bassi and Rebay's
BR2 lifting written as a weak form (``oracle.dg.dg_br2_diffusion_residual``).
Parallelograms of different sizes make the lifting's |J| and area terms
differ between the two sides of a face; planted mistakes in the lifting
(penalty 2, flipped sign) fail the check."""
import numpy as np
import pytest
import torch

import cases
from oracle.basis import basis
from oracle.dg import dg_br2_diffusion_residual
from oracle.fr import FR
from oracle.physics import Diffusion

MU = 0.7


def _sheared_nonuniform_box(p, n=4):
    """Periodic parallelogram mesh with element sizes varying in both directions."""
    def pmap(S):
        x = S[..., 0] + 0.08 * np.sin(2 * np.pi * S[..., 0])
        y = S[..., 1] + 0.06 * np.sin(2 * np.pi * S[..., 1])
        return np.stack([x + 0.3 * y, y], -1)
    return cases._structured(2, [n, n], 1, pmap, [True, True], [0, 0], [0, 0], p, "br2")


def _fr_vs_dg(p):
    m = _sheared_nonuniform_box(p)
    q = torch.from_numpy(cases.uniform(3, int(m.n_sp().sum())) - 0.5)
    R_fr = FR(m, Diffusion(2, MU)).residual(q).numpy()
    R_dg = dg_br2_diffusion_residual(m, q.numpy(), MU)
    return np.abs(R_fr - R_dg).max() / np.abs(R_fr).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fr_br2_equals_dg_br2_scalar_diffusion(p):
    assert _fr_vs_dg(p) <= 1e-13


def test_elements_differ_in_size():
    """The check is not vacuous for the |J| terms: the element Jacobians differ."""
    m = _sheared_nonuniform_box(2)
    X = m.nodes
    a, b = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
    det = np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    assert det.max() / det.min() > 1.5


@pytest.mark.parametrize("factor", [2.0, -1.0])
def test_planted_lifting_mistake_fails(monkeypatch, factor):
    """g_s'(face) scaled (penalty 2) or negated in the oracle's lifting."""
    for p in (1, 2):
        b = basis(p)
        monkeypatch.setattr(b, "dg_face", b.dg_face * factor)
    assert _fr_vs_dg(1) > 1e-2 and _fr_vs_dg(2) > 1e-2
