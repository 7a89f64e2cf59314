"""Pin of the oracle's wall boundary (the paper's no-slip adiabatic wall,
Sec. 4.1; ghost state with rho and rho E kept and the momentum reversed, no
energy viscous flux through the wall): on a box closed by walls in one
direction and periodic in the others, mass and total energy are conserved to
round-off by the FR residual, inviscid and viscous, while the momentum
normal to the wall is not (the wall pushes on the fluid).  Planted mistakes
(momentum not reversed, rho E reversed, heat flux left through the wall) each
break one of the conservation checks."""
import numpy as np
import pytest
import torch

import cases
from oracle.fr import FR
from oracle.physics import Euler


def _walled_box(nd, p, mixed=False):
    """Walls at y = 0 and y = 1 (faces 2, 3); periodic in x (and z)."""
    n = 3

    def pmap(S):
        X = S.copy()
        X[..., 0] = S[..., 0] + 0.2 * S[..., 1]            # sheared: walls not axis-aligned in x
        return X

    periodic = [True, False] + ([True] if nd == 3 else [])
    lo = [0, cases.WALL] + ([0] if nd == 3 else [])
    m = cases._structured(nd, [n] * nd, 1, pmap, periodic, lo, lo, p, "walled")
    if mixed:
        m = m.with_p((cases.uniform(13, m.n_elem) * 3 + 1).astype(np.int8))
    return m


def _totals(nd, mu, mixed, seed=4):
    m = _walled_box(nd, 2, mixed)
    fr = FR(m, Euler(nd, 1.4, mu, 0.71))
    q = torch.from_numpy(cases.random_state(m, seed, amp=0.1))
    parts = fr.to_groups(fr.quadrature_weights() * fr.residual(q))
    tot = sum(t.flatten(2).sum(dim=(0, 2)) for t in parts.values())
    scale = sum(t.abs().flatten(2).sum(dim=(0, 2)) for t in parts.values())
    return (tot.abs() / scale).numpy()


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("mu", [0.0, 0.05])
@pytest.mark.parametrize("nd", [2, 3])
def test_walls_conserve_mass_and_energy(nd, mu, mixed):
    rel = _totals(nd, mu, mixed)
    assert rel[0] <= 1e-13 and rel[nd + 1] <= 1e-13, rel
    assert rel[2] > 1e-4, rel          # wall-normal momentum (y) is not conserved


_GHOST = Euler.ghost


def _ghost_momentum_kept(self, q, kind):
    return q.clone() if kind == cases.WALL else _GHOST(self, q, kind)


def _ghost_energy_reversed(self, q, kind):
    g = _GHOST(self, q, kind)
    if kind == cases.WALL:
        g = torch.cat([g[:, :-1], -g[:, -1:]], dim=1)
    return g


@pytest.mark.parametrize("planted,var", [(_ghost_momentum_kept, 0), (_ghost_energy_reversed, -1)])
def test_planted_ghost_mistake_fails(monkeypatch, planted, var):
    monkeypatch.setattr(Euler, "ghost", planted)
    rel = _totals(2, 0.0, False)
    assert rel[var] > 1e-6, rel


def test_planted_heat_flux_through_wall_fails(monkeypatch):
    """With the energy row of the viscous wall flux kept, energy leaks."""
    import oracle.fr as ofr
    monkeypatch.setattr(ofr, "WALL", -99)        # the adiabatic branch no longer matches
    rel = _totals(2, 0.05, False, seed=6)
    assert rel[3] > 1e-6, rel
