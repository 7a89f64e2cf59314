"""Pin of the oracle's Euler Rusanov flux (the common inviscid flux of the
hot-path workloads): its wave speed |u.n| + c must be the spectral radius of
the normal flux Jacobian d(f.n)/dq, taken here by automatic differentiation of
the flux and ``torch.linalg.eigvals``; and for a small jump delta the
dissipation (F(q, q + delta) - (f(q) + f(q + delta)).n / 2) / delta must tend
to -lambda/2 with that independent lambda.  Planted mistakes (c without gamma,
dissipation without its factor 1/2) fail one of them."""
import pytest
import torch

from oracle.physics import Euler

G = 1.4


def _states(nd, seed, n=30):
    g = torch.Generator().manual_seed(seed)
    r = lambda *s: torch.rand(*s, generator=g, dtype=torch.float64)
    rho = 0.5 + r(n)
    p = (0.5 + r(n)) / G
    u = (2 * r(n, nd) - 1) * 0.8
    E = p / ((G - 1) * rho) + 0.5 * (u * u).sum(1)
    q = torch.cat([rho[:, None], rho[:, None] * u, (rho * E)[:, None]], 1)
    nrm = torch.randn(n, nd, generator=g, dtype=torch.float64)
    return q, nrm / nrm.norm(dim=1, keepdim=True)


def _spectral_radius(ph, q, n):
    out = []
    for i in range(q.shape[0]):
        fn = lambda x: (ph.flux(x[None])[0] * n[i][:, None]).sum(0)
        A = torch.autograd.functional.jacobian(fn, q[i])
        out.append(torch.linalg.eigvals(A).abs().max())
    return torch.stack(out)


def _wave_speed_error(ph, nd):
    q, n = _states(nd, 1)
    lam = ph.wave_speed(q, n)
    ref = _spectral_radius(ph, q, n)
    return float(((lam - ref).abs() / ref).max())


def _dissipation_limit_error(ph, nd, h=1e-7):
    q, n = _states(nd, 2)
    ref = _spectral_radius(ph, q, n)
    g = torch.Generator().manual_seed(3)
    d = h * q.abs().max(1, keepdim=True).values * (2 * torch.rand(q.shape, generator=g, dtype=torch.float64) - 1)
    fn = lambda x: (ph.flux(x) * n[:, :, None]).sum(1)
    diss = ph.rusanov(q, q + d, n) - 0.5 * (fn(q) + fn(q + d))
    ratio = diss / d                                   # every component: -lambda/2
    return float(((ratio + 0.5 * ref[:, None]).abs() / ref[:, None]).max())


@pytest.mark.parametrize("nd", [2, 3])
def test_wave_speed_is_spectral_radius_of_normal_flux_jacobian(nd):
    assert _wave_speed_error(Euler(nd, G), nd) <= 1e-12


@pytest.mark.parametrize("nd", [2, 3])
def test_small_jump_dissipation_tends_to_minus_half_lambda(nd):
    assert _dissipation_limit_error(Euler(nd, G), nd) <= 1e-5


def test_planted_sound_speed_without_gamma_fails(monkeypatch):
    def wave_speed(self, q, n):
        rho, vel, pres = self.primitives(q)
        un = (vel * n).sum(1)
        return torch.where(un < 0, -un, un) + torch.sqrt(pres / rho)
    monkeypatch.setattr(Euler, "wave_speed", wave_speed)
    assert _wave_speed_error(Euler(3, G), 3) > 1e-2


def test_planted_dissipation_factor_fails(monkeypatch):
    orig = Euler.rusanov
    def rusanov(self, qL, qR, n):
        fL = (self.flux(qL) * n[:, :, None]).sum(1)
        fR = (self.flux(qR) * n[:, :, None]).sum(1)
        return 2.0 * orig(self, qL, qR, n) - 0.5 * (fL + fR)
    monkeypatch.setattr(Euler, "rusanov", rusanov)
    assert _dissipation_limit_error(Euler(2, G), 2) > 0.5
