"""The differentiation check of the workload on 24^3 hexahedra at p = 4 with
the integrated kinetic-energy functional

    Phi(q) = sum_sp w |J| (1/2) |rho u|^2 / rho    evaluated on  q~ = q + dt R(q)

(the reading of "integrated kinetic-energy functional": the quadrature of the
FR solution's kinetic energy after one explicit step of size dt).  Its
gradient, grad Phi = (I + dt dR/dq)^T grad K(q~), is formed by the chain rule
with the library's VJP behind torch.autograd (``autograd_residual``), FP64 and
FP32, and checked against the oracle's gradient by automatic differentiation
of the oracle residual; the GPU's own Phi is checked by directional central
differences over a step sweep (1e-2 .. 1e-8), whose error must trace the
V-curve: truncation error falling as h^2, rounding error rising as 1/h.
"""
import numpy as np
import pytest
import torch

import cases
from helpers import generic_state, gpu_ctx, oracle_fr

pytestmark = pytest.mark.gpu

DT = 0.01


@pytest.fixture(scope="module")
def diff():
    from paper_1910_03693_gb300 import build as B
    B.build()
    m, q, ph = cases.workload_diff()          # 13,824 hexahedra, p = 4, 8,640,000 DOF
    qg = generic_state(q)                     # away from Rusanov's ties (see helpers)
    fr = oracle_fr(m, ph)
    W = fr.quadrature_weights()
    # oracle gradient of Phi by reverse-mode automatic differentiation
    qt = torch.from_numpy(qg).clone().requires_grad_(True)
    phi = _phi_canonical(fr.residual(qt), qt, W, m.nd)
    (g_ref,) = torch.autograd.grad(phi, qt)
    ctx = gpu_ctx(m, ph, 4, 4)
    return m, qg, ph, ctx, W, float(phi.detach()), g_ref.numpy()


def _phi_canonical(R, q, W, nd):
    nv = nd + 2
    qt = (q + DT * R).reshape(-1, nv)
    mom = qt[:, 1:1 + nd]
    return (W.reshape(-1, nv)[:, 0] * 0.5 * (mom * mom).sum(1) / qt[:, 0]).sum()


def _state_selectors(ctx, nd):
    """Boolean masks of rho and rho u_i in the state layout (from the packed
    variable index of every canonical value)."""
    nv = nd + 2
    vid = torch.arange(ctx.n_dof, dtype=torch.float64, device="cuda") % nv
    vs = ctx.pack(vid)
    return [vs == v for v in range(nv)]


def _phi_gpu(ctx, q, Wst, sel, nd):
    from paper_1910_03693_gb300.api import autograd_residual
    qt = q + DT * autograd_residual(ctx, q)
    mom2 = sum(qt[sel[1 + i]] ** 2 for i in range(nd))
    return (Wst[sel[0]] * 0.5 * mom2 / qt[sel[0]]).sum()


def _grad_gpu(ctx, qg, W, nd, dtype):
    sel = _state_selectors(ctx, nd)
    Wst = ctx.pack(W.cuda(), dtype)
    q = ctx.pack(torch.from_numpy(qg).cuda(), dtype).requires_grad_(True)
    phi = _phi_gpu(ctx, q, Wst, sel, nd)
    (g,) = torch.autograd.grad(phi, q)
    return float(phi.detach()), ctx.unpack(g).cpu().numpy()


def test_functional_gradient_fp64_matches_oracle(diff):
    m, qg, ph, ctx, W, phi_ref, g_ref = diff
    phi, g = _grad_gpu(ctx, qg, W, m.nd, torch.float64)
    assert abs(phi - phi_ref) <= 1e-12 * abs(phi_ref)
    err = np.abs(g - g_ref).max() / np.abs(g_ref).max()
    assert err <= 1e-12, err


def test_functional_gradient_fp32_matches_oracle(diff):
    """FP32 residual and VJP (FP32 arithmetic throughout, q~ and the functional's
    own gradient included) against the oracle's FP64 gradient.  The bound is
    derived, not fitted: the FP32 residual is within 2e-5 of the flux scale of
    the FP64 one (the FP32 parity bound), dt times that error enters q~, and
    grad K = (-|u|^2/2, u, 0) w|J| moves by at most (1 + |u|)/rho times it."""
    from helpers import flux_scale
    m, qg, ph, ctx, W, phi_ref, g_ref = diff
    phi, g = _grad_gpu(ctx, qg, W, m.nd, torch.float32)
    assert abs(phi - phi_ref) <= 1e-5 * abs(phi_ref)
    Q = qg.reshape(-1, m.nd + 2)
    u_max = float(np.abs(Q[:, 1:1 + m.nd] / Q[:, :1]).max())
    dq = DT * 2e-5 * flux_scale(m, qg)
    tol = dq * (1.0 + u_max) / float(Q[:, 0].min()) * float(W.max()) / np.abs(g_ref).max() + 1e-5
    err = np.abs(g - g_ref).max() / np.abs(g_ref).max()
    assert err <= tol, (err, tol)


def test_functional_directional_fd_sweep(diff):
    """<grad Phi, v> from the GPU's VJP against central differences of the GPU's
    own Phi (FP64) for h = 1e-2 .. 1e-11.  The error is measured against
    ||grad Phi|| ||v||, the scale of the inner product's terms: for a random
    direction the inner product itself is ~sqrt(N) smaller, and the rounding
    of Phi would otherwise hide the curve.  Its minimum is below 1e-8 and both
    arms rise at least 10 times above it (the V-curve: truncation falling as
    h^2 from h = 1e-2, rounding rising as 1/h below h = 1e-9)."""
    m, qg, ph, ctx, W, _, _ = diff
    nd = m.nd
    sel = _state_selectors(ctx, nd)
    Wst = ctx.pack(W.cuda())
    q = ctx.pack(torch.from_numpy(qg).cuda()).requires_grad_(True)
    (g,) = torch.autograd.grad(_phi_gpu(ctx, q, Wst, sel, nd), q)
    v = ctx.pack(torch.from_numpy((cases.uniform(908, qg.size) - 0.5) * np.abs(qg).mean()).cuda())
    d_exact = float(torch.dot(g, v))
    scale = float(g.norm() * v.norm())
    errs = {}
    with torch.no_grad():
        for k in range(2, 12):
            h = 10.0 ** -k
            fp = float(_phi_gpu(ctx, q.detach() + h * v, Wst, sel, nd))
            fm = float(_phi_gpu(ctx, q.detach() - h * v, Wst, sel, nd))
            errs[k] = abs((fp - fm) / (2 * h) - d_exact) / scale
    best = min(errs.values())
    assert best <= 1e-8, errs
    assert errs[2] >= 10 * best and max(errs[10], errs[11]) >= 10 * best, errs
