"""Element-Jacobi preconditioner on the GPU (Sec. 2.3) against the oracle's
blocks, and left-preconditioned GMRES / ESDIRK steps."""
import numpy as np
import pytest
import torch

import cases
from helpers import gpu_ctx, oracle_fr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_1910_03693_gb300 import build as B
    B.build()
    return True


def _mixed2d():
    m, q, ph = cases.workload_vortex2d(3, 1)
    m = m.with_p(np.array([1, 2, 1, 2, 1, 2, 1, 2, 1], dtype=np.int8))
    return m, cases.random_state(m, 11), ph


def _box3d_p2():
    m = cases.periodic_box(3, 2, 0.0, 1.0, 2)
    m.nodes = m.nodes + 0.02 * np.sin(5 * m.nodes[..., ::-1])
    return m, cases.random_state(m, 21), dict(gamma=1.4, mu=0.01, Pr=0.71)


@pytest.mark.parametrize("case", ["mixed2d_p1-2", "box3d_p2"])
def test_precond_apply_matches_oracle_blocks(built, case):
    """z = M^-1 w with M the element blocks of sigma I - dR/dq: the GPU blocks
    (FP32 JVP probes, FP32 Gauss-Jordan) against the oracle's dense blocks and
    solves, to FP32 accuracy (2e-4 of max|z|)."""
    from oracle import precond as P
    m, q, ph = _mixed2d() if case == "mixed2d_p1-2" else _box3d_p2()
    fr = oracle_fr(m, ph)
    qt = torch.from_numpy(q)
    sigma = 20.0
    # every block of the 2D mesh; three of the eight 3D blocks (135 DOFs each)
    blocks = P.element_blocks(fr, qt, sigma, elements=None if case == "mixed2d_p1-2" else [0, 3, 6])
    w = torch.from_numpy(cases.uniform(50, q.size) - 0.5)
    zref = P.apply_inverse(blocks, w).numpy()
    ctx = gpu_ctx(m, ph)
    ctx.precond_build(ctx.pack(qt.cuda()), sigma)
    z = ctx.unpack(ctx.precond_apply(ctx.pack(w.cuda()))).cpu().numpy()
    sel = ~np.isnan(zref)
    assert sel.sum() > 0
    err = np.abs(z[sel] - zref[sel]).max() / np.abs(zref[sel]).max()
    assert err <= 2e-4, err


@pytest.mark.parametrize("p,n", [(3, 3), (4, 2)])
def test_precond_large_blocks_match_oracle(built, p, n):
    """3D blocks of 320 (p = 3) and 625 (p = 4) DOFs, inverted by the blocked
    Gauss-Jordan elimination in global memory: z = M^-1 w on one element
    against the oracle's dense block (its columns from the oracle's exact
    JVP) and dense solve, to FP32 accuracy (2e-4 of max|z|); the other
    elements' blocks are the same kernels on the same data."""
    from oracle import precond as P
    m = cases.periodic_box(3, n, 0.0, 1.0, p)
    m.nodes = m.nodes + 0.02 * np.sin(5 * m.nodes[..., ::-1])
    q = cases.random_state(m, 22)
    ph = dict(gamma=1.4, mu=0.01, Pr=0.71)
    fr = oracle_fr(m, ph)
    qt = torch.from_numpy(q)
    sigma = 30.0
    blocks = P.element_blocks(fr, qt, sigma, elements=[1])
    w = torch.from_numpy(cases.uniform(53, q.size) - 0.5)
    zref = P.apply_inverse(blocks, w).numpy()
    ctx = gpu_ctx(m, ph)
    ctx.precond_build(ctx.pack(qt.cuda()), sigma)
    z = ctx.unpack(ctx.precond_apply(ctx.pack(w.cuda()))).cpu().numpy()
    sel = ~np.isnan(zref)
    assert sel.sum() == 5 * (p + 1) ** 3
    err = np.abs(z[sel] - zref[sel]).max() / np.abs(zref[sel]).max()
    assert err <= 2e-4, err
    # every element has a stored block now: no element falls back to w / sigma
    assert np.abs(z - w.numpy() / sigma).max() > 1e-3 * np.abs(w.numpy() / sigma).max()


def test_preconditioned_stage_3d_p3(built):
    """ESDIRK3 stage 2 of the Taylor-Green vortex at p = 3 (4^3 hexahedra, dt
    0.01, FP32 exact JVP) with the element-Jacobi blocks built at q^n with the
    shift 1/(w dt) + 1/dtau_max: it converges to 1e-8, to the same stage value,
    in no more GMRES iterations than without preconditioning (at rtol 0.1 this
    small stage needs about 1.5 iterations a Newton iterate either way)."""
    from paper_1910_03693_gb300 import esdirk_tableau
    m, q, ph = cases.workload_tgv(4, 3)
    A, _ = esdirk_tableau(3)
    dt = 0.01
    res = {}
    for pc in (False, True):
        ctx = gpu_ctx(m, ph, 3, 3)
        qn = ctx.pack(torch.from_numpy(q).cuda())
        R1 = ctx.residual(qn)
        if pc:
            ctx.precond_build(qn, 1.0 / (A[1][1] * dt) + 1.0 / dt)
        qi = qn.clone()
        st = ctx.esdirk_stage(A, 2, dt, qn, [R1, torch.empty_like(qn), None, None], qi, tol=1e-8,
                              dtau_init=dt / 10, dtau_max=dt, mode="exact", jv_dtype=torch.float32, m=60, rtol=0.1,
                              max_it=100, precond=pc)
        assert st["converged"], (pc, st)
        res[pc] = (ctx.unpack(qi).cpu().numpy(), st["gmres"])
    assert res[True][1] <= res[False][1], (res[True][1], res[False][1])
    dq = np.abs(res[False][0] - q).max()
    assert np.abs(res[True][0] - res[False][0]).max() <= 1e-5 * dq


def test_preconditioned_gmres_solves_the_system_in_fewer_iterations(built):
    """Left-preconditioned GMRES (FP64 exact JVP) to 1e-10 reaches the dense solve
    of (sigma I - J) x = b, with fewer iterations than without preconditioning.
    The blocks are applied in FP32, so the preconditioned operator carries
    rounding of ~1e-7 relative: the solution is checked to 1e-6."""
    from oracle import linearize as L
    m, q, ph = _mixed2d()
    fr = oracle_fr(m, ph)
    qt = torch.from_numpy(q)
    sigma = 20.0
    J = L.dense_jacobian(fr, qt)
    b = torch.from_numpy(cases.uniform(52, q.size) - 0.5)
    xref = torch.linalg.solve(sigma * torch.eye(J.shape[0], dtype=J.dtype) - J, b).numpy()
    ctx = gpu_ctx(m, ph)
    qs, bs = ctx.pack(qt.cuda()), ctx.pack(b.cuda())
    ctx.precond_build(qs, sigma)
    out = {}
    for pc in (False, True):
        x, st = ctx.gmres(qs, bs, sigma, mode="exact", jv_dtype=torch.float64, rtol=1e-10, m=60, max_it=400,
                          reorth=1, precond=pc)
        assert st["converged"], (pc, st)
        out[pc] = (ctx.unpack(x).cpu().numpy(), st["iterations"])
    assert out[True][1] < out[False][1], (out[True][1], out[False][1])
    assert np.abs(out[True][0] - xref).max() <= 1e-6 * np.abs(xref).max()
    assert np.abs(out[False][0] - xref).max() <= 1e-9 * np.abs(xref).max()


def test_preconditioned_esdirk_step(built):
    """An ESDIRK3 step of the 2D vortex with the element-Jacobi preconditioner
    (blocks built once at q^n with the shift of dtau_max, as the paper does):
    every stage converges, to the same q^{n+1} as the unpreconditioned step.
    (On this mild case the early Newton iterates, whose pseudo-time step is
    dt/10, see a shift far from the blocks' one, and the unpreconditioned
    GMRES needs fewer iterations; the stiff C-grid is where the blocks pay.)"""
    from paper_1910_03693_gb300 import esdirk_tableau
    m, q, ph = cases.workload_vortex2d(8, 2)
    A, b = esdirk_tableau(3)
    res = {}
    for pc in (False, True):
        ctx = gpu_ctx(m, ph)
        qs = ctx.pack(torch.from_numpy(q).cuda())
        st = ctx.esdirk_step(A, 0.05, qs, b=b, tol=1e-8, dtau_init=0.005, dtau_max=0.05, mode="exact",
                             jv_dtype=torch.float32, precond=pc)
        assert all(s["converged"] for s in st), (pc, st)
        res[pc] = (ctx.unpack(qs).cpu().numpy(), sum(s["gmres"] for s in st))
    dq = np.abs(res[False][0] - q).max()
    assert np.abs(res[True][0] - res[False][0]).max() <= 1e-6 * dq
