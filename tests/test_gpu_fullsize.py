"""GPU parity at the workloads' full sizes, in the configuration bench.py times.

Every check compares the CUDA path with the FP64 oracle on the same seeded
input: elementwise where the oracle computes the full vector in seconds
(residual, JVP, VJP), by a property that holds at any size otherwise (the
converged ESDIRK stage solves the oracle's stage equation).  Tolerances are
those of the small-size tests (FP64 1e-12 of max|R| or of the flux scale,
1e-11 on curved meshes; double-float 2e-10, 2e-9 curved; FP32 2e-5).
"""
import math

import numpy as np
import pytest
import torch

import cases
from helpers import generic_state, gpu_ctx, oracle_fr, parity_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_1910_03693_gb300 import build as B
    B.build()
    return True


@pytest.fixture(scope="module")
def tgv():
    m, q, ph = cases.workload_tgv()          # 32^3 hexahedra, p = 3, 10,485,760 DOF
    return m, q, ph, oracle_fr(m, ph)


def test_tgv_full_residual(built, tgv):
    m, q, ph, fr = tgv
    ctx = gpu_ctx(m, ph, 3, 3)
    Rref = fr.residual(torch.from_numpy(q)).numpy()
    qd = torch.from_numpy(q).cuda()
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
        R = ctx.unpack(ctx.residual(ctx.pack(qd, dtype))).cpu().numpy()
        ok, rel, fs = parity_ok(R, Rref, m, q, tol)
        assert ok, (str(dtype), rel, fs)


def test_tgv_full_df_residual(built, tgv):
    """The double-float residual the bench's early Newton iterates use."""
    m, q, ph, fr = tgv
    ctx = gpu_ctx(m, ph, 3, 3)
    Rref = fr.residual(torch.from_numpy(q)).numpy()
    R = ctx.unpack(ctx.residual(ctx.pack(torch.from_numpy(q).cuda()), double_float=True)).cpu().numpy()
    ok, rel, fs = parity_ok(R, Rref, m, q, 2e-10)
    assert ok, (rel, fs)


def test_tgv_full_roe_residual(built, tgv):
    """Roe's flux at full size: FP64, double-float and FP32 residuals against
    the oracle's Roe residual (eigenvector matrices and dense solves)."""
    m, q, ph, _ = tgv
    ph = dict(ph, flux="roe")
    Rref = oracle_fr(m, ph).residual(torch.from_numpy(q)).numpy()
    ctx = gpu_ctx(m, ph, 3, 3)
    qd = torch.from_numpy(q).cuda()
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
        R = ctx.unpack(ctx.residual(ctx.pack(qd, dtype))).cpu().numpy()
        ok, rel, fs = parity_ok(R, Rref, m, q, tol)
        assert ok, (str(dtype), rel, fs)
    R = ctx.unpack(ctx.residual(ctx.pack(qd), double_float=True)).cpu().numpy()
    ok, rel, fs = parity_ok(R, Rref, m, q, 2e-10)
    assert ok, ("double-float", rel, fs)


def test_tgv_full_fp32_exact_jvp(built, tgv):
    """The JVP the bench's GMRES applies (FP32, exact), on a generic nearby state."""
    from oracle import linearize as L
    m, q, ph, fr = tgv
    qg = generic_state(q)
    v = cases.uniform(904, q.size) - 0.5
    Jref = L.jvp(fr, torch.from_numpy(qg), torch.from_numpy(v)).numpy()
    ctx = gpu_ctx(m, ph, 3, 3)
    J = ctx.unpack(ctx.jvp(ctx.pack(torch.from_numpy(qg).cuda(), torch.float32),
                           ctx.pack(torch.from_numpy(v).cuda(), torch.float32))).cpu().numpy()
    ok, rel, fs = parity_ok(J, Jref, m, qg, 2e-5)
    assert ok, (rel, fs)


@pytest.mark.parametrize("low_above", [0.0, 1e-8])
def test_tgv_full_stage_solves_oracle_stage_equation(built, tgv, low_above):
    """ESDIRK3 stage 2 exactly as bench.py runs it (dt 0.01, FP32 exact-JVP
    GMRES(60) with one Gram-Schmidt pass, tolerance 1e-8; F in FP64 throughout,
    or double-float until ||F|| <= 1e-8 ||F0|| and FP64 after): the converged
    q^2 makes the oracle's stage residual
    F(q) = -q/(w dt) + R(q) + (q^n + dt a21 R(q^n))/(w dt) small to the same tolerance."""
    from paper_1910_03693_gb300 import esdirk_tableau
    m, q, ph, fr = tgv
    A, _ = esdirk_tableau(3)
    ctx = gpu_ctx(m, ph, 3, 3)
    dt = 0.01
    qn = ctx.pack(torch.from_numpy(q).cuda())
    R1 = ctx.residual(qn)
    qi = qn.clone()
    R2 = torch.empty_like(qn)
    st = ctx.esdirk_stage(A, 2, dt, qn, [R1, R2, None, None], qi, tol=1e-8, dtau_init=dt / 10, dtau_max=dt,
                          mode="exact", jv_dtype=torch.float32, m=60, rtol=0.1, max_it=100, reorth=0,
                          low_above=low_above, low_precision="df")
    assert st["converged"]
    assert (st["low_evaluations"] > 0) == (low_above > 0)
    w = A[1][1]
    qi_h = torch.from_numpy(ctx.unpack(qi).cpu().numpy())
    qn_h = torch.from_numpy(q)
    Rn = fr.residual(qn_h)
    F0 = (-qn_h / (w * dt) + Rn + (qn_h + dt * A[1][0] * Rn) / (w * dt))
    F = (-qi_h / (w * dt) + fr.residual(qi_h) + (qn_h + dt * A[1][0] * Rn) / (w * dt))
    ratio = float(torch.linalg.vector_norm(F) / torch.linalg.vector_norm(F0))
    assert ratio <= 2e-8, ratio


def test_cylinder_full_residual(built):
    m, q, ph = cases.workload_cylinder()      # 98,304 curved hexahedra, p in 1..4
    fr = oracle_fr(m, ph)
    Rref = fr.residual(torch.from_numpy(q)).numpy()
    ctx = gpu_ctx(m, ph, 1, 4)
    qd = torch.from_numpy(q).cuda()
    for dtype, tol in ((torch.float64, 1e-11), (torch.float32, 2e-5)):
        R = ctx.unpack(ctx.residual(ctx.pack(qd, dtype))).cpu().numpy()
        ok, rel, fs = parity_ok(R, Rref, m, q, tol)
        assert ok, (str(dtype), rel, fs)
    R = ctx.unpack(ctx.residual(ctx.pack(qd), double_float=True)).cpu().numpy()   # curved, four buckets
    ok, rel, fs = parity_ok(R, Rref, m, q, 2e-9)
    assert ok, ("double-float", rel, fs)


def test_naca_full_residual_and_adaptation(built):
    """C-grid with wake cut, 393,216 elements at p = 1, then one adaptation pass
    (nu = 0.1, 0.001, p in [1, 4]) on a perturbed state: p-map and bucket
    permutation bit-exact, transferred state and new residual to tolerance."""
    from oracle import adapt
    m, q, ph = cases.workload_naca()
    fr = oracle_fr(m, ph)
    qt = torch.from_numpy(q)
    Rref = fr.residual(qt).numpy()
    ctx = gpu_ctx(m, ph, 1, 4)
    buf = torch.zeros(ctx.n_dof_capacity, dtype=torch.float64, device="cuda")
    ctx.pack(qt.cuda(), out=buf[:ctx.n_dof])
    R = ctx.unpack(ctx.residual(buf[:ctx.n_dof])).cpu().numpy()
    ok, rel, fs = parity_ok(R, Rref, m, q, 1e-11)
    assert ok, (rel, fs)
    p_ref, _ = adapt.adapt_p(fr, qt, 0.1, 0.001, 1, 4)
    eta, emax = ctx.indicator(buf[:ctx.n_dof])
    perm = torch.empty(ctx.n_elem, dtype=torch.int32, device="cuda")
    ctx.rebucket(eta, emax, buf, 0.1, 0.001, 1, 4, perm=perm)
    assert np.array_equal(ctx.p_map(), p_ref.astype(np.int8))
    assert np.array_equal(perm.cpu().numpy(), adapt.bucket_order(p_ref))
    m2 = m.with_p(p_ref.astype(np.int8))
    fr2 = oracle_fr(m2, ph)
    q2 = adapt.transfer(fr, qt, fr2).numpy()
    got = ctx.unpack(buf[:ctx.n_dof]).cpu().numpy()
    assert np.abs(got - q2).max() <= 1e-13 * np.abs(q2).max()


def test_diff_full_vjp_and_dot_product(built):
    """Differentiation workload (24^3, p = 4): FP64 VJP against the oracle's
    reverse-mode derivative (1e-12); the FP32 VJP and JVP against those FP64
    products in relative 2-norm (1e-5); and the FP32 adjoint identity
    <w, Jv> = <J^T w, v>.  Its discrepancy is <w, d_Jv> - <d_JTw, v> with d
    the FP32 rounding of each product, measured here against FP64: for w
    independent of d_Jv (and v of d_JTw) each inner product is about
    |w| |d_Jv| / sqrt(N), so the bound is 10 (|w| |d_Jv| + |v| |d_JTw|) / sqrt(N)
    (a factor 10 of safety over that estimate) plus the FP64 part."""
    from oracle import linearize as L
    m, q, ph = cases.workload_diff()
    qg = generic_state(q)
    fr = oracle_fr(m, ph)
    w = cases.uniform(905, q.size) - 0.5
    ref = L.vjp(fr, torch.from_numpy(qg), torch.from_numpy(w)).numpy()
    ctx = gpu_ctx(m, ph, 4, 4)
    qs = ctx.pack(torch.from_numpy(qg).cuda())
    got = ctx.unpack(ctx.vjp(qs, ctx.pack(torch.from_numpy(w).cuda()))).cpu().numpy()
    ok, rel, fs = parity_ok(got, ref, m, qg, 1e-12)
    assert ok, (rel, fs)
    q32 = ctx.pack(torch.from_numpy(qg).cuda(), torch.float32)
    v32 = ctx.pack(torch.from_numpy(cases.uniform(906, q.size) - 0.5).cuda(), torch.float32)
    w32 = ctx.pack(torch.from_numpy(cases.uniform(907, q.size) - 0.5).cuda(), torch.float32)
    v64, w64 = v32.double(), w32.double()
    Jv, JTw = ctx.jvp(q32, v32).double(), ctx.vjp(q32, w32).double()
    Jv64, JTw64 = ctx.jvp(qs, v64), ctx.vjp(qs, w64)
    dJv, dJTw = float((Jv - Jv64).norm()), float((JTw - JTw64).norm())
    assert dJTw <= 1e-5 * float(JTw64.norm()), dJTw / float(JTw64.norm())
    assert dJv <= 1e-5 * float(Jv64.norm()), dJv / float(Jv64.norm())
    lhs = float(torch.dot(w64, Jv))
    rhs = float(torch.dot(JTw, v64))
    n = q.size
    bound = 10.0 * (float(w64.norm()) * dJv + float(v64.norm()) * dJTw) / math.sqrt(n)
    bound += 1e-13 * float(w64.norm() * Jv64.norm() + v64.norm() * JTw64.norm())
    assert abs(lhs - rhs) <= bound, (lhs, rhs, bound)


def test_vortex_batch_full_residual(built):
    m, q, ph = cases.workload_vortex_batch()  # 32 instances, n in 8..64, p in 1..5
    fr = oracle_fr(m, ph)
    Rref = fr.residual(torch.from_numpy(q)).numpy()
    ctx = gpu_ctx(m, ph)
    R = ctx.unpack(ctx.residual(ctx.pack(torch.from_numpy(q).cuda()))).cpu().numpy()
    ok, rel, fs = parity_ok(R, Rref, m, q, 1e-12)
    assert ok, (rel, fs)
