"""GPU parity with Roe's common flux (FR_FLUX_ROE) against the oracle's Roe
(the paper's R |Lambda| R^-1 formula with a dense solve; the kernels use the
closed-form wave strengths): residual in FP64, FP32 and double-float, exact
JVP in FP64 and FP32, VJP in FP64, on every small workload (mortars, walls,
far field, curved and batched meshes).  Tolerances are those of the Rusanov
tests (FP64 1e-12 of max|R| or of the flux scale, 1e-11 curved; FP32 2e-5;
double-float 2e-10, 2e-9 curved)."""
import numpy as np
import pytest
import torch

from helpers import generic_state, gpu_ctx, oracle_fr, parity_ok, small_workloads

pytestmark = pytest.mark.gpu

WL = small_workloads()
CURVED = ("cylinder", "naca", "box_curved")


def tol64(name):
    return 1e-11 if name.startswith(CURVED) else 1e-12


def tol_df(name):
    return 2e-9 if name.startswith(CURVED) else 2e-10


@pytest.fixture(scope="module")
def built():
    from paper_1910_03693_gb300 import build as B
    B.build()
    return True


def _pair(name):
    m, q, ph = WL[name]
    ph = dict(ph, flux="roe")
    return m, q, ph, oracle_fr(m, ph), gpu_ctx(m, ph)


@pytest.mark.parametrize("name", list(WL))
def test_roe_residual_parity(built, name):
    m, q, ph, fr, ctx = _pair(name)
    Rref = fr.residual(torch.from_numpy(q)).numpy()
    qd = torch.from_numpy(q).cuda()
    for dtype, tol in ((torch.float64, tol64(name)), (torch.float32, 2e-5)):
        R = ctx.unpack(ctx.residual(ctx.pack(qd, dtype))).cpu().numpy()
        ok, rel, fs = parity_ok(R, Rref, m, q, tol)
        assert ok, (name, str(dtype), rel, fs)
    R = ctx.unpack(ctx.residual(ctx.pack(qd), double_float=True)).cpu().numpy()
    ok, rel, fs = parity_ok(R, Rref, m, q, tol_df(name))
    assert ok, (name, "double-float", rel, fs)


@pytest.mark.parametrize("name", list(WL))
def test_roe_exact_jvp_parity(built, name):
    from cases import uniform
    from oracle import linearize as L
    m, q, ph, fr, ctx = _pair(name)
    q = generic_state(q)
    qt = torch.from_numpy(q)
    v = (uniform(911, q.size) - 0.5) * np.abs(q).mean()
    Jref = L.jvp(fr, qt, torch.from_numpy(v)).numpy()
    for dtype, tol in ((torch.float64, tol64(name)), (torch.float32, 2e-5)):
        J = ctx.unpack(ctx.jvp(ctx.pack(qt.cuda(), dtype), ctx.pack(torch.from_numpy(v).cuda(), dtype))).cpu().numpy()
        ok, rel, fs = parity_ok(J, Jref, m, q, tol)
        assert ok, (name, str(dtype), rel, fs)


@pytest.mark.parametrize("name", ["vortex2d_mixed_p1-4", "ns2d_mixed_p1-4", "tgv_5^3_p3", "cylinder_4x12x2_mixed"])
def test_roe_vjp_parity(built, name):
    from cases import uniform
    from oracle import linearize as L
    m, q, ph, fr, ctx = _pair(name)
    q = generic_state(q)
    qt = torch.from_numpy(q)
    w = uniform(912, q.size) - 0.5
    Gref = L.vjp(fr, qt, torch.from_numpy(w)).numpy()
    G = ctx.unpack(ctx.vjp(ctx.pack(qt.cuda()), ctx.pack(torch.from_numpy(w).cuda()))).cpu().numpy()
    ok, rel, fs = parity_ok(G, Gref, m, q, tol64(name) * 10)
    assert ok, (name, rel, fs)


def test_roe_free_stream_on_gpu(built):
    import cases
    m = cases.naca_cgrid(24, 4, 2, n_wake=6, p=2)
    m.nbr = m.nbr.copy()
    m.nbr[m.nbr == cases.WALL] = cases.FARFIELD
    qinf = cases.free_stream_q(3, vel=(0.3, 0.2, 0.1), mach=0.3)
    ctx = gpu_ctx(m, dict(gamma=1.4, mu=1e-2, Pr=0.7, q_inf=qinf, flux="roe"))
    q = torch.from_numpy(cases.freestream_state(m, vel=(0.3, 0.2, 0.1), mach=0.3)).cuda()
    R = ctx.residual(ctx.pack(q))
    assert float(R.abs().max()) < 1e-12 * (1 / (1.4 * 0.09)) / 0.002


def test_roe_and_rusanov_differ_and_unknown_flux_is_refused(built):
    m, q, ph = WL["vortex2d_16x16_p2"]
    qd = torch.from_numpy(q).cuda()
    a = gpu_ctx(m, dict(ph, flux="roe"))
    b = gpu_ctx(m, ph)
    Ra, Rb = a.residual(a.pack(qd)), b.residual(b.pack(qd))
    assert float((Ra - Rb).abs().max()) > 1e-6 * float(Rb.abs().max())
    from paper_1910_03693_gb300 import FRContext
    with pytest.raises(ValueError):
        FRContext(m, gamma=1.4, flux="hllc")


def test_roe_esdirk_stage_matches_oracle(built):
    """ESDIRK3 stage 2 on the 2D vortex with Roe's flux, exact FP32 JVP GMRES and
    double-float F above the tolerance, against the oracle's stage solve with
    the FD product: the converged stage values agree to the tolerance."""
    from oracle import esdirk
    from oracle import linearize as L
    m, q, ph = WL["vortex2d_16x16_p2"]
    ph = dict(ph, flux="roe")
    fr, ctx = oracle_fr(m, ph), gpu_ctx(m, ph)
    tab = esdirk.esdirk3()
    qn = torch.from_numpy(q)
    Rn = fr.residual(qn)
    opts = esdirk.NewtonOpts(tol=1e-8, dtau_init=0.05, dtau_max=10.0)
    jv = lambda qq, v, Rq: L.fd_jv(fr, qq, v, 1e-6, Rq)
    qo, Ro, so = esdirk.solve_stage(fr.residual, jv, qn, [Rn], 1, tab, 0.05, qn, opts)
    qns = ctx.pack(qn.cuda())
    R1 = ctx.residual(qns)
    qi = qns.clone()
    R2 = torch.empty_like(qns)
    st = ctx.esdirk_stage(tab.A, 2, 0.05, qns, [R1, R2, None, None], qi, tol=1e-8, dtau_init=0.05,
                          dtau_max=10.0, mode="exact", jv_dtype=torch.float32, low_above=1e-8, low_precision="df")
    assert st["converged"] and st["norm_final"] <= 1e-8 * st["norm0"]
    qg = ctx.unpack(qi).cpu().numpy()
    dq = np.abs(qo.numpy() - q).max()
    assert np.abs(qg - qo.numpy()).max() <= 1e-6 * dq
