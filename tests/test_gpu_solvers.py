"""GPU parity of the VJP, GMRES and the ESDIRK stage against the FP64 oracle."""
import numpy as np
import pytest
import torch

import cases
from helpers import generic_state, gpu_ctx, oracle_fr, parity_ok, small_workloads

pytestmark = pytest.mark.gpu

WL = small_workloads()


@pytest.fixture(scope="module")
def built():
    from paper_1910_03693_gb300 import build as B
    B.build()
    return True


@pytest.mark.parametrize("name", list(WL))
def test_vjp_parity(built, name):
    """J^T w against the oracle's reverse-mode derivative (FP64 1e-12, FP32 2e-5)."""
    from oracle import linearize as L
    m, q, ph = WL[name]
    q = generic_state(q)
    fr, ctx = oracle_fr(m, ph), gpu_ctx(m, ph)
    w = cases.uniform(903, q.size) - 0.5
    ref = L.vjp(fr, torch.from_numpy(q), torch.from_numpy(w)).numpy()
    tol64 = 1e-11 if name.startswith(("cylinder", "naca", "box_curved")) else 1e-12
    for dtype, tol in ((torch.float64, tol64), (torch.float32, 2e-5)):
        qs = ctx.pack(torch.from_numpy(q).cuda(), dtype)
        ws = ctx.pack(torch.from_numpy(w).cuda(), dtype)
        got = ctx.unpack(ctx.vjp(qs, ws)).cpu().numpy()
        ok, rel, fs = parity_ok(got, ref, m, q, tol)
        assert ok, (name, str(dtype), rel, fs)


def test_vjp_dot_product_and_autograd(built):
    """<w, J v> = <J^T w, v> on the GPU in FP64, to 1e-13 of |w| |Jv| + |v| |J^T w|
    (each side's rounding scales with those norms), and torch.autograd through
    the residual."""
    from paper_1910_03693_gb300 import autograd_residual
    m, q, ph = WL["diff_3^3_p4_mu0.05"]
    ctx = gpu_ctx(m, ph)
    qs = ctx.pack(torch.from_numpy(q).cuda())
    v = ctx.pack(torch.from_numpy(cases.uniform(908, q.size) - 0.5).cuda())
    w = ctx.pack(torch.from_numpy(cases.uniform(909, q.size) - 0.5).cuda())
    Jv, JTw = ctx.jvp(qs, v), ctx.vjp(qs, w)
    lhs = float(torch.dot(w, Jv))
    rhs = float(torch.dot(JTw, v))
    assert abs(lhs - rhs) <= 1e-13 * float(w.norm() * Jv.norm() + v.norm() * JTw.norm()), (lhs, rhs)
    qg = qs.clone().requires_grad_(True)
    R = autograd_residual(ctx, qg)
    (g,) = torch.autograd.grad(R, qg, w)
    assert torch.allclose(g, ctx.vjp(qs, w), rtol=0, atol=0)


def _small_system():
    m, q, ph = cases.workload_vortex2d(3, 2)
    return m, cases.random_state(m, 2), ph


@pytest.mark.parametrize("reorth", [1, 2])
def test_gmres_matches_dense_solve(built, reorth):
    from oracle import linearize as L
    m, q, ph = _small_system()
    fr, ctx = oracle_fr(m, ph), gpu_ctx(m, ph)
    qt = torch.from_numpy(q)
    J = L.dense_jacobian(fr, qt)
    sigma = 20.0
    A = sigma * torch.eye(J.shape[0]) - J
    b = torch.from_numpy(cases.uniform(4, J.shape[0]) - 0.5)
    xref = torch.linalg.solve(A, b).numpy()
    qs = ctx.pack(qt.cuda())
    bs = ctx.pack(b.cuda())
    x, st = ctx.gmres(qs, bs, sigma, mode="exact", rtol=1e-13, m=30, max_it=3000, reorth=reorth)
    assert st["converged"] and st["restarts"] >= 1
    xg = ctx.unpack(x).cpu().numpy()
    assert np.abs(xg - xref).max() <= 1e-10 * np.abs(xref).max()


@pytest.mark.parametrize("reorth", [0, 1, 2])
def test_gmres_iterates_match_oracle(built, reorth):
    """At the paper's tolerance (1e-1) the GPU (classical Gram-Schmidt once, with
    the DGKS second pass, or twice) and the oracle (modified Gram-Schmidt) build
    the same Krylov space: same iteration count, same x."""
    from oracle import krylov
    from oracle import linearize as L
    m, q, ph = cases.workload_vortex2d(6, 2)
    fr, ctx = oracle_fr(m, ph), gpu_ctx(m, ph)
    qt = torch.from_numpy(q)
    b = torch.from_numpy(cases.uniform(5, q.size) - 0.5)
    sigma = 1.0 / (0.4358665215 * 0.05) + 1.0 / 0.05
    xo, so = krylov.gmres(lambda v: sigma * v - L.jvp(fr, qt, v), b, m=30, rtol=1e-1, max_it=100)
    qs = ctx.pack(qt.cuda())
    x, st = ctx.gmres(qs, ctx.pack(b.cuda()), sigma, mode="exact", rtol=1e-1, m=30, max_it=100, reorth=reorth)
    assert st["iterations"] == so["iterations"]
    xg = ctx.unpack(x).cpu().numpy()
    assert np.abs(xg - xo.numpy()).max() <= 1e-9 * np.abs(xo.numpy()).max()


@pytest.mark.parametrize("mode,jv_dtype,low_above,low_precision",
                         [("fd", torch.float64, 0.0, "df"), ("exact", torch.float64, 0.0, "df"),
                          ("exact", torch.float32, 0.0, "df"), ("exact", torch.float32, 1e-3, "f32"),
                          ("exact", torch.float32, 1e-7, "df")])
def test_esdirk3_stage_matches_oracle(built, mode, jv_dtype, low_above, low_precision):
    """Stage 2 of ESDIRK3 on the 2D vortex to ||F|| <= 1e-8 ||F0|| (the oracle
    with the paper's FD Jv); the converged stage values agree to the tolerance.
    With low_above the early Newton iterations use the FP32 or double-float
    residual and the later ones, including the final check, the FP64 residual."""
    from oracle import esdirk
    from oracle import linearize as L
    m, q, ph = cases.workload_vortex2d(8, 2)
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
                          dtau_max=10.0, mode=mode, jv_dtype=jv_dtype, low_above=low_above,
                          low_precision=low_precision)
    assert st["converged"] and st["norm_final"] <= 1e-8 * st["norm0"]
    assert st["f64_evaluations"] >= 1
    assert (st["low_evaluations"] > 0) == (low_above > 0)
    qg = ctx.unpack(qi).cpu().numpy()
    dq = np.abs(qo.numpy() - q).max()
    assert np.abs(qg - qo.numpy()).max() <= 1e-6 * dq
    assert abs(st["newton"] - so["newton"]) <= 2
    assert torch.allclose(R2, ctx.residual(qi), rtol=0, atol=0)


@pytest.mark.parametrize("jv", [torch.float64, torch.float32])
def test_double_float_arnoldi_matches_fp64(built, jv):
    """The Arnoldi dot products in double-float arithmetic (FP64 values split
    into FP32 pairs, error-free products and sums on the FP32 pipe, about
    1e-14 of |u| |w|) against FP64 FMAs (the default): the same iteration count
    and the same solution to 1e-9 (FP64 products) or 1e-5 (FP32 products)."""
    m, q, ph = WL["diff_3^3_p4_mu0.05"]
    ctx = gpu_ctx(m, ph)
    qs = ctx.pack(torch.from_numpy(generic_state(q)).cuda())
    b = ctx.pack(torch.from_numpy(cases.uniform(915, q.size) - 0.5).cuda())
    out = {}
    for df in (True, False):
        t = ctx.tuning()
        t["df_arnoldi"] = df
        ctx.set_tuning(t)
        x, st = ctx.gmres(qs, b, 40.0, mode="exact", jv_dtype=jv, m=30, rtol=1e-8, max_it=300)
        assert st["converged"], (df, st)
        out[df] = (x.cpu().numpy(), st["iterations"])
    assert abs(out[True][1] - out[False][1]) <= 1, (out[True][1], out[False][1])
    tol = 1e-9 if jv == torch.float64 else 1e-5
    x0 = out[False][0]
    assert np.abs(out[True][0] - x0).max() <= tol * np.abs(x0).max()


def test_arnoldi_slot_walks_agree(built):
    """The Arnoldi dots and updates with each warp reading runs of 4 x 512 bytes
    of every column (the default) and with single 512-byte segments one grid
    apart: the same iteration count and the same solution to 1e-12 (only the
    order of the partial sums differs)."""
    m, q, ph = WL["tgv_5^3_p3"]
    ctx = gpu_ctx(m, ph)
    qs = ctx.pack(torch.from_numpy(generic_state(q)).cuda())
    b = ctx.pack(torch.from_numpy(cases.uniform(916, q.size) - 0.5).cuda())
    out = {}
    for runs in (True, False):
        t = ctx.tuning()
        t["arnoldi_runs"] = runs
        ctx.set_tuning(t)
        x, st = ctx.gmres(qs, b, 60.0, mode="exact", jv_dtype=torch.float64, m=20, rtol=1e-10, max_it=200,
                          reorth=1)
        assert st["converged"], (runs, st)
        out[runs] = (x.cpu().numpy(), st["iterations"])
    assert out[True][1] == out[False][1]
    assert np.abs(out[True][0] - out[False][0]).max() <= 1e-12 * np.abs(out[False][0]).max()


def _set_flag(ctx, key, value):
    t = ctx.tuning()
    t[key] = value
    ctx.set_tuning(t)


@pytest.mark.parametrize("name,jv,reorth,pc", [
    ("tgv_5^3_p3", torch.float64, 0, False),
    ("tgv_5^3_p3", torch.float32, 2, False),
    ("diff_3^3_p4_mu0.05", torch.float32, 0, False),
    ("cylinder_4x12x2_mixed", torch.float64, 0, True),
    ("box_mixed_p4-5_ns", torch.float32, 0, True)])
def test_device_gmres_matches_host_driven(built, name, jv, reorth, pc):
    """GMRES with the Givens rotations and the convergence test on the device
    (iterations launched in batches, the default) against one host round trip
    per iteration: the products and Gram-Schmidt passes are the same kernels,
    so the iteration and restart counts agree and x agrees to rounding, with
    restarts (m = 8), one or two passes, and the element-Jacobi
    preconditioner (its column scale then read on the device; the blocks are
    rebuilt after the tuning change, which drops them).  Tolerances the
    products can meet: 1e-9 with FP64 products, 1e-5 with FP32 ones (below
    1e-4 the basis stays FP64); FP32 products after a restart start from a
    true residual that carries their rounding, so the final residual
    estimates agree to 1e-2 there and to 1e-6 with FP64 products."""
    m, q, ph = WL[name]
    ctx = gpu_ctx(m, ph)
    qs = ctx.pack(torch.from_numpy(generic_state(q)).cuda())
    b = ctx.pack(torch.from_numpy(cases.uniform(917, q.size) - 0.5).cuda())
    sigma = 40.0 if name.startswith("tgv") else 500.0
    rtol = 1e-9 if jv == torch.float64 else 1e-5
    out = {}
    for dev in (False, True):
        _set_flag(ctx, "device_gmres", dev)
        if pc:
            ctx.precond_build(qs, sigma)
        x, st = ctx.gmres(qs, b, sigma, mode="exact", jv_dtype=jv, m=8, rtol=rtol, max_it=400, reorth=reorth,
                          precond=pc)
        assert st["converged"], (dev, st)
        out[dev] = (x.cpu().numpy(), st)
    assert out[True][1]["iterations"] == out[False][1]["iterations"]
    assert out[True][1]["restarts"] == out[False][1]["restarts"]
    rtol_res = 1e-6 if jv == torch.float64 else 1e-2
    assert abs(out[True][1]["rel_res"] - out[False][1]["rel_res"]) <= rtol_res * out[False][1]["rel_res"] + 1e-13
    x0 = out[False][0]
    tol = 1e-10 if jv == torch.float64 else 1e-5
    assert np.abs(out[True][0] - x0).max() <= tol * np.abs(x0).max()


def test_device_gmres_batch_past_convergence(built):
    """A first batch longer than the cycle needs (the previous cycle ran 30
    iterations): the launches past convergence return at entry, leave x as
    the host-driven loop computes it, and their timing records are dropped,
    so the per-kernel launch counts equal the iterations that ran."""
    m, q, ph = WL["tgv_5^3_p3"]
    ctx = gpu_ctx(m, ph)
    qs = ctx.pack(torch.from_numpy(generic_state(q)).cuda())
    b = ctx.pack(torch.from_numpy(cases.uniform(918, q.size) - 0.5).cuda())
    kw = dict(mode="exact", jv_dtype=torch.float32, m=30)
    _, st_long = ctx.gmres(qs, b, 40.0, rtol=1e-14, max_it=30, **kw)
    assert st_long["iterations"] == 30
    ctx.timing(True)
    x, st = ctx.gmres(qs, b, 40.0, rtol=1e-1, max_it=100, **kw)
    rep, _ = ctx.timing_report()
    ctx.timing(False)
    its = st["iterations"]
    assert st["converged"] and 1 <= its < 29, st
    products = sum(rep.get(k, (0,))[0] for k in ("vol_jvp_f32", "fused_jvp_f32"))
    assert products == its, (products, its)
    # + the norm of b before the cycle, + the final combination x += V y
    assert rep["arnoldi_dot"][0] == its + 1 and rep["arnoldi_update"][0] == its + 1
    _set_flag(ctx, "device_gmres", False)
    xh, sth = ctx.gmres(qs, b, 40.0, rtol=1e-1, max_it=100, **kw)
    assert sth["iterations"] == its
    xh = xh.cpu().numpy()
    assert np.abs(x.cpu().numpy() - xh).max() <= 1e-6 * np.abs(xh).max()


@pytest.mark.parametrize("name,m,rtol,pc", [("tgv_5^3_p3", 30, 1e-1, False), ("tgv_5^3_p3", 8, 1e-4, False),
                                            ("diff_3^3_p4_mu0.05", 30, 1e-2, False),
                                            ("vortex2d_mixed_p1-4", 8, 1e-4, False),
                                            ("box_mixed_p4-5_ns", 30, 1e-1, False),
                                            ("box_mixed_p4-5_ns", 8, 1e-4, True),
                                            ("cylinder_4x12x2_mixed", 30, 1e-2, True)])
def test_f32_basis_matches_f64_basis(built, name, m, rtol, pc):
    """GMRES with FP32 products and the Krylov basis stored in FP32 (dots and
    norms summed in FP32 over 16 values, FP64 beyond; the default for such
    products at rtol >= 1e-4) against the FP64 basis, both device-driven and
    host-driven: the same Krylov space to about 1e-6, so the iteration counts
    agree within one and x to 1e-4 of max|x|, with and without restarts, on
    one and on several degree buckets, on a vector whose length is not a
    multiple of four (the 3^3 p = 4 box: 16,875 values), and with the
    element-Jacobi preconditioner applied to the FP32 vectors."""
    mm, q, ph = WL[name]
    ctx = gpu_ctx(mm, ph)
    qs = ctx.pack(torch.from_numpy(generic_state(q)).cuda())
    b = ctx.pack(torch.from_numpy(cases.uniform(919, q.size) - 0.5).cuda())
    out = {}
    sigma = 500.0 if pc else 40.0
    for dev in (True, False):
        for b32 in (True, False):
            _set_flag(ctx, "device_gmres", dev)
            _set_flag(ctx, "f32_basis", b32)
            if pc:
                ctx.precond_build(qs, sigma)   # the tuning change dropped the blocks
            x, st = ctx.gmres(qs, b, sigma, mode="exact", jv_dtype=torch.float32, m=m, rtol=rtol, max_it=400,
                              precond=pc)
            assert st["converged"], (dev, b32, st)
            out[dev, b32] = (x.cpu().numpy(), st["iterations"])
    x0, i0 = out[False, False]
    for key, (x, its) in out.items():
        assert abs(its - i0) <= 1, (key, its, i0)
        assert np.abs(x - x0).max() <= 1e-4 * np.abs(x0).max(), key
