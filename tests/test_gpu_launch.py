"""GPU launch configurations: the multi-bucket persistent launch against one
launch per degree bucket, tuned elements-per-CTA tables, the autotuner, and
the CUDA-graph Arnoldi product against direct launches.  None of these may
change a result beyond rounding order; most are bit-identical because every
solution point runs the same arithmetic whatever CTA it lands in."""
import numpy as np
import pytest
import torch

import cases
from helpers import generic_state, gpu_ctx, oracle_fr, parity_ok, small_workloads

pytestmark = pytest.mark.gpu

MIXED = ["vortex2d_mixed_p1-4", "ns2d_mixed_p1-4", "box_curved_mixed_p1-3", "cylinder_4x12x2_mixed",
         "naca_24x4x2_mixed", "vortex_batch_5"]


@pytest.fixture(scope="module")
def built():
    from paper_1910_03693_gb300 import build as B
    B.build()
    return True


@pytest.fixture(scope="module")
def works():
    return small_workloads()


def _ops(ctx, q, v):
    """FP64 and FP32 residual and JVP at q along v (state layout)."""
    out = []
    for dt in (torch.float64, torch.float32):
        qs, vs = ctx.pack(q, dt), ctx.pack(v, dt)
        out += [ctx.residual(qs), ctx.jvp(qs, vs)]
    return out


def _close(a, b):
    scale = max(float(b.abs().max()), 1e-300)
    return float((a - b).abs().max()) <= (1e-13 if a.dtype == torch.float64 else 1e-6) * scale


def _epb_table(nd, value):
    """Every degree, kernel and precision set to `value` elements per CTA
    (halved until the elements fit 256 threads)."""
    tab = [0] * 42
    for prec in range(2):
        for kind in range(3):
            for P in range(2, 7):
                nsp = P ** nd
                e = value
                while e > 1 and e * nsp > 256:
                    e //= 2
                tab[(prec * 3 + kind) * 7 + P] = e
    return tab


@pytest.mark.parametrize("name", MIXED)
def test_multi_bucket_launch_matches_per_bucket(built, works, name):
    m, q, ph = works[name]
    qg = generic_state(q)
    v = cases.uniform(301, q.size) - 0.5
    ctx = gpu_ctx(m, ph)
    qd, vd = torch.from_numpy(qg).cuda(), torch.from_numpy(v).cuda()
    ctx.set_tuning({"multi_launch": True})
    assert ctx.tuning()["multi_launch"]
    a = _ops(ctx, qd, vd)
    ctx.set_tuning({"multi_launch": False})
    assert not ctx.tuning()["multi_launch"]
    b = _ops(ctx, qd, vd)
    for x, y in zip(a, b):
        assert _close(x, y), float((x - y).abs().max())


@pytest.mark.parametrize("name", ["vortex2d_mixed_p1-4", "box_curved_mixed_p1-3", "vortex_batch_5"])
@pytest.mark.parametrize("epb", [1, 2, 3, 64])
def test_elements_per_cta_table(built, works, name, epb):
    """Any admissible elements-per-CTA choice, including 3 (tiles that end
    mid-bucket) and one CTA per element, gives the default launch's result."""
    m, q, ph = works[name]
    qg = generic_state(q)
    v = cases.uniform(302, q.size) - 0.5
    ctx = gpu_ctx(m, ph)
    qd, vd = torch.from_numpy(qg).cuda(), torch.from_numpy(v).cuda()
    ref = _ops(ctx, qd, vd)
    for multi in (True, False):
        ctx.set_tuning({"epb": _epb_table(m.nd, epb), "multi_launch": multi})
        got = _ops(ctx, qd, vd)
        for x, y in zip(got, ref):
            assert _close(x, y), (multi, float((x - y).abs().max()))


def test_tuning_rejects_bad_entries(built, works):
    from paper_1910_03693_gb300 import FRError
    m, q, ph = works["vortex2d_16x16_p2"]
    ctx = gpu_ctx(m, ph)
    with pytest.raises(FRError):
        ctx.set_tuning({"epb": [-1] + [0] * 41})
    with pytest.raises(FRError):
        ctx.set_tuning({"epb": [0] * 20 + [257] + [0] * 21})
    # the exact JVP's choice (slot [precision][2][P = 1]) lies in [0, 4]; the
    # weight model (slot [0][0][P = 1]) in [0, 3]
    for prec in (0, 1):
        bad = [0] * 42
        bad[prec * 21 + 2 * 7 + 1] = 5
        with pytest.raises(FRError):
            ctx.set_tuning({"epb": bad})
        ok = [0] * 42
        ok[prec * 21 + 2 * 7 + 1] = 4
        ctx.set_tuning({"epb": ok})
    bad = [0] * 42
    bad[1] = 4
    with pytest.raises(FRError):
        ctx.set_tuning({"epb": bad})


@pytest.mark.parametrize("name", ["cylinder_4x12x2_mixed", "vortex_batch_5", "tgv_5^3_p3"])
def test_autotune_keeps_parity(built, works, name):
    """After the autotuner picked its launch table the residual and the JVP
    still match the oracle (FP64 1e-12 / 1e-11 curved, FP32 2e-5)."""
    from oracle import linearize as L
    m, q, ph = works[name]
    qg = generic_state(q)
    v = cases.uniform(303, q.size) - 0.5
    fr = oracle_fr(m, ph)
    Rref = fr.residual(torch.from_numpy(qg)).numpy()
    Jref = L.jvp(fr, torch.from_numpy(qg), torch.from_numpy(v)).numpy()
    ctx = gpu_ctx(m, ph)
    qd, vd = torch.from_numpy(qg).cuda(), torch.from_numpy(v).cuda()
    t = ctx.autotune(ctx.pack(qd))
    nd = m.nd
    for prec in range(2):
        for kind in range(3):
            for P in range(2, 7):
                e = t["epb"][(prec * 3 + kind) * 7 + P]
                assert e == 0 or e * P ** nd <= 256
    tol64 = 1e-11 if name.startswith("cylinder") else 1e-12
    for dt, tol in ((torch.float64, tol64), (torch.float32, 2e-5)):
        qs, vs = ctx.pack(qd, dt), ctx.pack(vd, dt)
        R = ctx.unpack(ctx.residual(qs)).cpu().numpy()
        ok, rel, fs = parity_ok(R, Rref, m, qg, tol)
        assert ok, ("residual", str(dt), rel, fs)
        J = ctx.unpack(ctx.jvp(qs, vs)).cpu().numpy()
        ok, rel, fs = parity_ok(J, Jref, m, qg, tol if dt == torch.float32 else 1e-11)
        assert ok, ("jvp", str(dt), rel, fs)


@pytest.mark.parametrize("jv_dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("name", ["vortex2d_mixed_p1-4", "tgv_5^3_p3"])
def test_graph_arnoldi_matches_direct(built, works, name, jv_dtype):
    """Host-driven GMRES (one round trip per iteration; the device-driven cycle
    always launches directly) with the Arnoldi product replayed from a CUDA
    graph and with direct launches: same iterations, same solution bit for
    bit, across three solves
    (timing off, then on twice: turning it on recaptures the graph with event
    nodes, the third solve replays it).  The timed JVP volume launches count
    every product, replayed ones included: the same number as with direct
    launches, at least one per Arnoldi iteration (restarts add a product for
    the true residual)."""
    m, q, ph = works[name]
    ctx = gpu_ctx(m, ph)
    qs = ctx.pack(torch.from_numpy(generic_state(q)).cuda())
    b = ctx.pack(torch.from_numpy(cases.uniform(304, q.size) - 0.5).cuda())
    sigma = 1.0 / (0.4358665215 * 0.01)
    res, counts = {}, {}
    for graphs in (False, True):
        ctx.set_tuning({"graphs": graphs, "device_gmres": False})
        runs = []
        for timing in (False, True, True):
            ctx.timing(timing)
            x, st = ctx.gmres(qs, b, sigma, mode="exact", jv_dtype=jv_dtype, rtol=1e-6, m=12, max_it=60)
            if timing:
                rep, launches = ctx.timing_report()
                n_vol = sum(v[0] for k, v in rep.items() if k.startswith(("vol_jvp", "fused_jvp")))
                n_buckets = len(set(int(p) for p in ctx.p_map()))
                per = 1 if (n_buckets == 1 or ctx.tuning()["multi_launch"]) else n_buckets
                assert n_vol >= per * st["iterations"], (n_vol, st["iterations"], graphs)
                assert counts.setdefault(graphs, n_vol) == n_vol
                assert launches > 0
            ctx.timing(False)
            runs.append((x.clone(), st))
        for x, st in runs[1:]:
            assert torch.equal(x, runs[0][0]) and st["iterations"] == runs[0][1]["iterations"]
        res[graphs] = runs[0]
    assert counts[True] == counts[False]
    assert res[True][1]["iterations"] == res[False][1]["iterations"]
    assert torch.equal(res[True][0], res[False][0])


@pytest.mark.parametrize("name", ["cylinder_4x12x2_mixed", "tgv_5^3_p3"])
def test_operators_capture_into_cuda_graph(built, works, name):
    """Residual, exact and finite-difference JVP and VJP launch only
    stream-ordered work once their workspaces exist: captured into a CUDA graph
    (on the capture stream torch hands them) and replayed, they reproduce the
    direct calls bit for bit, with the multi-bucket launch on mixed degrees."""
    m, q, ph = works[name]
    ctx = gpu_ctx(m, ph)
    q64 = ctx.pack(torch.from_numpy(generic_state(q)).cuda())
    v64 = ctx.pack(torch.from_numpy(cases.uniform(305, q.size) - 0.5).cuda())
    q32, v32 = q64.float(), v64.float()
    calls = [
        lambda o: ctx.residual(q64, out=o[0]), lambda o: ctx.residual(q32, out=o[1]),
        lambda o: ctx.jvp(q64, v64, out=o[0]), lambda o: ctx.jvp(q32, v32, out=o[1]),
        lambda o: ctx.jvp(q64, v64, out=o[0], mode="fd"),
        lambda o: ctx.vjp(q64, v64, out=o[0]), lambda o: ctx.vjp(q32, v32, out=o[1]),
    ]
    for fn in calls:
        direct = (torch.empty_like(q64), torch.empty_like(q32))
        fn(direct)
        torch.cuda.synchronize()
        got = (torch.full_like(q64, float("nan")), torch.full_like(q32, float("nan")))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            fn(got)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        i = 0 if not torch.isnan(got[0]).all() else 1
        assert torch.equal(got[i], direct[i])


@pytest.mark.parametrize("name", ["tgv_5^3_p3", "diff_3^3_p4_mu0.05", "box_curved_mixed_p1-3"])
def test_diagonal_metric_kernels_match_general(built, works, name):
    """Axis-aligned boxes run trace and volume kernels that skip the zero
    metric terms; they agree with the general kernels to rounding (FP64 1e-13,
    FP32 1e-6 of max|R|).  On a curved mesh the switch changes nothing."""
    m, q, ph = works[name]
    qg = generic_state(q)
    v = cases.uniform(306, q.size) - 0.5
    ctx = gpu_ctx(m, ph)
    qd, vd = torch.from_numpy(qg).cuda(), torch.from_numpy(v).cuda()
    ctx.set_tuning({"diag_metrics": True})
    a = _ops(ctx, qd, vd)
    ctx.set_tuning({"diag_metrics": False})
    b = _ops(ctx, qd, vd)
    for x, y in zip(a, b):
        if name.startswith("box_curved"):
            assert torch.equal(x, y)
        else:
            assert _close(x, y), float((x - y).abs().max())


@pytest.mark.parametrize("name", ["cylinder_4x12x2_mixed", "vortex_batch_5"])
def test_work_weight_models_do_not_change_results(built, works, name):
    """The element weight that orders the multi-bucket work table (n_sp (p+1),
    n_sp, n_sp^2, n_sp^3) only changes which CTA takes which tile: residual and
    JVP are bit-identical."""
    m, q, ph = works[name]
    qg = generic_state(q)
    v = cases.uniform(309, q.size) - 0.5
    ctx = gpu_ctx(m, ph)
    qd, vd = torch.from_numpy(qg).cuda(), torch.from_numpy(v).cuda()
    ref = None
    for model in range(4):
        tab = [0] * 42
        tab[1] = model
        ctx.set_tuning({"epb": tab, "multi_launch": True})
        got = _ops(ctx, qd, vd)
        if ref is None:
            ref = got
        for x, y in zip(got, ref):
            assert torch.equal(x, y)
    with pytest.raises(Exception):
        bad = [0] * 42
        bad[1] = 4
        ctx.set_tuning({"epb": bad})


def test_timing_select(built, works):
    """With a selection only the named kernels carry event pairs (device time
    above zero); every launch is still counted, with the same counts, bytes
    and launch total as with every kernel timed."""
    m, q, ph = works["tgv_5^3_p3"]
    ctx = gpu_ctx(m, ph)
    q64 = ctx.pack(torch.from_numpy(generic_state(q)).cuda())
    q32, v32 = q64.float(), ctx.pack(torch.from_numpy(cases.uniform(306, q.size) - 0.5).cuda()).float()
    out = {}
    for sel in (None, ["vol_jvp_f32"]):
        ctx.timing_select(sel)
        ctx.timing(True)
        ctx.residual(q64)
        for _ in range(2):
            ctx.jvp(q32, v32)
        rep, n = ctx.timing_report()
        ctx.timing(False)
        out[sel is None] = ({k: (v[0], v[2]) for k, v in rep.items()}, n)
        if sel:
            assert rep["vol_jvp_f32"][0] == 2 and rep["vol_jvp_f32"][1] > 0
            assert all(v[1] == 0.0 for k, v in rep.items() if k != "vol_jvp_f32"), rep
        else:
            assert all(v[1] > 0.0 for v in rep.values()), rep
    ctx.timing_select(None)
    assert out[True] == out[False]
