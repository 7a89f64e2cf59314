"""The fused exact JVP (compact traces + one face-and-volume kernel per element
tile), used when every face of the mesh is interior and conforming.

Checked against the three-pass JVP of the same library (FP64, the same
arithmetic up to its order: 1e-13), against the oracle's JVP (FP64 1e-12, or
1e-11 on curved elements; FP32 2e-5), for conservation of the linearised
operator (both sides of a face receive exactly opposite fluxes), in GMRES
(the prepared product replayed from a CUDA graph), and on meshes whose
elements are rotated so that faces meet with non-trivial orientation codes.
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


def rotate_elements(m, q, elems):
    """Rotate the reference frame of the given elements by 90 degrees about the
    zeta axis (new xi = old eta, new eta = -old xi), keeping the physical mesh and
    state: node and solution-point order, faces, neighbour faces and orientation
    codes are rewritten.  The elements must not be face neighbours of one
    another, start with orientation code 0 on every face, and have geometry
    order 1."""
    assert m.geom_order == 1
    nd, nv = m.nd, m.nd + 2
    P = None
    nodes = m.nodes.copy()
    nbr, nbr_face, orient = m.nbr.copy(), m.nbr_face.copy(), m.orient.copy()
    off = m.offsets()
    q = np.asarray(q).copy()
    old_of_new = {0: 2, 1: 3, 2: 1, 3: 0, 4: 4, 5: 5}    # new face -> old face
    # face point order: new faces 0, 1 flip their first tangential axis; in 3D
    # faces 4, 5 swap the tangential axes and flip the (new) first one
    own_code = {0: 2, 1: 2, 2: 0, 3: 0, 4: 3, 5: 3}
    nbr_code = {0: 2, 1: 2, 2: 0, 3: 0, 4: 5, 5: 5}     # the inverse mapping, seen from the neighbour
    rot = set(int(e) for e in elems)
    for e in rot:
        assert np.all(m.orient[e] == 0)
        for f in range(2 * nd):
            assert int(m.nbr[e, f]) not in rot
        P = int(m.p[e]) + 1
        # nodes (2 per direction): new (i', j', k) = old (1 - j', i', k)
        nn = 2
        for a in range(nn ** nd):
            i, j = a % nn, (a // nn) % nn
            k = a // (nn * nn) if nd == 3 else 0
            src = (1 - j) + nn * i + nn * nn * k
            nodes[e, a] = m.nodes[e, src]
        # solution points: new (i', j', k) = old (P-1-j', i', k)
        blk = q[off[e]:off[e + 1]].reshape(-1, nv)
        new = blk.copy()
        for sp in range(P ** nd):
            i, j = sp % P, (sp // P) % P
            k = sp // (P * P) if nd == 3 else 0
            new[sp] = blk[(P - 1 - j) + P * i + P * P * k]
        q[off[e]:off[e + 1]] = new.reshape(-1)
        for fn in range(2 * nd):
            fo = old_of_new[fn]
            n, g = int(m.nbr[e, fo]), int(m.nbr_face[e, fo])
            nbr[e, fn], nbr_face[e, fn] = n, g
            orient[e, fn] = own_code[fn] if nd == 3 else (2 if fn < 2 else 0)
            nbr_face[n, g] = fn
            orient[n, g] = nbr_code[fn] if nd == 3 else (2 if fn < 2 else 0)
    out = cases.Mesh(nd, 1, nodes, nbr, nbr_face, orient, m.p.copy(), m.name + "_rot")
    cases.check_connectivity(out)
    return out, q


def _sheared_box(p, n=3, mu=0.02):
    m = cases.periodic_box(3, n, 0.0, 1.0, p)
    m.nodes = m.nodes.copy()
    m.nodes[..., 0] += 0.3 * m.nodes[..., 1] + 0.2 * m.nodes[..., 2]     # affine, not axis-aligned
    return m, cases.random_state(m, 41), dict(gamma=1.4, mu=mu, Pr=0.71)


def _curved_box(p):
    m = cases.periodic_box(3, 3, 0.0, 1.0, p)
    m.nodes = m.nodes + 0.02 * np.sin(5 * m.nodes[..., ::-1])
    return m, cases.random_state(m, 42), dict(gamma=1.4, mu=0.01, Pr=0.71)


def _workloads():
    out = {}
    m, q, ph = cases.workload_vortex2d(16, 2)
    out["vortex2d_16_p2_euler"] = (m, q, ph)
    out["vortex2d_16_p2_ns"] = (m, cases.random_state(m, 43), dict(ph, mu=0.02))
    m, q, ph = cases.workload_tgv(5, 3)
    out["tgv_5_p3"] = (m, q, ph)
    m, q, ph = cases.workload_diff(3, 4)
    out["diff_3_p4_mu0.05"] = (m, q, dict(ph, mu=0.05))
    out["diff_3_p4_roe"] = (m, q, dict(ph, mu=0.05, flux="roe"))
    out["sheared_box_p2"] = _sheared_box(2)
    out["curved_box_p2"] = _curved_box(2)
    out["box_p5_ns"] = _sheared_box(5, n=2)
    out["box_p1_ns"] = _sheared_box(1, n=4)
    mb, qb, ph = cases.workload_vortex_batch(5, 3, 9, 1, 5)
    out["vortex_batch_5"] = (mb, qb, ph)
    m, q, ph = cases.workload_vortex2d(6, 3)
    rot = [e for e in range(m.n_elem) if ((e % 6) + (e // 6)) % 2 == 0]
    mr, qr = rotate_elements(m, cases.random_state(m, 44), rot)
    out["vortex2d_rotated_ns"] = (mr, qr, dict(ph, mu=0.02))
    m, q, ph = _sheared_box(2, n=4)
    rot = [e for e in range(m.n_elem) if ((e % 4) + (e // 4) % 4 + e // 16) % 2 == 0]
    mr, qr = rotate_elements(m, q, rot)
    out["sheared_box_rotated"] = (mr, qr, ph)
    return out


WL = _workloads()


MODES = {"fused": 1, "classic": 2, "compact": 3}
KERNEL = {"fused": "fused_jvp", "classic": "face_jvp", "compact": "cface_jvp"}


def _choose(ctx, mode):
    """Force the exact JVP's kernels in both precisions: the fused
    face-and-volume kernel, the trace-gradient three passes or the compact
    three passes (the flag and the tuning slot [precision][volume JVP][P = 1])."""
    t = ctx.tuning()
    t["fused_jvp"] = True
    for prec in (0, 1):
        t["epb"][prec * 21 + 2 * 7 + 1] = MODES[mode]
    ctx.set_tuning(t)


def _jvp(ctx, q, v, dtype, mode):
    _choose(ctx, mode)
    ctx.timing(True)
    qs = ctx.pack(torch.from_numpy(q).cuda(), dtype)
    vs = ctx.pack(torch.from_numpy(v).cuda(), dtype)
    J = ctx.unpack(ctx.jvp(qs, vs)).cpu().numpy()
    rep, _ = ctx.timing_report()
    ctx.timing(False)
    return J, rep


@pytest.mark.parametrize("name", list(WL))
def test_fused_jvp_parity(built, name):
    """The fused and the compact three-pass JVPs against the trace-gradient
    three passes (FP64, 1e-13) and the oracle (FP64 1e-12 / 1e-11 curved;
    FP32 2e-5), with the kernels of each choice checked to have run."""
    from oracle import linearize as L
    m, q, ph = WL[name]
    q = generic_state(q)
    v = cases.uniform(911, q.size) - 0.5
    ctx = gpu_ctx(m, ph)
    J3, rep3 = _jvp(ctx, q, v, torch.float64, "classic")
    assert "fused_jvp_f64" not in rep3 and "cface_jvp_f64" not in rep3
    Jref = L.jvp(oracle_fr(m, ph), torch.from_numpy(q), torch.from_numpy(v)).numpy()
    tol = 1e-11 if name.startswith("curved") else 1e-12
    for mode in ("fused", "compact"):
        J, rep = _jvp(ctx, q, v, torch.float64, mode)
        assert rep.get(KERNEL[mode] + "_f64", (0,))[0] > 0, (mode, rep.keys())
        assert np.abs(J - J3).max() <= 1e-13 * np.abs(J3).max(), mode
        ok, rel, fs = parity_ok(J, Jref, m, q, tol)
        assert ok, (name, mode, rel, fs)
        J32, rep32 = _jvp(ctx, q, v, torch.float32, mode)
        assert rep32.get(KERNEL[mode] + "_f32", (0,))[0] > 0
        ok, rel, fs = parity_ok(J32, Jref, m, q, 2e-5)
        assert ok, (name, mode, "f32", rel, fs)


@pytest.mark.parametrize("mode", ["fused", "compact"])
@pytest.mark.parametrize("name", ["tgv_5_p3", "vortex2d_rotated_ns", "sheared_box_rotated", "diff_3_p4_roe"])
def test_fused_jvp_conserves(built, name, mode):
    """On a periodic mesh sum_sp w|J| (J v)_var = 0 to round-off for every
    variable: the two sides of every face receive exactly opposite fluxes."""
    m, q, ph = WL[name]
    q = generic_state(q)
    v = cases.uniform(912, q.size) - 0.5
    ctx = gpu_ctx(m, ph)
    J, _ = _jvp(ctx, q, v, torch.float64, mode)
    W = oracle_fr(m, ph).quadrature_weights().numpy()
    nv = m.nd + 2
    tot = (W * J).reshape(-1, nv).sum(0)
    scale = np.abs(W * J).reshape(-1, nv).sum(0)
    assert np.all(np.abs(tot) <= 1e-13 * scale), (tot, scale)


def test_mixed_degree_mesh_uses_three_passes(built):
    """Mortar faces make the mesh ineligible: the three-pass kernels run."""
    m, q, ph = cases.workload_vortex2d(8, 2)
    m = m.with_p((1 + np.floor(cases.uniform(71, m.n_elem) * 3)).astype(np.int8))
    m = m.with_p(cases.limit_jumps_down(m, m.p))
    q = cases.random_state(m, 45)
    ctx = gpu_ctx(m, ph)
    for mode in ("fused", "compact"):
        _, rep = _jvp(ctx, q, cases.uniform(913, q.size) - 0.5, torch.float64, mode)
        assert "fused_jvp_f64" not in rep and "cface_jvp_f64" not in rep
        assert rep.get("face_jvp_f64", (0,))[0] > 0


@pytest.mark.parametrize("jv", [torch.float32, torch.float64])
def test_fused_gmres_matches_three_pass(built, jv):
    """GMRES with the prepared fused and compact products (compact traces of q
    once, the product replayed from a CUDA graph) against GMRES with the
    trace-gradient three passes."""
    m, q, ph = WL["diff_3_p4_mu0.05"]
    q = generic_state(q)
    ctx = gpu_ctx(m, ph)
    q64 = ctx.pack(torch.from_numpy(q).cuda())
    b = ctx.pack(torch.from_numpy(cases.uniform(914, q.size) - 0.5).cuda())
    out = {}
    for mode in ("classic", "fused", "compact"):
        _choose(ctx, mode)
        x, st = ctx.gmres(q64, b, sigma=50.0, mode="exact", jv_dtype=jv, m=30, rtol=1e-6, max_it=200)
        assert st["converged"], (mode, st)
        out[mode] = (x.cpu().numpy(), st["iterations"])
    x0 = out["classic"][0]
    tol = 1e-9 if jv == torch.float64 else 1e-4
    for mode in ("fused", "compact"):
        assert abs(out[mode][1] - out["classic"][1]) <= (0 if jv == torch.float64 else 2), mode
        assert np.abs(out[mode][0] - x0).max() <= tol * np.abs(x0).max(), mode


def test_default_choice_and_autotune(built):
    """Undecided, the exact JVP on an eligible mesh runs the compact three
    passes; fr_autotune times the three choices and records one in the slot."""
    m, q, ph = WL["tgv_5_p3"]
    ctx = gpu_ctx(m, ph)
    ctx.timing(True)
    qs = ctx.pack(torch.from_numpy(q).cuda(), torch.float32)
    ctx.jvp(qs, qs)
    rep, _ = ctx.timing_report()
    ctx.timing(False)
    assert rep.get("cface_jvp_f32", (0,))[0] > 0 and rep.get("vol_jvp_f32", (0,))[0] > 0
    t = ctx.autotune(ctx.pack(torch.from_numpy(q).cuda()))
    assert t["epb"][21 + 2 * 7 + 1] in (1, 2, 3, 4) and t["epb"][2 * 7 + 1] in (1, 2, 3)


@pytest.mark.parametrize("name", ["tgv_5_p3", "box_p1_ns", "box_p5_ns", "sheared_box_rotated", "diff_3_p4_roe"])
def test_tma_staged_faces_match_thread_staged(built, name):
    """The compact face kernel with its tiles filled by bulk asynchronous copies
    (persistent, double-buffered; FP32 3D p = 1, 3, 5) against the same kernel
    with the threads' own loads: the same arithmetic on the same staged values,
    so the JVPs agree bit for bit; no bounded wait gave up (status word 0).
    Meshes whose blocks are not multiples of 16 bytes take the threads' loads
    either way."""
    m, q, ph = WL[name]
    q = generic_state(q)
    v = cases.uniform(917, q.size) - 0.5
    ctx = gpu_ctx(m, ph)
    out = {}
    for tma in (True, False):
        _choose(ctx, "compact")
        t = ctx.tuning()
        t["tma_faces"] = tma
        ctx.set_tuning(t)
        qs = ctx.pack(torch.from_numpy(q).cuda(), torch.float32)
        vs = ctx.pack(torch.from_numpy(v).cuda(), torch.float32)
        out[tma] = ctx.unpack(ctx.jvp(qs, vs)).cpu().numpy()
        assert ctx.device_status() == 0
    assert np.array_equal(out[True], out[False])


def _vt_cases():
    out = {"tgv_5_p3": WL["tgv_5_p3"], "box_p1_ns": WL["box_p1_ns"],
           "vortex2d_rotated_ns": WL["vortex2d_rotated_ns"]}
    m, q, ph = WL["tgv_5_p3"]
    out["tgv_5_p3_euler"] = (m, q, dict(ph, mu=0.0))
    m, q, ph = _sheared_box(3, n=4)
    rot = [e for e in range(m.n_elem) if ((e % 4) + (e // 4) % 4 + e // 16) % 2 == 0]
    mr, qr = rotate_elements(m, q, rot)
    out["box_p3_rotated"] = (mr, qr, ph)
    return out


VT = _vt_cases()


def _jvp_choice(ctx, qs, vs, choice):
    t = ctx.tuning()
    t["fused_jvp"] = True
    t["epb"][21 + 2 * 7 + 1] = choice
    ctx.set_tuning(t)
    ctx.timing(True)
    J = ctx.unpack(ctx.jvp(qs, vs)).cpu().numpy()
    rep, _ = ctx.timing_report()
    ctx.timing(False)
    return J, rep


@pytest.mark.parametrize("name", list(VT))
def test_face_kernel_tangent_traces_match_compact_passes(built, name):
    """The compact face kernel that forms the tangent's traces itself (FP32,
    tuning slot value 4; 3D p = 1 and 3, 2D p = 3) against the three compact
    passes: both form the traces with the same explicit fused multiply-adds,
    so the JVPs agree bit for bit.  The trace pass runs over q only, no
    bounded wait gave up, and the product meets the oracle at the FP32
    tolerance (Euler and Navier-Stokes; rotated elements give non-trivial
    orientation codes between the two sides' point numberings)."""
    from oracle import linearize as L
    m, q, ph = VT[name]
    q = generic_state(q)
    v = cases.uniform(918, q.size) - 0.5
    ctx = gpu_ctx(m, ph)
    qs = ctx.pack(torch.from_numpy(q).cuda(), torch.float32)
    vs = ctx.pack(torch.from_numpy(v).cuda(), torch.float32)
    J3, rep3 = _jvp_choice(ctx, qs, vs, 3)
    assert rep3.get("cface_jvp_f32", (0,))[0] > 0 and "cface_vt_jvp_f32" not in rep3
    J4, rep4 = _jvp_choice(ctx, qs, vs, 4)
    assert rep4.get("cface_vt_jvp_f32", (0,))[0] > 0 and "cface_jvp_f32" not in rep4, rep4.keys()
    assert rep4["ctrace_f32"][0] == rep3["ctrace_f32"][0] // 2
    assert ctx.device_status() == 0
    assert np.array_equal(J4, J3)
    Jref = L.jvp(oracle_fr(m, ph), torch.from_numpy(q), torch.from_numpy(v)).numpy()
    ok, rel, fs = parity_ok(J4, Jref, m, q, 2e-5)
    assert ok, (name, rel, fs)


@pytest.mark.parametrize("name", ["tgv_5_p3", "box_p5_ns", "diff_3_p4_mu0.05", "vortex_batch_5"])
def test_face_kernel_tangent_traces_fall_back(built, name):
    """Where the face kernel cannot form the tangent's traces (FP64, or a
    degree whose face points straddle warps or whose blocks are not
    multiples of 16 bytes), slot value 4 runs the three compact passes."""
    m, q, ph = WL[name]
    q = generic_state(q)
    v = cases.uniform(919, q.size) - 0.5
    ctx = gpu_ctx(m, ph)
    for dtype in ((torch.float64,) if name == "tgv_5_p3" else (torch.float64, torch.float32)):
        qs = ctx.pack(torch.from_numpy(q).cuda(), dtype)
        vs = ctx.pack(torch.from_numpy(v).cuda(), dtype)
        J3, _ = _jvp_choice(ctx, qs, vs, 3)
        J4, rep4 = _jvp_choice(ctx, qs, vs, 4)
        assert not any(k.startswith("cface_vt") for k in rep4), rep4.keys()
        assert np.array_equal(J4, J3)


@pytest.mark.parametrize("rtol", [1e-6, 1e-3])
def test_face_kernel_tangent_traces_in_gmres(built, rtol):
    """GMRES with FP32 products (the compact traces of q prepared once per
    solve, the Krylov column read in place; an FP64 basis at rtol 1e-6, the
    FP32 basis at 1e-3) takes the same iterates with either compact choice."""
    m, q, ph = VT["tgv_5_p3"]
    q = generic_state(q)
    ctx = gpu_ctx(m, ph)
    q64 = ctx.pack(torch.from_numpy(q).cuda())
    b = ctx.pack(torch.from_numpy(cases.uniform(920, q.size) - 0.5).cuda())
    out = {}
    for choice in (3, 4):
        t = ctx.tuning()
        t["fused_jvp"] = True
        t["epb"][21 + 2 * 7 + 1] = choice
        ctx.set_tuning(t)
        ctx.timing(True)
        x, st = ctx.gmres(q64, b, sigma=50.0, mode="exact", jv_dtype=torch.float32, m=30, rtol=rtol, max_it=200)
        rep, _ = ctx.timing_report()
        ctx.timing(False)
        assert st["converged"], (choice, st)
        assert ("cface_vt_jvp_f32" in rep) == (choice == 4), rep.keys()
        out[choice] = (x.cpu().numpy(), st["iterations"])
    assert ctx.device_status() == 0
    assert out[3][1] == out[4][1]
    assert np.array_equal(out[3][0], out[4][0])
