"""The BF16-operator trial: FP32 kernels whose operator matrices (Lagrange
interpolation and differentiation, correction derivatives, mortar tables) are
rounded to bfloat16.  Checked against the FP64 oracle with the error stated
per result; the FP32 path on the same input is the reference point."""
import numpy as np
import pytest
import torch

import cases
from helpers import flux_scale, generic_state, gpu_ctx, oracle_fr, small_workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_1910_03693_gb300 import build as B
    B.build()
    return True


@pytest.fixture(scope="module")
def works():
    return small_workloads()


def _fs_err(got, ref, m, q):
    return float(np.abs(got - ref).max()) / flux_scale(m, q)


@pytest.mark.parametrize("name,bound", [("vortex2d_mixed_p1-4", 2e-2), ("tgv_5^3_p3", 2e-2),
                                        ("cylinder_4x12x2_mixed", None)])
def test_bf16_operators_residual_and_jvp(built, works, name, bound):
    """Rounding the operators to 8 significant bits costs accuracy: the
    flux-scaled error grows well beyond the FP32 path's.  On affine meshes it
    stays at the bfloat16 level (below 2e-2 of the flux scale); on the curved
    3D mixed-degree cylinder (two rounded mortar factors per face, rounded
    interpolation weights that no longer sum to one) it does not, and the
    trial is only reported there (finite, worse than FP32)."""
    from oracle import linearize as L
    m, q, ph = works[name]
    qg = generic_state(q)
    v = cases.uniform(307, q.size) - 0.5
    fr = oracle_fr(m, ph)
    Rref = fr.residual(torch.from_numpy(qg)).numpy()
    Jref = L.jvp(fr, torch.from_numpy(qg), torch.from_numpy(v)).numpy()
    ctx = gpu_ctx(m, ph)
    q32 = ctx.pack(torch.from_numpy(qg).cuda(), torch.float32)
    v32 = ctx.pack(torch.from_numpy(v).cuda(), torch.float32)
    out = {}
    for bf in (False, True):
        R = ctx.unpack(ctx.residual(q32, bf16_operators=bf)).cpu().numpy()
        J = ctx.unpack(ctx.jvp(q32, v32, bf16_operators=bf)).cpu().numpy()
        out[bf] = (_fs_err(R, Rref, m, qg), _fs_err(J, Jref, m, qg))
    (r32, j32), (r16, j16) = out[False], out[True]
    assert r16 > 4 * r32 and j16 > 4 * j32, out
    assert np.isfinite(r16) and np.isfinite(j16), out
    if bound is not None:
        assert r16 < bound and j16 < bound, out


def test_bf16_operators_stage_converges(built):
    """ESDIRK3 stage 2 on the 2D vortex with the bfloat16-operator JVP inside
    GMRES (FP64 F): the stage still reaches ||F|| <= 1e-8 ||F0||."""
    from paper_1910_03693_gb300 import esdirk_tableau
    m, q, ph = cases.workload_vortex2d(8, 2)
    ctx = gpu_ctx(m, ph)
    A, _ = esdirk_tableau(3)
    qn = ctx.pack(torch.from_numpy(q).cuda())
    R1 = ctx.residual(qn)
    res = {}
    for jv in (torch.float32, "bf16op"):
        qi = qn.clone()
        R2 = torch.empty_like(qn)
        st = ctx.esdirk_stage(A, 2, 0.05, qn, [R1, R2, None, None], qi, tol=1e-8, dtau_init=0.05,
                              dtau_max=10.0, mode="exact", jv_dtype=jv)
        assert st["converged"] and st["norm_final"] <= 1e-8 * st["norm0"], (jv, st)
        res[str(jv)] = (qi.clone(), st)
    dq = (res["bf16op"][0] - res["torch.float32"][0]).abs().max().item()
    assert dq <= 1e-6 * (qn.abs().max().item()), dq
