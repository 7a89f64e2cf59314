"""Full ESDIRK time steps through the C ABI (esdirk_step), against the oracle's
time step, and with the p-adaptation after the step (the paper adapts after
every time step)."""
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


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("mode,jv_dtype", [("fd", torch.float64), ("exact", torch.float32)])
def test_esdirk_step_matches_oracle(built, order, mode, jv_dtype):
    """One ESDIRK2 / ESDIRK3 step (dt 0.05) of the 2D vortex, every implicit
    stage to ||F|| <= 1e-8 ||F0||: q^{n+1} agrees with the oracle's step (FD Jv,
    the paper's product) to 1e-6 of the change over the step."""
    from oracle import esdirk
    from oracle import linearize as L
    from paper_1910_03693_gb300 import esdirk_tableau
    m, q, ph = cases.workload_vortex2d(8, 2)
    fr, ctx = oracle_fr(m, ph), gpu_ctx(m, ph)
    tab = esdirk.esdirk2() if order == 2 else esdirk.esdirk3()
    A, b = esdirk_tableau(order)
    assert np.allclose(np.array(A), np.array(tab.A), rtol=0, atol=1e-15)
    assert np.allclose(np.array(b), np.array(tab.b), rtol=0, atol=1e-15)
    qn = torch.from_numpy(q)
    opts = esdirk.NewtonOpts(tol=1e-8, dtau_init=0.05, dtau_max=10.0)
    jv = lambda qq, v, Rq: L.fd_jv(fr, qq, v, 1e-6, Rq)
    qo, so = esdirk.esdirk_step(fr.residual, jv, qn, tab, 0.05, opts)
    qs = ctx.pack(qn.cuda())
    st = ctx.esdirk_step(A, 0.05, qs, b=b, tol=1e-8, dtau_init=0.05, dtau_max=10.0, mode=mode, jv_dtype=jv_dtype)
    assert len(st) == len(A) - 1
    assert all(s["converged"] and s["norm_final"] <= 1e-8 * s["norm0"] for s in st), st
    qg = ctx.unpack(qs).cpu().numpy()
    dq = np.abs(qo.numpy() - q).max()
    assert np.abs(qg - qo.numpy()).max() <= 1e-6 * dq, (np.abs(qg - qo.numpy()).max(), dq)


def test_esdirk_step_with_adaptation(built):
    """A step of the mixed-degree 2D vortex with adaptation: the degrees and
    the state after the step are those of a step without adaptation followed
    by the indicator and the rebucketing, and the p-map is the oracle's
    decision on the oracle's own step result."""
    from oracle import adapt as OA
    from oracle import esdirk
    from oracle import linearize as L
    from paper_1910_03693_gb300 import esdirk_tableau
    m, q, ph = cases.workload_vortex2d(8, 2)
    m = m.with_p((1 + np.floor(cases.uniform(308, m.n_elem) * 3)).astype(np.int8))
    q = cases.vortex_state(m)
    A, b = esdirk_tableau(3)
    ad = dict(nu_max=0.1, nu_min=0.001, p_min=1, p_max=3, var=1)
    res = []
    for with_adapt in (True, False):
        ctx = gpu_ctx(m, ph, 1, 3)
        buf = torch.zeros(ctx.n_dof_capacity, dtype=torch.float64, device="cuda")
        ctx.pack(torch.from_numpy(q).cuda(), out=buf[:ctx.n_dof])
        st = ctx.esdirk_step(A, 0.05, buf, b=b, adapt=ad if with_adapt else None, tol=1e-8, dtau_init=0.05,
                             dtau_max=10.0, mode="exact", jv_dtype=torch.float32)
        assert all(s["converged"] for s in st)
        if not with_adapt:
            eta, emax = ctx.indicator(buf[:ctx.n_dof], var=1)
            ctx.rebucket(eta, emax, buf, 0.1, 0.001, 1, 3)
        res.append((ctx.p_map(), ctx.unpack(buf[:ctx.n_dof]).cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    # the oracle's step and decision
    fr = oracle_fr(m, ph)
    tab = esdirk.esdirk3()
    jv = lambda qq, v, Rq: L.jvp(fr, qq, v)
    qo, _ = esdirk.esdirk_step(fr.residual, jv, torch.from_numpy(q), tab, 0.05,
                               esdirk.NewtonOpts(tol=1e-8, dtau_init=0.05, dtau_max=10.0))
    p_ref, _ = OA.adapt_p(fr, qo, 0.1, 0.001, 1, 3)
    assert np.array_equal(res[0][0], p_ref.astype(np.int8))
