"""Invalid arguments are refused on the host with a status code (FRError in
Python) before anything is launched, and the context stays usable."""
import numpy as np
import pytest
import torch

import cases
from helpers import gpu_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_1910_03693_gb300 import build as B
    B.build()
    return True


@pytest.fixture()
def setup(built):
    m, q, ph = cases.workload_vortex2d(4, 2)
    ctx = gpu_ctx(m, ph, 1, 3)
    qs = ctx.pack(torch.from_numpy(q).cuda())
    return ctx, qs, m


def _still_works(ctx, qs):
    R = ctx.residual(qs)
    torch.cuda.synchronize()
    assert torch.isfinite(R).all()


def test_gmres_rejects_bad_options(setup):
    from paper_1910_03693_gb300 import FRError
    ctx, qs, _ = setup
    b = torch.ones_like(qs)
    for kw in (dict(m=0), dict(m=64), dict(rtol=0.0), dict(rtol=-1.0), dict(max_it=0), dict(reorth=3),
               dict(mode="fd", eps=0.0), dict(precond=True)):
        with pytest.raises(FRError):
            ctx.gmres(qs, b, 10.0, **kw)
    _still_works(ctx, qs)


def test_stage_and_step_reject_bad_arguments(setup):
    from paper_1910_03693_gb300 import FRError, esdirk_tableau
    ctx, qs, _ = setup
    A, b = esdirk_tableau(3)
    R1 = ctx.residual(qs)
    qi = qs.clone()
    R2 = torch.empty_like(qs)
    with pytest.raises(FRError):   # stage 1 is the explicit one
        ctx.esdirk_stage(A, 1, 0.01, qs, [R1, R2, None, None], qi)
    with pytest.raises(FRError):   # dt <= 0
        ctx.esdirk_stage(A, 2, 0.0, qs, [R1, R2, None, None], qi)
    with pytest.raises(FRError):   # R(q^1) missing
        ctx.esdirk_stage(A, 2, 0.01, qs, [None, R2, None, None], qi)
    bad = [row[:] for row in A]
    bad[0][0] = 0.3                # first stage not explicit
    with pytest.raises(FRError):
        ctx.esdirk_step(bad, 0.01, qs.clone(), b=b)
    with pytest.raises(FRError):
        ctx.esdirk_step(A, 0.01, torch.zeros(ctx.n_dof_capacity, dtype=torch.float64, device="cuda"), b=b,
                        adapt=dict(p_min=1, p_max=3, var=9))
    with pytest.raises(ValueError):  # the low-precision residual is double-float or FP32
        ctx.esdirk_stage(A, 2, 0.01, qs, [R1, R2, None, None], qi, low_above=1e-6, low_precision="bf16")
    _still_works(ctx, qs)


def test_adaptation_filter_and_preconditioner_reject_bad_arguments(setup):
    from paper_1910_03693_gb300 import FRError
    ctx, qs, m = setup
    eta, emax = ctx.indicator(qs)
    buf = torch.zeros(ctx.n_dof_capacity, dtype=torch.float64, device="cuda")
    buf[:ctx.n_dof] = qs
    with pytest.raises(FRError):   # degrees outside the context's limits
        ctx.rebucket(eta, emax, buf, p_min=0, p_max=3)
    with pytest.raises(FRError):
        ctx.rebucket(eta, emax, buf, p_min=1, p_max=5)
    with pytest.raises(FRError):
        ctx.filter(qs.clone(), alpha=1.5)
    with pytest.raises(FRError):   # nothing built yet
        ctx.precond_apply(qs)
    with pytest.raises(FRError):
        ctx.precond_build(qs, -1.0)
    with pytest.raises(TypeError):
        ctx.residual(qs.to(torch.float16))
    _still_works(ctx, qs)
    assert np.array_equal(ctx.p_map(), m.p.astype(np.int8))
