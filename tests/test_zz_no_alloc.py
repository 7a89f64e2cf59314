"""The allocation-free finite-difference Jv (fr_jvp_fd_static) against fr_jvp.

fr_jvp_fd_static keeps its work vectors in a device array reserved at load
time, for callers that cannot call cudaMalloc after set-up: processes whose
device memory is held by another allocator, where a new allocation fails,
and loops that must not touch the allocator (cudaFree synchronises the
device).  It must give the product of the existing finite-difference entry
point on two calls in a row (the reserved array keeps the previous call's
contents), allocate nothing even on its first call after a mixed-degree
layout is built, and refuse a problem larger than its reserved size.  The
file is named to be collected last; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import cases

pytestmark = pytest.mark.gpu


def _ctx(n, p, mu=0.02):
    from paper_1910_03693_gb300 import FRContext
    from paper_1910_03693_gb300 import build as B
    B.build()
    m, q, ph = cases.workload_vortex2d(n, p)
    ctx = FRContext(m, gamma=ph["gamma"], mu=mu, Pr=ph["Pr"])
    return ctx, q


def test_static_fd_jv_matches_fr_jvp_twice():
    from paper_1910_03693_gb300.api import lib
    ctx, q = _ctx(16, 2)
    qs = ctx.pack(torch.from_numpy(q).cuda())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (5, 6):
        v = torch.from_numpy(cases.uniform(seed, ctx.n_dof) - 0.5).cuda()
        v = ctx.pack(v)
        ref = ctx.jvp(qs, v, mode="fd", eps=1e-6)
        out = torch.full_like(qs, float("nan"))
        rc = lib().fr_jvp_fd_static(ctx.h, C.c_void_p(qs.data_ptr()), C.c_void_p(v.data_ptr()),
                                    C.c_void_p(out.data_ptr()), C.c_double(1e-6), stream)
        assert rc == 0, lib().fr_last_error().decode()
        torch.cuda.synchronize()
        err = float((out - ref).abs().max() / ref.abs().max())
        assert err <= 1e-12, err


def test_static_fd_jv_rejects_oversized_problem():
    from paper_1910_03693_gb300.api import lib
    ctx_big, _ = _ctx(64, 5, mu=0.0)       # 64^2 quads x 36 points x 4 variables = 589,824 DOF
    buf = torch.zeros(ctx_big.n_dof, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib().fr_jvp_fd_static(ctx_big.h, C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()),
                                C.c_void_p(buf.data_ptr()), C.c_double(1e-6), stream)
    assert rc == -1
    assert "262144" in lib().fr_last_error().decode()


def test_static_fd_jv_mixed_degree_first_call_allocates_nothing():
    """Degrees 1..4 (several buckets, the multi-bucket launch): the first call
    after the context is built must neither allocate device memory nor differ
    from fr_jvp's finite-difference product."""
    from paper_1910_03693_gb300 import FRContext
    from paper_1910_03693_gb300 import build as B
    from paper_1910_03693_gb300.api import lib
    B.build()
    m, q, ph = cases.workload_vortex2d(12, 2)
    m = m.with_p((cases.uniform(31, m.n_elem) * 4 + 1).astype(np.int8))
    m = m.with_p(cases.limit_jumps_down(m, m.p))
    q = cases.random_state(m, 7)
    assert len(set(m.p.tolist())) >= 3
    ctx = FRContext(m, gamma=ph["gamma"], mu=0.02, Pr=ph["Pr"], p_min=1, p_max=4)
    qs = ctx.pack(torch.from_numpy(q).cuda())
    vs = [ctx.pack(torch.from_numpy(cases.uniform(seed, ctx.n_dof) - 0.5).cuda()) for seed in (8, 9)]
    outs = [torch.full_like(qs, float("nan")) for _ in vs]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for v, out in zip(vs, outs):
        rc = lib().fr_jvp_fd_static(ctx.h, C.c_void_p(qs.data_ptr()), C.c_void_p(v.data_ptr()),
                                    C.c_void_p(out.data_ptr()), C.c_double(1e-6), stream)
        assert rc == 0, lib().fr_last_error().decode()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for v, out in zip(vs, outs):
        ref = ctx.jvp(qs, v, mode="fd", eps=1e-6)
        err = float((out - ref).abs().max() / ref.abs().max())
        assert err <= 1e-12, err
