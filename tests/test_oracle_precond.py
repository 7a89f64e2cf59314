"""Pins of the oracle's element-Jacobi preconditioner (Sec. 2.3)."""
import numpy as np
import torch

import cases
from helpers import oracle_fr


_CACHE = {}


def _system():
    """3 x 3 vortex mesh with degrees 1 and 2 (224 DOF), its oracle and dense Jacobian."""
    if not _CACHE:
        from oracle import linearize as L
        m, q, ph = cases.workload_vortex2d(3, 1)
        m = m.with_p(np.array([1, 2, 1, 2, 1, 2, 1, 2, 1], dtype=np.int8))
        q = cases.random_state(m, 11)
        fr = oracle_fr(m, ph)
        _CACHE.update(m=m, q=q, ph=ph, fr=fr, J=L.dense_jacobian(fr, torch.from_numpy(q)))
    return _CACHE["m"], _CACHE["q"], _CACHE["ph"]


def test_blocks_are_the_self_coupling_of_each_element():
    """B_e u = (sigma u - J u) restricted to e for u supported on element e
    alone (checked with the JVP, not with the dense Jacobian's slices); the
    neighbours see u too, so the coupling left out of the blocks is real."""
    from oracle import linearize as L
    from oracle import precond as P
    m, q, ph = _system()
    fr = _CACHE["fr"]
    qt = torch.from_numpy(q)
    sigma = 7.0
    blocks = P.element_blocks(fr, qt, sigma, J=_CACHE["J"])
    assert len(blocks) == m.n_elem
    for e in (0, 4, 7):
        lo, hi, B = blocks[e]
        u = torch.zeros(q.size, dtype=torch.float64)
        u[lo:hi] = torch.from_numpy(cases.uniform(40 + e, hi - lo) - 0.5)
        Au = sigma * u - L.jvp(fr, qt, u)
        assert torch.allclose(B @ u[lo:hi], Au[lo:hi], rtol=0, atol=1e-12 * float(Au.abs().max()))
        outside = torch.cat([Au[:lo], Au[hi:]])
        assert float(outside.abs().max()) > 1e-3 * float(Au.abs().max())


def test_apply_inverse_inverts_each_block():
    from oracle import precond as P
    rng = np.random.default_rng(3)
    sizes = [4, 9, 16, 9]
    blocks, lo = [], 0
    for s in sizes:
        B = torch.from_numpy(rng.standard_normal((s, s)) + 5 * np.eye(s))
        blocks.append((lo, lo + s, B))
        lo += s
    w = torch.from_numpy(rng.standard_normal(lo))
    z = P.apply_inverse(blocks, w)
    for a, b_, B in blocks:
        assert torch.allclose(B @ z[a:b_], w[a:b_], rtol=0, atol=1e-12)


def test_left_preconditioned_gmres_is_exact_on_block_diagonal_operators():
    """With A the block-diagonal part of sigma I - J and M the same blocks,
    M^-1 A = I: left-preconditioned GMRES converges in one iteration to A^-1 b."""
    from oracle import krylov
    from oracle import precond as P
    m, q, ph = _system()
    blocks = P.element_blocks(_CACHE["fr"], torch.from_numpy(q), 5.0, J=_CACHE["J"])
    n = q.size

    def A(v):
        out = torch.empty_like(v)
        for lo, hi, B in blocks:
            out[lo:hi] = B @ v[lo:hi]
        return out

    b = torch.from_numpy(cases.uniform(12, n) - 0.5)
    x, st = krylov.gmres(lambda v: P.apply_inverse(blocks, A(v)), P.apply_inverse(blocks, b), m=10, rtol=1e-12,
                         max_it=10)
    assert st["iterations"] == 1 and st["converged"]
    assert torch.allclose(A(x), b, rtol=0, atol=1e-10)


def test_left_preconditioned_gmres_solves_the_full_system_in_fewer_iterations():
    from oracle import krylov
    from oracle import linearize as L
    from oracle import precond as P
    m, q, ph = _system()
    fr = _CACHE["fr"]
    qt = torch.from_numpy(q)
    sigma = 20.0
    J = _CACHE["J"]
    A = sigma * torch.eye(J.shape[0], dtype=J.dtype) - J
    b = torch.from_numpy(cases.uniform(13, q.size) - 0.5)
    xref = torch.linalg.solve(A, b)
    blocks = P.element_blocks(fr, qt, sigma, J=J)
    x0, s0 = krylov.gmres(lambda v: A @ v, b, m=60, rtol=1e-10, max_it=400)
    x1, s1 = krylov.gmres(lambda v: P.apply_inverse(blocks, A @ v), P.apply_inverse(blocks, b), m=60,
                          rtol=1e-10, max_it=400)
    assert s0["converged"] and s1["converged"]
    assert s1["iterations"] < s0["iterations"]
    assert float((x1 - xref).abs().max()) <= 1e-8 * float(xref.abs().max())


def test_blocks_of_selected_elements_equal_the_dense_slices():
    """The element-by-element construction (unit vectors of one element's DOFs)
    gives the dense Jacobian's diagonal blocks."""
    from oracle import precond as P
    m, q, ph = _system()
    qt = torch.from_numpy(q)
    full = P.element_blocks(_CACHE["fr"], qt, 3.0, J=_CACHE["J"])
    some = P.element_blocks(_CACHE["fr"], qt, 3.0, elements=[1, 6])
    for e in range(m.n_elem):
        if e in (1, 6):
            assert torch.allclose(some[e][2], full[e][2], rtol=0, atol=1e-12 * float(full[e][2].abs().max()))
        else:
            assert some[e][2] is None

