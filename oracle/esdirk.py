"""ESDIRK time integration with pseudo-transient continuation, FP64, test only.

Sec. 2.3 of the paper:
* Eq. ESDIRK_ns: q^1 = q^n; q^i = dt w R(q^i) + q^n + dt sum_{j<i} a_ij R(q^j);
  q^{n+1} = q^n + dt sum_i b_i R(q^i).
* Eq. ESDIRK_conservative: F(q) = -q/(w dt) + R(q) + (q^n + dt sum_{j<i} a_ij R(q^j))/(w dt).
* Eq. linearized_pseudo_transient_final: (1/(w dt) + 1/dtau - dR/dq) dq = F(q^m),
  q^{m+1} = q^m + dq.
* Eq. ser: dtau^{m+1} = min(dtau^m ||F^{m-1}|| / ||F^m||, dtau_max).
* GMRES tolerance 1e-1 within 100 iterations, else halve dtau and redo.

Readings: the initial guess of stage i is q^{i-1}; norms are Euclidean over
all DOFs; convergence is relative to ||F|| at the stage's first iterate.

Tableaus (coefficients are not printed in the paper; derived here from the
order conditions, see ``esdirk2`` and ``esdirk3``).
"""
import math
from dataclasses import dataclass

import torch

from .krylov import gmres


@dataclass
class Tableau:
    name: str
    A: list
    b: list
    c: list
    order: int

    @property
    def s(self):
        return len(self.b)


def esdirk2() -> Tableau:
    """Three-stage, stiffly accurate, L-stable, order 2: diagonal g = 1 - sqrt(2)/2,
    c = (0, 2g, 1); b from sum b = 1, sum b c = 1/2 with b3 = g."""
    g = 1.0 - math.sqrt(2.0) / 2.0
    b2 = (0.5 - g) / (2.0 * g)
    b1 = 1.0 - g - b2
    A = [[0.0, 0.0, 0.0], [g, g, 0.0], [b1, b2, g]]
    return Tableau("ESDIRK2", A, [b1, b2, g], [0.0, 2 * g, 1.0], 2)


def esdirk3_gamma() -> float:
    """Root near 0.4359 of 6 g^3 - 18 g^2 + 9 g - 1 = 0 (by Newton)."""
    g = 0.44
    for _ in range(100):
        f = 6 * g ** 3 - 18 * g ** 2 + 9 * g - 1
        df = 18 * g ** 2 - 36 * g + 9
        g -= f / df
    return g


def esdirk3(c3: float = 0.6) -> Tableau:
    """Four-stage, stiffly accurate, order 3, explicit first stage.

    Diagonal g solves 6g^3 - 18g^2 + 9g - 1 = 0 (stability function vanishes at
    infinity); c2 = 2g, c4 = 1, c3 chosen (0.6).  b (= last row) solves
    sum b = 1, sum b c = 1/2, sum b c^2 = 1/3 with b4 = g; a32 from
    sum_i b_i sum_j a_ij c_j = 1/6; a31 = c3 - g - a32.
    """
    g = esdirk3_gamma()
    c2 = 2 * g
    # b2 c2 + b3 c3 = 1/2 - g ; b2 c2^2 + b3 c3^2 = 1/3 - g
    r1, r2 = 0.5 - g, 1.0 / 3.0 - g
    det = c2 * c3 ** 2 - c3 * c2 ** 2
    b2 = (r1 * c3 ** 2 - c3 * r2) / det
    b3 = (c2 * r2 - r1 * c2 ** 2) / det
    b1 = 1.0 - g - b2 - b3
    a32 = (1.0 / 6.0 - 0.5 * g - 2 * g * g * b2 - g * c3 * b3) / (2 * g * b3)
    a31 = c3 - g - a32
    A = [[0.0] * 4, [g, g, 0.0, 0.0], [a31, a32, g, 0.0], [b1, b2, b3, g]]
    return Tableau("ESDIRK3", A, [b1, b2, b3, g], [0.0, c2, c3, 1.0], 3)


def order_condition_residuals(t: Tableau):
    A, b, c = t.A, t.b, t.c
    s = t.s
    Ac = [sum(A[i][j] * c[j] for j in range(s)) for i in range(s)]
    res = {
        "sum b = 1": sum(b) - 1.0,
        "sum b c = 1/2": sum(b[i] * c[i] for i in range(s)) - 0.5,
        "row sums = c": max(abs(sum(A[i]) - c[i]) for i in range(s)),
    }
    if t.order >= 3:
        res["sum b c^2 = 1/3"] = sum(b[i] * c[i] ** 2 for i in range(s)) - 1.0 / 3.0
        res["sum b A c = 1/6"] = sum(b[i] * Ac[i] for i in range(s)) - 1.0 / 6.0
    return res


def stability_function(t: Tableau, z: complex) -> complex:
    """R(z) = 1 + z b^T (I - z A)^{-1} 1."""
    s = t.s
    M = torch.eye(s, dtype=torch.complex128) - z * torch.tensor(t.A, dtype=torch.complex128)
    y = torch.linalg.solve(M, torch.ones(s, dtype=torch.complex128))
    return complex(1.0 + z * (torch.tensor(t.b, dtype=torch.complex128) @ y))


@dataclass
class NewtonOpts:
    tol: float = 1e-8
    dtau_init: float = 0.05
    dtau_max: float = 10.0
    gmres_m: int = 30
    gmres_rtol: float = 1e-1
    gmres_max_it: int = 100
    max_newton: int = 200
    max_halvings: int = 20


def solve_stage(R_fn, jv_fn, qn, Rs, i, tab: Tableau, dt, q0, opts: NewtonOpts):
    """Solve stage i (0-based, i >= 1) by pseudo-transient continuation.

    ``Rs[j]`` holds R(q^j) for j < i; ``jv_fn(q, v, Rq)`` approximates dR(q) v.
    Returns (q^i, R(q^i), stats)."""
    w = tab.A[i][i]
    inv_wdt = 1.0 / (w * dt)
    acc = qn.clone()
    for j in range(i):
        if tab.A[i][j] != 0.0:
            acc = acc + dt * tab.A[i][j] * Rs[j]
    rhs = acc * inv_wdt

    def F(q):
        Rq = R_fn(q)
        return -q * inv_wdt + Rq + rhs, Rq

    q = q0.clone()
    Fq, Rq = F(q)
    norm0 = float(torch.linalg.vector_norm(Fq))
    dtau = opts.dtau_init
    norm_prev = None
    st = dict(newton=0, gmres=0, halvings=0, norms=[norm0], converged=False)
    for m in range(opts.max_newton):
        norm = float(torch.linalg.vector_norm(Fq))
        if norm <= opts.tol * norm0:
            st["converged"] = True
            break
        if norm_prev is not None:
            dtau = min(dtau * norm_prev / norm, opts.dtau_max)
        for _ in range(opts.max_halvings + 1):
            sigma = inv_wdt + 1.0 / dtau
            dq, gs = gmres(lambda v: sigma * v - jv_fn(q, v, Rq), Fq, opts.gmres_m,
                           opts.gmres_rtol, opts.gmres_max_it)
            st["gmres"] += gs["iterations"]
            if gs["converged"]:
                break
            dtau *= 0.5
            st["halvings"] += 1
        q = q + dq
        norm_prev = norm
        Fq, Rq = F(q)
        st["newton"] += 1
        st["norms"].append(float(torch.linalg.vector_norm(Fq)))
    else:
        st["converged"] = float(torch.linalg.vector_norm(Fq)) <= opts.tol * norm0
    st["final_norm"] = float(torch.linalg.vector_norm(Fq))
    return q, Rq, st


def esdirk_step(R_fn, jv_fn, qn, tab: Tableau, dt, opts: NewtonOpts):
    """One physical time step; returns (q^{n+1}, per-stage stats)."""
    Rs = [R_fn(qn)]
    qs = [qn]
    stats = []
    for i in range(1, tab.s):
        qi, Ri, st = solve_stage(R_fn, jv_fn, qn, Rs, i, tab, dt, qs[-1], opts)
        qs.append(qi)
        Rs.append(Ri)
        stats.append(st)
    qnew = qn.clone()
    for i in range(tab.s):
        qnew = qnew + dt * tab.b[i] * Rs[i]
    return qnew, stats
