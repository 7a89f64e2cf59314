"""Shared helpers of the test-suite: small seeded workloads, oracle/GPU pairs."""
import math

import numpy as np
import torch

import cases

PHYS_KEYS = ("gamma", "mu", "Pr")


def small_workloads():
    """name -> (mesh, canonical state, physics dict); sized for the oracle in seconds,
    spanning several blocks of every kernel and a ragged tail."""
    out = {}
    m, q, ph = cases.workload_vortex2d(16, 2)
    out["vortex2d_16x16_p2"] = (m, q, ph)
    m2 = m.with_p((1 + np.floor(cases.uniform(71, m.n_elem) * 4)).astype(np.int8))
    out["vortex2d_mixed_p1-4"] = (m2, cases.random_state(m2, 72), dict(ph))
    ph_ns = dict(ph, mu=0.02, Pr=0.72)
    out["ns2d_mixed_p1-4"] = (m2, cases.random_state(m2, 73), ph_ns)
    m, q, ph = cases.workload_tgv(5, 3)
    out["tgv_5^3_p3"] = (m, q, ph)
    m, q, ph = cases.workload_diff(3, 4)
    ph = dict(ph, mu=0.05)
    out["diff_3^3_p4_mu0.05"] = (m, q, ph)
    mb = cases.periodic_box(3, 4, 0.0, 1.0, 2)
    mb.nodes = mb.nodes + 0.02 * np.sin(5 * mb.nodes[..., ::-1])
    mb = mb.with_p((1 + np.floor(cases.uniform(74, mb.n_elem) * 3)).astype(np.int8))
    out["box_curved_mixed_p1-3"] = (mb, cases.random_state(mb, 75), dict(gamma=1.4, mu=0.01, Pr=0.71))
    mc = cases.cylinder_ogrid(4, 12, 2, g=2, p=2)
    mc.p = cases.smooth_random_p_field(mc, 76, levels=(1, 2, 3, 4))
    qc = cases.freestream_state(mc, vel=(1.0, 0.0, 0.0), mach=0.2, noise=0.05, seed=77)
    out["cylinder_4x12x2_mixed"] = (mc, qc, dict(gamma=1.4, mu=1e-2, Pr=0.71,
                                                  q_inf=cases.free_stream_q(3, vel=(1.0, 0.0, 0.0), mach=0.2)))
    mn = cases.naca_cgrid(24, 4, 2, n_wake=6, p=1)
    mn.p = (1 + np.floor(cases.uniform(78, mn.n_elem) * 3)).astype(np.int8)
    a = math.radians(8.0)
    vel = (math.cos(a), math.sin(a), 0.0)
    qn = cases.freestream_state(mn, vel=vel, mach=0.2, noise=0.05, seed=79)
    out["naca_24x4x2_mixed"] = (mn, qn, dict(gamma=1.4, mu=1e-3, Pr=0.72,
                                              q_inf=cases.free_stream_q(3, vel=vel, mach=0.2)))
    mbat, qb, ph = cases.workload_vortex_batch(5, 3, 9, 1, 5)
    out["vortex_batch_5"] = (mbat, qb, ph)
    # the highest degree: 3D p = 5 (216 points an element, one element a CTA)
    # beside p = 4 through p-4/5 mortars, viscous; and 2D p = 5
    mh = cases.periodic_box(3, 3, 0.0, 1.0, 4)
    mh = mh.with_p((4 + np.floor(cases.uniform(80, mh.n_elem) * 2)).astype(np.int8))
    out["box_mixed_p4-5_ns"] = (mh, cases.random_state(mh, 81), dict(gamma=1.4, mu=0.02, Pr=0.71))
    m5, q5, ph5 = cases.workload_vortex2d(4, 5)
    out["vortex2d_4x4_p5"] = (m5, q5, ph5)
    return out


def oracle_fr(mesh, phys):
    from oracle.fr import FR
    from oracle.physics import Euler
    return FR(mesh, Euler(mesh.nd, phys["gamma"], phys.get("mu", 0.0), phys.get("Pr", 0.72),
                          phys.get("q_inf"), flux=phys.get("flux", "rusanov")))


def gpu_ctx(mesh, phys, p_min=None, p_max=None):
    from paper_1910_03693_gb300 import FRContext
    return FRContext(mesh, gamma=phys["gamma"], mu=phys.get("mu", 0.0), Pr=phys.get("Pr", 0.72),
                     q_inf=phys.get("q_inf"), p_min=p_min, p_max=p_max, flux=phys.get("flux", "rusanov"))


def rel_err(a, b):
    """max |a - b| / max |b| (global, all variables)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def per_var_err(a, b, nv):
    """max over variables of max|a_v - b_v| / max|b_v| (canonical layout: variable fastest)."""
    a = np.asarray(a).reshape(-1, nv)
    b = np.asarray(b).reshape(-1, nv)
    return max(float(np.abs(a[:, v] - b[:, v]).max() / max(np.abs(b[:, v]).max(), 1e-300)) for v in range(nv))


def flux_scale(mesh, q, gamma=1.4):
    """max|f_inviscid| * P_max^2 / h_min: the size of the terms that cancel in R."""
    nd, nv = mesh.nd, mesh.nd + 2
    Q = np.asarray(q).reshape(-1, nv)
    rho = Q[:, 0]
    vel = Q[:, 1:1 + nd] / rho[:, None]
    p = (gamma - 1) * (Q[:, nv - 1] - 0.5 * rho * (vel ** 2).sum(1))
    fmax = max(np.abs(Q[:, 1:1 + nd]).max(), (np.abs(Q[:, 1:1 + nd]) * np.abs(vel).max() + np.abs(p).max()).max(),
               (np.abs(Q[:, nv - 1] + p) * np.abs(vel).max(axis=1)).max())
    ext = mesh.nodes.max(axis=1) - mesh.nodes.min(axis=1)
    h_min = float(np.linalg.norm(ext, axis=1).min() / np.sqrt(nd))
    P = int(mesh.p.max()) + 1
    return float(fmax * P * P / h_min)


class Parity(tuple):
    """(ok, rel, flux_scaled) with ``legs``: per variable, which bound held
    ("rel": max|d_v| / max|ref_v|, "flux": max|d_v| / flux scale, or None)."""
    legs = ()


def parity_ok(gpu, ref, mesh, q, tol):
    """Per variable v: max|d_v| / max|ref_v| <= tol, or (where R_v is small next
    to the fluxes that cancel in it) max|d_v| / flux_scale <= tol.  Returns
    (ok, rel, flux_scaled) with rel and flux_scaled the worst variable's values
    and ``.legs`` naming the bound each variable met."""
    nv = mesh.nd + 2
    d = np.abs(np.asarray(gpu) - np.asarray(ref)).reshape(-1, nv)
    r = np.abs(np.asarray(ref)).reshape(-1, nv)
    fsc = flux_scale(mesh, q)
    legs, rels, fss = [], [], []
    for v in range(nv):
        dv = float(d[:, v].max())
        rel = dv / max(float(r[:, v].max()), 1e-300)
        fs = dv / fsc
        rels.append(rel)
        fss.append(fs)
        legs.append("rel" if rel <= tol else ("flux" if fs <= tol else None))
    out = Parity((all(l is not None for l in legs), max(rels), max(fss)))
    out.legs = tuple(legs)
    return out


def generic_state(q, seed=77, amp=1e-3):
    """q plus a seeded additive perturbation of amp * mean|q|.

    Rusanov's |u.n| and max(lam-, lam+) are not differentiable where a face
    sits exactly on a tie, and symmetric inputs (the Taylor-Green state with
    rho w = 0, periodic copies of the vortex) put many faces there; the
    derivative is then not unique and either one-sided value is correct.  JVP
    and VJP parity is checked on this generic nearby state instead."""
    import cases
    q = np.asarray(q)
    return q + amp * np.abs(q).mean() * (2.0 * cases.uniform(seed, q.size) - 1.0)
