"""p-adaptation (Sec. 3.1), FP64 / integer, test infrastructure only.

* Spectral decay indicator eta = ||s_p - s_{p-1}|| / ||s_p|| with the paper's
  weighted "norm" sum((.)^2 w_xi w_eta w_zeta |J|) / sum(w_xi w_eta w_zeta |J|)
  (Eq. eta_k and the following definition).  Reading: the printed norm has no
  square root, so eta = sum(w|J|(s_p - s_{p-1})^2) / sum(w|J| s_p^2); s_{p-1}
  is the reference-space Legendre truncation that drops every tensor mode with
  an index equal to p; eta = 0 where the denominator is 0.  Variable: rho*u.
* Criteria: p+1 if eta > nu_max eta_max, p-1 if eta < nu_min eta_max (strict),
  clamp to [p_min, p_max]; eta_max is the maximum over all elements; nothing
  changes when eta_max = 0.
* Jump limit |p_e - p_n| <= 1 across faces: raise-only fixed point
  p_e <- max(p_e, max_n p_n - 1) (reading of "limit the difference ... to one").
* Prolongation: interpolation of the degree-p polynomial at the new points;
  projection: Legendre truncation, then evaluation at the new points.
* Bucket order: ascending (p, element id).
"""
import numpy as np
import torch

from .basis import basis, lagrange, legendre
from .geometry import apply1d


def _weights(p, nd):
    w = basis(p).w
    if nd == 2:
        return w[:, None] * w[None, :]
    return w[:, None, None] * w[None, :, None] * w[None, None, :]


def truncate(s: torch.Tensor, p: int, nd: int) -> torch.Tensor:
    """Drop every Legendre mode with an index equal to p (tensor Q_{p-1})."""
    b = basis(p)
    c = s
    for d in range(nd):
        c = apply1d(b.to_modal, c, d)
    keep = torch.ones(p + 1)
    keep[p] = 0.0
    for d in range(nd):
        shape = [1] * c.dim()
        shape[c.dim() - 1 - d] = p + 1
        c = c * keep.reshape(shape)
    for d in range(nd):
        c = apply1d(b.to_nodal, c, d)
    return c


def indicator(fr, q: torch.Tensor, var: int = 1) -> np.ndarray:
    """eta per element (element id order)."""
    nd = fr.nd
    Q = fr.to_groups(q)
    eta = np.zeros(fr.mesh.n_elem)
    for pg, G in fr.groups.items():
        s = Q[pg][:, var]
        sl = truncate(s, pg, nd)
        wj = _weights(pg, nd) * G["geom"].J
        num = (wj * (s - sl) ** 2).flatten(1).sum(1)
        den = (wj * s * s).flatten(1).sum(1)
        e = torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)), torch.zeros_like(den))
        eta[G["elems"]] = e.numpy()
    return eta


def decide(eta, p, nu_max=0.1, nu_min=0.001, p_min=1, p_max=3):
    eta = np.asarray(eta, dtype=np.float64)
    p = np.asarray(p, dtype=np.int64).copy()
    emax = float(eta.max()) if eta.size else 0.0
    if emax > 0.0:
        up = eta > nu_max * emax
        dn = eta < nu_min * emax
        p = p + up.astype(np.int64) - dn.astype(np.int64)
    return np.clip(p, p_min, p_max)


def limit_jumps(mesh, p):
    """Smallest p' >= p (elementwise) with |p'_e - p'_n| <= 1 across every face."""
    p = np.asarray(p, dtype=np.int64).copy()
    while True:
        new = p.copy()
        for f in range(2 * mesh.nd):
            nb = mesh.nbr[:, f]
            ok = nb >= 0
            new[ok] = np.maximum(new[ok], p[nb[ok]] - 1)
        if np.array_equal(new, p):
            return p
        p = new


def adapt_p(fr, q, nu_max=0.1, nu_min=0.001, p_min=1, p_max=3, var=1):
    eta = indicator(fr, q, var)
    p_dec = decide(eta, fr.mesh.p, nu_max, nu_min, p_min, p_max)
    return limit_jumps(fr.mesh, p_dec), eta


def transfer_element(s: torch.Tensor, p_old: int, p_new: int, nd: int) -> torch.Tensor:
    """Move a nodal field [..., (P,)*nd] from degree p_old to p_new."""
    if p_new == p_old:
        return s
    b_old, b_new = basis(p_old), basis(p_new)
    if p_new < p_old:
        # Legendre truncation to degree p_new, then evaluation at the new points
        c = s
        for d in range(nd):
            c = apply1d(b_old.to_modal, c, d)
        idx = torch.arange(p_new + 1)
        for d in range(nd):
            c = torch.index_select(c, c.dim() - 1 - d, idx)
        V = torch.stack([legendre(m, b_new.x)[0] for m in range(p_new + 1)], dim=1)
        for d in range(nd):
            c = apply1d(V, c, d)
        return c
    M = lagrange(b_old.x, b_new.x)
    for d in range(nd):
        s = apply1d(M, s, d)
    return s


def transfer(fr_old, q_old: torch.Tensor, fr_new) -> torch.Tensor:
    """State transfer between two discretisations of the same mesh."""
    nd, nv = fr_old.nd, fr_old.nv
    Q = fr_old.to_groups(q_old)
    p_old = fr_old.mesh.p.astype(np.int64)
    p_new = fr_new.mesh.p.astype(np.int64)
    parts = {}
    for pg, G in fr_new.groups.items():
        P = pg + 1
        out = torch.zeros((len(G["elems"]), nv) + (P,) * nd)
        for po in sorted(set(p_old[G["elems"]].tolist())):
            sel = np.nonzero(p_old[G["elems"]] == po)[0]
            src = fr_old.pos[G["elems"][sel]]
            out[torch.from_numpy(sel)] = transfer_element(Q[po][torch.from_numpy(src)], po, pg, nd)
        parts[pg] = out
    return fr_new.from_groups(parts)


def bucket_order(p) -> np.ndarray:
    """Element ids sorted by (p, id): position -> element id."""
    p = np.asarray(p, dtype=np.int64)
    return np.lexsort((np.arange(len(p)), p))


def nodal_filter(fr, q: torch.Tensor, alpha: float = 0.2, p_above: int = 2) -> torch.Tensor:
    """Nodal polynomial filter (Sec. 4.2, after Fischer and Mullen): every element
    of degree p > p_above becomes (1 - alpha) q + alpha P_{p-1} q, P_{p-1} the
    projection onto the degree p-1 space (the modal truncation above).  The
    paper states it for p = 3 and projection onto p = 2; for higher degrees the
    projection is onto p - 1.  Lower-degree elements are unchanged."""
    parts = fr.to_groups(q)
    out = {}
    for p, s in parts.items():
        if p > p_above:
            out[p] = (1.0 - alpha) * s + alpha * truncate(s, p, fr.nd)
        else:
            out[p] = s
    return fr.from_groups(out)

