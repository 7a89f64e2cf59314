"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA library.

This module holds no arithmetic of the flux-reconstruction method itself: it
builds meshes (element geometry nodes and face connectivity), polynomial-degree
maps, and initial states sampled at solution-point positions.  Both the oracle
(``oracle/``) and the GPU tests take their inputs from here, so neither side
ever produces an input for the other.

Conventions shared by both consumers
------------------------------------
* ``nd`` is 2 or 3; ``nv = nd + 2`` conservative variables (rho, rho*u_i, rho*E).
* Element faces are numbered ``f = 2*d + s`` with ``d`` the reference direction
  (0 = xi, 1 = eta, 2 = zeta) and ``s = 0`` for the face at xi_d = -1,
  ``s = 1`` for xi_d = +1.
* ``nbr[e, f] >= 0`` is the neighbouring element; ``-1`` marks a no-slip
  adiabatic wall and ``-2`` a far-field boundary.
* Face-local point indices use the tangential reference directions in
  increasing order (a = first, b = second).  ``orient[e, f]`` maps point
  ``(ia, ib)`` of element ``e`` to the neighbour's face-local indices: bit 0
  swaps the two axes, then bit 1 flips the first axis (i -> P-1-i) and bit 2
  flips the second.  Gauss points are symmetric, so a flip is xi -> -xi.
* Geometry nodes of an element are ``(g+1)**nd`` equispaced points of the
  reference cube, xi fastest (index ``i + (g+1)*j + (g+1)**2*k``).
* The canonical state layout is, element by element in id order,
  ``n_sp(p_e) = (p_e+1)**nd`` solution points (xi fastest) times ``nv``
  variables (variable fastest), FP64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

WALL = -1
FARFIELD = -2
GAMMA = 1.4

# ----------------------------------------------------------------------------
# Counter-based random numbers (SplitMix64, Steele, Lea & Flood 2014)
# ----------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """``n`` 64-bit outputs of SplitMix64 for ``seed``; ``stream`` offsets the counter."""
    with np.errstate(over="ignore"):
        ctr = np.arange(1, n + 1, dtype=np.uint64) + np.uint64((stream * 0x100000000) & (2**64 - 1))
        z = np.uint64(seed & (2**64 - 1)) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n, stream) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """Standard normal doubles by Box-Muller on two uniform streams."""
    u1 = uniform(seed, n, 2 * stream + 1)
    u2 = uniform(seed, n, 2 * stream + 2)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


SEED_BASE = 1903693


def config_seed(index: int) -> int:
    """Seed of workload ``index`` (1-based numbering of the five workloads)."""
    return SEED_BASE + index


# ----------------------------------------------------------------------------
# Mesh container
# ----------------------------------------------------------------------------
@dataclass
class Mesh:
    nd: int
    geom_order: int
    nodes: np.ndarray          # [E, (g+1)**nd, nd] float64
    nbr: np.ndarray            # [E, 2*nd] int32
    nbr_face: np.ndarray       # [E, 2*nd] int8
    orient: np.ndarray         # [E, 2*nd] int8
    p: np.ndarray              # [E] int8
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_elem(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def nv(self) -> int:
        return self.nd + 2

    def n_sp(self) -> np.ndarray:
        return (self.p.astype(np.int64) + 1) ** self.nd

    def n_dof(self) -> int:
        return int(self.n_sp().sum()) * self.nv

    def offsets(self) -> np.ndarray:
        """Start of each element's block in the canonical state vector."""
        sizes = self.n_sp() * self.nv
        off = np.zeros(self.n_elem + 1, dtype=np.int64)
        np.cumsum(sizes, out=off[1:])
        return off

    def with_p(self, p) -> "Mesh":
        p = np.broadcast_to(np.asarray(p, dtype=np.int8), (self.n_elem,)).copy()
        return Mesh(self.nd, self.geom_order, self.nodes, self.nbr, self.nbr_face,
                    self.orient, p, self.name, dict(self.meta))


def check_connectivity(m: Mesh) -> None:
    """Every interior face must point back at itself through its neighbour."""
    nf = 2 * m.nd
    for e in range(m.n_elem):
        for f in range(nf):
            n = int(m.nbr[e, f])
            if n < 0:
                continue
            g = int(m.nbr_face[e, f])
            assert int(m.nbr[n, g]) == e and int(m.nbr_face[n, g]) == f, (e, f, n, g)


# ----------------------------------------------------------------------------
# Structured-block mesh builder
# ----------------------------------------------------------------------------
def _structured(nd, dims, g, param_map, periodic, bc_lo, bc_hi, p, name,
                jitter=None):
    """Build a structured block of ``prod(dims)`` elements.

    ``param_map(s)`` maps parametric coordinates ``s`` in [0,1]^nd (array
    ``[..., nd]``) to physical coordinates.  Geometry nodes of degree ``g`` are
    placed at equispaced parametric positions inside each element.  ``jitter``
    optionally returns a displacement added to element *vertex* parameters.
    Element index is ``i + n0*(j + n1*k)`` (i along xi).
    """
    dims = list(dims)
    E = int(np.prod(dims))
    nn = g + 1
    # global parametric grid of geometry nodes, size g*dims+1 per direction
    axes = [np.arange(g * n + 1) / (g * n) for n in dims]
    grids = np.meshgrid(*axes, indexing="ij")
    S = np.stack(grids, axis=-1)            # [..., nd] indexed (i, j, k)
    if jitter is not None:
        S = S + jitter(S)
    X = param_map(S)                         # [..., nd]
    # gather element nodes
    nodes = np.zeros((E,) + (nn ** nd, nd))
    # local node a = i + nn*j + nn^2*k  (xi fastest)
    loc = np.array([[(a // nn ** d) % nn for d in range(nd)] for a in range(nn ** nd)])
    eidx = np.stack(np.meshgrid(*[np.arange(n) for n in dims], indexing="ij"), -1).reshape(-1, nd)
    # element linear index: i + n0*(j + n1*k)
    lin = np.zeros(len(eidx), dtype=np.int64)
    mul = 1
    for d in range(nd):
        lin += eidx[:, d] * mul
        mul *= dims[d]
    gidx = eidx[:, None, :] * g + loc[None, :, :]          # [E, nn^nd, nd]
    nodes[lin] = X[tuple(np.moveaxis(gidx, -1, 0))]
    nbr = np.zeros((E, 2 * nd), dtype=np.int32)
    nbr_face = np.zeros((E, 2 * nd), dtype=np.int8)
    orient = np.zeros((E, 2 * nd), dtype=np.int8)
    for d in range(nd):
        for s in (0, 1):
            f = 2 * d + s
            jj = eidx.copy()
            jj[:, d] += 1 if s == 1 else -1
            out = (jj[:, d] < 0) | (jj[:, d] >= dims[d])
            jj[:, d] %= dims[d]
            ne = np.zeros(E, dtype=np.int64)
            mul = 1
            for dd in range(nd):
                ne += jj[:, dd] * mul
                mul *= dims[dd]
            nb = ne.astype(np.int32)
            nf = np.full(E, 2 * d + (1 - s), dtype=np.int8)
            if not periodic[d]:
                nb[out] = (bc_hi if s == 1 else bc_lo)[d]
                nf[out] = -1
            nbr[lin, f] = nb
            nbr_face[lin, f] = nf
    pp = np.broadcast_to(np.asarray(p, dtype=np.int8), (E,)).copy()
    return Mesh(nd, g, nodes, nbr, nbr_face, orient, pp, name)


def periodic_box(nd, n, lo, hi, p, g=1, name="box", jitter_frac=0.0, seed=0):
    """Uniform periodic box of ``n**nd`` elements on ``[lo, hi]**nd``.

    ``jitter_frac`` moves every interior vertex by a uniform random amount in
    ``+-jitter_frac*h`` per coordinate (boundary vertices stay fixed so that
    periodic images match).
    """
    dims = [n] * nd
    L = hi - lo

    def pmap(S):
        return lo + L * S

    jit = None
    if jitter_frac > 0.0:
        assert g == 1

        def jit(S):
            shp = S.shape
            u = uniform(seed, int(np.prod(shp)), stream=7).reshape(shp)
            dS = (2.0 * u - 1.0) * jitter_frac / n
            interior = np.ones(shp[:-1], dtype=bool)
            for d in range(nd):
                idx = [slice(None)] * nd
                idx[d] = 0
                interior[tuple(idx)] = False
                idx[d] = -1
                interior[tuple(idx)] = False
            return dS * interior[..., None]

    return _structured(nd, dims, g, pmap, [True] * nd, [0] * nd, [0] * nd, p, name, jit)


def merge(meshes, name="batch") -> Mesh:
    """Disjoint union of meshes of equal ``nd`` and geometry order."""
    nd = meshes[0].nd
    g = meshes[0].geom_order
    off = 0
    nodes, nbr, nf, ori, p = [], [], [], [], []
    sizes = []
    for m in meshes:
        assert m.nd == nd and m.geom_order == g
        nodes.append(m.nodes)
        b = m.nbr.copy()
        b[b >= 0] += off
        nbr.append(b)
        nf.append(m.nbr_face)
        ori.append(m.orient)
        p.append(m.p)
        sizes.append(m.n_elem)
        off += m.n_elem
    return Mesh(nd, g, np.concatenate(nodes), np.concatenate(nbr), np.concatenate(nf),
                np.concatenate(ori), np.concatenate(p), name, {"instance_sizes": sizes})


# ----------------------------------------------------------------------------
# Cylinder O-grid and NACA0012 C-grid
# ----------------------------------------------------------------------------
def _geometric_ratio(first, total, n):
    """Ratio q with first*(q**n - 1)/(q - 1) == total (bisection)."""
    lo, hi = 1.0 + 1e-12, 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if first * (mid ** n - 1.0) / (mid - 1.0) > total:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def cylinder_ogrid(nr=64, nt=96, nz=16, r0=0.5, r1=20.0, first=0.005, span=2.0,
                   g=2, p=1, name="cylinder"):
    """O-grid around a cylinder of diameter 1, extruded along z (periodic).

    Direction 0 = radial (wall at r0, far field at r1), 1 = azimuthal
    (periodic), 2 = span (periodic).  Radial spacing grows geometrically from
    ``first``.  Geometry nodes of degree ``g`` sit on the exact polar map.
    """
    q = _geometric_ratio(first, r1 - r0, nr)

    def pmap(S):
        s, t, u = S[..., 0], S[..., 1], S[..., 2]
        r = r0 + first * (q ** (s * nr) - 1.0) / (q - 1.0)
        th = 2.0 * np.pi * t    # (r, theta, z) right-handed: positive Jacobian
        return np.stack([r * np.cos(th), r * np.sin(th), span * u], axis=-1)

    m = _structured(3, [nr, nt, nz], g, pmap, [False, True, True], [WALL, 0, 0],
                    [FARFIELD, 0, 0], p, name)
    m.meta.update(dict(nr=nr, nt=nt, nz=nz, r0=r0, r1=r1))
    return m


def naca0012_half_thickness(x):
    """Closed-trailing-edge NACA 0012 half thickness (last coefficient -0.1036)."""
    t = 0.12
    x = np.clip(x, 0.0, 1.0)
    return 5.0 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2
                      + 0.2843 * x ** 3 - 0.1036 * x ** 4)


def naca_cgrid(ni=256, nj=64, nk=24, n_wake=48, span=0.2, r_far=10.0, x_far=10.0,
               first=2e-3, p=1, name="naca0012"):
    """Extruded C-grid around a NACA 0012 profile (chord 1, trilinear hexes).

    Direction 0 runs along the C from the lower wake exit, round the profile, to
    the upper wake exit; direction 1 points away from the profile (j = 0 is the
    wall on the profile and the wake cut elsewhere); direction 2 is the span
    (periodic).  Elements on the two sides of the wake cut are face neighbours
    with the first face axis reversed.
    """
    assert ni > 2 * n_wake
    n_foil = ni - 2 * n_wake
    half = n_foil // 2
    q = _geometric_ratio(first, 1.0, nj)

    def inner(i):
        """Inner boundary point for vertex index i in [0, ni] (float allowed)."""
        i = np.asarray(i, dtype=np.float64)
        x = np.empty_like(i)
        y = np.zeros_like(i)
        w_lo = i <= n_wake
        w_hi = i >= ni - n_wake
        foil = ~(w_lo | w_hi)
        # lower wake: from x_far back to the trailing edge, stretched toward TE
        t = (n_wake - i[w_lo]) / n_wake
        x[w_lo] = 1.0 + (x_far - 1.0) * (t ** 1.8)
        t = (i[w_hi] - (ni - n_wake)) / n_wake
        x[w_hi] = 1.0 + (x_far - 1.0) * (t ** 1.8)
        # profile: cosine clustering at both edges; lower then upper surface
        s = (i[foil] - n_wake) / n_foil       # 0..1 around the profile
        lower = s < 0.5
        th = np.where(lower, s / 0.5, (s - 0.5) / 0.5) * np.pi
        xl = 0.5 * (1.0 + np.cos(th))          # lower: TE(1) -> LE(0)
        xu = 0.5 * (1.0 - np.cos(th))          # upper: LE(0) -> TE(1)
        xx = np.where(lower, xl, xu)
        yy = np.where(lower, -naca0012_half_thickness(xl), naca0012_half_thickness(xu))
        x[foil] = xx
        y[foil] = yy
        return np.stack([x, y], -1)

    def outer(i):
        """Outer boundary: a C made of a half circle round the nose and two lines."""
        i = np.asarray(i, dtype=np.float64)
        s = i / ni
        # lengths: lower line, half circle, upper line
        L_line = x_far - 0.5
        L_arc = np.pi * r_far
        Ltot = 2 * L_line + L_arc
        a = s * Ltot
        x = np.empty_like(s)
        y = np.empty_like(s)
        m1 = a <= L_line
        m3 = a >= L_line + L_arc
        m2 = ~(m1 | m3)
        x[m1] = x_far - a[m1]
        y[m1] = -r_far
        th = (a[m2] - L_line) / r_far     # 0 .. pi
        x[m2] = 0.5 - r_far * np.sin(th)
        y[m2] = -r_far * np.cos(th)
        x[m3] = 0.5 + (a[m3] - L_line - L_arc)
        y[m3] = r_far
        return np.stack([x, y], -1)

    def pmap(S):
        s, t, u = S[..., 0], S[..., 1], S[..., 2]
        iv = s * ni
        a = inner(iv.reshape(-1)).reshape(iv.shape + (2,))
        b = outer(iv.reshape(-1)).reshape(iv.shape + (2,))
        w = first * (q ** (t * nj) - 1.0) / (q - 1.0)
        xy = a + w[..., None] * (b - a)
        return np.concatenate([xy, (span * u)[..., None]], axis=-1)

    m = _structured(3, [ni, nj, nk], 1, pmap, [False, False, True],
                    [FARFIELD, WALL, 0], [FARFIELD, FARFIELD, 0], p, name)
    # wake cut: (i, 0, k) <-> (ni-1-i, 0, k) through face 2 (eta = -1)
    for k in range(nk):
        for i in range(n_wake):
            e = i + ni * (0 + nj * k)
            o = (ni - 1 - i) + ni * (0 + nj * k)
            for a, b in ((e, o), (o, e)):
                m.nbr[a, 2] = b
                m.nbr_face[a, 2] = 2
                m.orient[a, 2] = 2     # flip first face axis (xi)
    m.meta.update(dict(ni=ni, nj=nj, nk=nk, n_wake=n_wake))
    return m


# ----------------------------------------------------------------------------
# Sampling helpers (solution-point positions for initial states)
# ----------------------------------------------------------------------------
def _gauss_1d(P):
    x, _ = np.polynomial.legendre.leggauss(P)
    return x


def _equi_basis(g, x):
    """Lagrange basis on g+1 equispaced nodes of [-1,1], evaluated at x: [len(x), g+1]."""
    nodes = np.linspace(-1.0, 1.0, g + 1)
    B = np.ones((len(x), g + 1))
    for a in range(g + 1):
        for b in range(g + 1):
            if b != a:
                B[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return B


def solution_point_positions(m: Mesh) -> list:
    """Physical positions of the solution points, one array [n_sp, nd] per element.

    Points are the tensor Gauss-Legendre points of degree p_e (xi fastest)
    pushed through the element's node map.  Used only to sample initial states.
    """
    out = [None] * m.n_elem
    for p in np.unique(m.p):
        P = int(p) + 1
        x = _gauss_1d(P)
        B = _equi_basis(m.geom_order, x)     # [P, g+1]
        if m.nd == 2:
            W = np.einsum("jb,ia->jiba", B, B).reshape(P * P, -1)
        else:
            W = np.einsum("kc,jb,ia->kjicba", B, B, B).reshape(P ** 3, -1)
        idx = np.nonzero(m.p == p)[0]
        X = np.einsum("sn,end->esd", W, m.nodes[idx])
        for r, e in enumerate(idx):
            out[e] = X[r]
    return out


def prim_to_cons(rho, vel, pres, gamma=GAMMA):
    """Conservative variables [..., nv] from density, velocity [..., nd], pressure."""
    nd = vel.shape[-1]
    q = np.empty(rho.shape + (nd + 2,))
    q[..., 0] = rho
    q[..., 1:1 + nd] = rho[..., None] * vel
    q[..., nd + 1] = pres / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, -1)
    return q


def _flatten(states):
    return np.concatenate([s.reshape(-1) for s in states])


def vortex_state(m: Mesh, alpha=5.0, phi=0.5, mach=0.5, u_inf=(1.0, 1.0), center=(0.0, 0.0),
                 gamma=GAMMA):
    """Isentropic vortex (paper's Sec. 3.3 definition) sampled at solution points.

    Free stream rho = 1, velocity ``u_inf``, pressure 1/(gamma*Ma^2) (Mach number
    referred to unit speed); T = p/rho; r is the distance to the vortex centre.
    """
    pinf = 1.0 / (gamma * mach ** 2)
    Tinf = pinf / 1.0
    out = []
    for X in solution_point_positions(m):
        dx = X[:, 0] - center[0]
        dy = X[:, 1] - center[1]
        r2 = dx * dx + dy * dy
        ex = np.exp(phi * (1.0 - r2))
        du = -alpha / (2 * np.pi) * dy * ex
        dv = alpha / (2 * np.pi) * dx * ex
        dT = -alpha ** 2 * (gamma - 1.0) / (16 * phi * gamma * np.pi ** 2) * ex * ex
        T = Tinf + dT
        rho = (T / Tinf) ** (1.0 / (gamma - 1.0))
        pres = rho * T
        vel = np.zeros((len(X), m.nd))
        vel[:, 0] = u_inf[0] + du
        vel[:, 1] = u_inf[1] + dv
        out.append(prim_to_cons(rho, vel, pres, gamma))
    return _flatten(out)


def vortex_exact(m: Mesh, t, alpha=5.0, phi=0.5, mach=0.5, u_inf=(1.0, 1.0), period=None,
                 gamma=GAMMA):
    """Vortex advected by ``u_inf*t``; with ``period`` the nearest periodic image is used."""
    cx, cy = u_inf[0] * t, u_inf[1] * t
    if period is not None:
        # sample with the centre wrapped into the box; images beyond the nearest neglected
        lo, L = period
        cx = lo + np.mod(cx - lo, L)
        cy = lo + np.mod(cy - lo, L)
    return vortex_state(m, alpha, phi, mach, u_inf, (cx, cy), gamma)


def tgv_state(m: Mesh, mach=0.1, gamma=GAMMA):
    """Taylor-Green vortex, rho0 = V0 = L = 1, p0 = 1/(gamma Ma^2), isothermal start."""
    p0 = 1.0 / (gamma * mach ** 2)
    out = []
    for X in solution_point_positions(m):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        u = np.sin(x) * np.cos(y) * np.cos(z)
        v = -np.cos(x) * np.sin(y) * np.cos(z)
        w = np.zeros_like(x)
        pres = p0 + (1.0 / 16.0) * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
        rho = pres / p0
        out.append(prim_to_cons(rho, np.stack([u, v, w], -1), pres, gamma))
    return _flatten(out)


def fourier_state(m: Mesh, seed, mach=0.3, amp=0.05, kmax=4, n_modes=24, gamma=GAMMA):
    """Uniform flow rho=1, u=(1,0,0) with each primitive variable perturbed by
    ``n_modes`` seeded Fourier modes (|k|_inf <= kmax), total amplitude ``amp``
    relative to the variable's scale (1 for rho and velocity, p_inf for p)."""
    pinf = 1.0 / (gamma * mach ** 2)
    nd = m.nd
    nvar = nd + 2
    ks = (np.floor(uniform(seed, n_modes * nvar * nd, 11) * (2 * kmax + 1)) - kmax).reshape(nvar, n_modes, nd)
    ph = 2 * np.pi * uniform(seed, n_modes * nvar, 12).reshape(nvar, n_modes)
    a = (2 * uniform(seed, n_modes * nvar, 13) - 1).reshape(nvar, n_modes)
    a = a / np.abs(a).sum(1, keepdims=True) * amp
    scale = np.array([1.0] + [1.0] * nd + [pinf])
    base = np.array([1.0, 1.0] + [0.0] * (nd - 1) + [pinf])
    out = []
    for X in solution_point_positions(m):
        prim = np.empty((len(X), nvar))
        for v in range(nvar):
            arg = X @ ks[v].T + ph[v]          # [n_sp, n_modes]
            prim[:, v] = base[v] + scale[v] * (np.cos(arg) @ a[v])
        out.append(prim_to_cons(prim[:, 0], prim[:, 1:1 + nd], prim[:, nd + 1], gamma))
    return _flatten(out)


def freestream_state(m: Mesh, rho=1.0, vel=(1.0, 0.0, 0.0), mach=0.2, gamma=GAMMA,
                     noise=0.0, seed=0):
    """Uniform state (unit speed reference for Mach), optional Gaussian velocity noise."""
    pinf = rho * 1.0 / (gamma * mach ** 2)
    nd = m.nd
    v0 = np.asarray(vel[:nd], dtype=np.float64)
    nsp = m.n_sp()
    n = int(nsp.sum())
    vel_all = np.broadcast_to(v0, (n, nd)).copy()
    if noise > 0.0:
        vel_all += noise * normal(seed, n * nd, 21).reshape(n, nd)
    q = prim_to_cons(np.full(n, rho), vel_all, np.full(n, pinf), gamma)
    return q.reshape(-1)


def random_state(m: Mesh, seed, mach=0.3, amp=0.05, gamma=GAMMA):
    """Smooth-free random perturbation of a uniform flow at every solution point."""
    nd = m.nd
    n = int(m.n_sp().sum())
    pinf = 1.0 / (gamma * mach ** 2)
    u = uniform(seed, n * (nd + 2), 31).reshape(n, nd + 2) * 2 - 1
    rho = 1.0 + amp * u[:, 0]
    vel = np.zeros((n, nd))
    vel[:, 0] = 1.0
    vel += amp * u[:, 1:1 + nd]
    pres = pinf * (1.0 + amp * u[:, nd + 1])
    return prim_to_cons(rho, vel, pres, gamma).reshape(-1)


def free_stream_q(nd, rho=1.0, vel=(1.0, 0.0, 0.0), mach=0.2, gamma=GAMMA):
    """Conservative free-stream state (length nv)."""
    pinf = rho / (gamma * mach ** 2)
    v = np.asarray(vel[:nd], dtype=np.float64)
    return prim_to_cons(np.array(rho), v, np.array(pinf), gamma)


# ----------------------------------------------------------------------------
# Polynomial-degree fields
# ----------------------------------------------------------------------------
def element_centroids(m: Mesh) -> np.ndarray:
    return m.nodes.mean(axis=1)


def smooth_random_p_field(m: Mesh, seed, fractions=(0.4, 0.3, 0.2, 0.1), levels=(1, 2, 3, 4),
                          n_modes=8, wall_bias=1.0, length=4.0):
    """Seeded smooth field (``n_modes`` random Fourier modes plus a bias toward
    small radius) ranked and split so that ``fractions`` of the elements get
    ``levels`` (lowest field -> lowest level)."""
    c = element_centroids(m)
    nd = m.nd
    k = (2 * uniform(seed, n_modes * nd, 41).reshape(n_modes, nd) - 1) * (2 * np.pi / length)
    ph = 2 * np.pi * uniform(seed, n_modes, 42)
    a = 2 * uniform(seed, n_modes, 43) - 1
    f = np.cos(c @ k.T + ph) @ a / n_modes
    r = np.sqrt(np.sum(c[:, :2] ** 2, -1))
    f = f - wall_bias * np.log(np.maximum(r, 1e-3))
    order = np.lexsort((np.arange(m.n_elem), f))
    p = np.empty(m.n_elem, dtype=np.int8)
    bounds = np.round(np.cumsum((0.0,) + tuple(fractions)) * m.n_elem).astype(int)
    for lv, a0, a1 in zip(levels, bounds[:-1], bounds[1:]):
        p[order[a0:a1]] = lv
    return p


def limit_jumps_down(m: Mesh, p) -> np.ndarray:
    """Input repair: lower any element more than one degree above a neighbour
    until neighbouring degrees differ by at most one."""
    p = p.astype(np.int64).copy()
    changed = True
    while changed:
        changed = False
        for f in range(2 * m.nd):
            nb = m.nbr[:, f]
            ok = nb >= 0
            pn = np.where(ok, p[np.maximum(nb, 0)], 0)
            bad = ok & (p > pn + 1)
            if bad.any():
                p[bad] = pn[bad] + 1
                changed = True
    return p.astype(np.int8)


# ----------------------------------------------------------------------------
# The five workloads
# ----------------------------------------------------------------------------
PHYS_VORTEX = dict(gamma=GAMMA, mu=0.0, Pr=0.72)
PHYS_TGV = dict(gamma=GAMMA, mu=1.0 / 1600.0, Pr=0.71)
PHYS_CYL = dict(gamma=GAMMA, mu=1.0 / 3900.0, Pr=0.71)
PHYS_DIFF = dict(gamma=GAMMA, mu=1.0 / 1600.0, Pr=0.71)
PHYS_NACA = dict(gamma=GAMMA, mu=1.0 / 60000.0, Pr=0.72)


def workload_vortex2d(n=16, p=2, jitter=0.1, lo=-5.0, hi=5.0):
    """2D Euler isentropic vortex on a periodic jittered n x n quad mesh."""
    m = periodic_box(2, n, lo, hi, p, g=1, name=f"vortex2d_{n}x{n}_p{p}",
                     jitter_frac=jitter, seed=config_seed(1))
    return m, vortex_state(m), dict(PHYS_VORTEX)


def workload_tgv(n=32, p=3):
    """3D Navier-Stokes Taylor-Green vortex, Re 1600, Ma 0.1, periodic box."""
    m = periodic_box(3, n, 0.0, 2 * np.pi, p, g=1, name=f"tgv_{n}^3_p{p}")
    return m, tgv_state(m, mach=0.1), dict(PHYS_TGV)


def workload_cylinder(nr=64, nt=96, nz=16, p_levels=(1, 2, 3, 4)):
    """Cylinder O-grid, quadratic geometry, seeded mixed p, free stream + 1% noise."""
    m = cylinder_ogrid(nr, nt, nz, g=2)
    m.p = smooth_random_p_field(m, config_seed(3), levels=p_levels)
    q = freestream_state(m, vel=(1.0, 0.0, 0.0), mach=0.2, noise=0.01, seed=config_seed(3))
    phys = dict(PHYS_CYL)
    phys["q_inf"] = free_stream_q(3, vel=(1.0, 0.0, 0.0), mach=0.2)
    return m, q, phys


def workload_diff(n=24, p=4):
    """Periodic box, seeded Fourier perturbation of uniform flow at Ma 0.3."""
    m = periodic_box(3, n, 0.0, 2 * np.pi, p, g=1, name=f"diff_{n}^3_p{p}")
    return m, fourier_state(m, config_seed(4), mach=0.3), dict(PHYS_DIFF)


def workload_naca(ni=256, nj=64, nk=24, n_wake=48, p=1, aoa_deg=8.0):
    """Extruded NACA 0012 C-grid at 8 degrees incidence, Re 6e4, Ma 0.2."""
    m = naca_cgrid(ni, nj, nk, n_wake=n_wake, p=p)
    a = math.radians(aoa_deg)
    vel = (math.cos(a), math.sin(a), 0.0)
    q = freestream_state(m, vel=vel, mach=0.2, noise=0.01, seed=config_seed(5))
    phys = dict(PHYS_NACA)
    phys["q_inf"] = free_stream_q(3, vel=vel, mach=0.2)
    return m, q, phys


def workload_vortex_batch(n_inst=32, nmin=8, nmax=64, pmin=1, pmax=5, seed=None):
    """Independent 2D vortex instances of uneven size and degree in one mesh."""
    seed = config_seed(5) if seed is None else seed
    u = uniform(seed, 2 * n_inst, 51).reshape(n_inst, 2)
    meshes, states = [], []
    for i in range(n_inst):
        n = int(nmin + np.floor(u[i, 0] * (nmax - nmin + 1)))
        p = int(pmin + np.floor(u[i, 1] * (pmax - pmin + 1)))
        mi = periodic_box(2, n, -5.0, 5.0, p, g=1, name=f"v{i}")
        meshes.append(mi)
        states.append(vortex_state(mi))
    m = merge(meshes, "vortex_batch")
    return m, np.concatenate(states), dict(PHYS_VORTEX)
