"""Seeded synthetic inputs for the immersed-boundary (IB) time step.

This module holds geometry and random numbers only: marker lattices (an
icosphere shell, a helicoidal basilar-membrane ribbon, tubular canal walls),
link lists, the graded membrane stiffness profile, the forcing region's
description and seeded random fields.  None of the method's arithmetic (the
force laws, the discrete delta function, spreading, interpolation or the fluid
solve) lives here: the CPU oracle and the CUDA path both take these arrays as
inputs, and neither imports the other.

Random numbers come from a counter-based SplitMix64 generator: value i of
stream ``s`` under seed ``q`` is ``mix64(base(q, s) + (i + 1) * 0x9E3779B97F4A7C15)``
with Steele, Lea and Flood's SplitMix64 finaliser ``mix64``.  Normal deviates
use the Box-Muller transform.

The synthetic cochlea stands in for the paper's anatomical model (Section 4:
six surfaces, 31 grids, about 750k points built from measurements that are
not available): a helicoidal membrane ribbon 3.5 cm long over 2.5 turns whose
width grows from base to apex, inside a tube of tethered wall markers.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, stream: int, n: int) -> np.ndarray:
    """n raw 64-bit values of stream ``stream`` under ``seed`` (counter based)."""
    base = _mix64(np.array([((seed & 0xFFFFFFFF) << 32) ^ (stream & 0xFFFFFFFF)], dtype=np.uint64))[0]
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = base + i * _GAMMA
    return _mix64(x)


def uniform(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n uniform deviates in [lo, hi) (53-bit mantissa)."""
    u = (splitmix64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal deviates (Box-Muller on two uniform streams)."""
    u1 = uniform(seed, stream, n)
    u2 = uniform(seed, stream + 0x10000, n)
    u1 = 1.0 - u1  # (0, 1]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# Problem description containers (plain arrays; no physics).
# ----------------------------------------------------------------------------
@dataclass
class Grid:
    n: tuple            # (nx, ny, nz) grid points per axis
    h: float            # mesh width (cm); box edge L_j = n_j * h
    rho: float          # fluid density (g/cm^3)
    mu: float           # viscosity (g/(cm s))
    dt: float           # time step (s)

    @property
    def G(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


@dataclass
class Sheet:
    """A rectangular marker lattice: marker (i, a) has index first + i*n2 + a.

    i runs along the membrane's length (n1 rows), a across its width (n2).
    ds is the length-wise spacing, dw[i] the width-wise spacing of row i and
    seg_of_row[i] the stiffness segment that row i belongs to.
    """
    first: int
    n1: int
    n2: int
    ds: float
    dw: np.ndarray
    seg_of_row: np.ndarray


@dataclass
class Forcing:
    """Body-force region: cells within ``radius`` of the axis through
    ``center`` along unit ``direction`` and within ``half_len`` of ``center``
    along it.  The force density there is rho*amp*omega*cos(omega t) times
    ``direction``; amp = 0 disables it."""
    center: np.ndarray = field(default_factory=lambda: np.zeros(3))
    direction: np.ndarray = field(default_factory=lambda: np.array([1.0, 0.0, 0.0]))
    radius: float = 0.0
    half_len: float = 0.0
    amp: float = 0.0
    omega: float = 0.0


@dataclass
class MarkerForcing:
    """External force amp * cos(omega t) * direction[:, j] on marker index[j]."""
    index: np.ndarray                   # (n,) int32
    direction: np.ndarray               # (3, n)
    amp: float = 0.0                    # dyn
    omega: float = 0.0                  # rad/s


@dataclass
class Structure:
    X0: np.ndarray                      # (3, m) reference positions (cm)
    spring_ij: np.ndarray               # (ns, 2) int32
    spring_k: np.ndarray                # (ns,) dyn/cm
    spring_L0: np.ndarray               # (ns,) cm
    tether_i: np.ndarray                # (nt,) int32
    tether_k: np.ndarray                # (nt,) dyn/cm
    sheets: list                        # list[Sheet]
    bend_b: np.ndarray                  # (n_seg,) dyn cm
    forcing: Forcing = field(default_factory=Forcing)
    normal0: np.ndarray | None = None   # (3, m) unit membrane normals (membrane markers), else None
    n_membrane: int = 0                 # membrane markers are 0 .. n_membrane-1
    faces: np.ndarray | None = None     # (F, 3) triangles of a closed shell, else None
    marker_forcing: MarkerForcing | None = None
    centerline: np.ndarray | None = None  # (n1,) marker ids of the membrane's centre line, else None

    @property
    def m(self) -> int:
        return int(self.X0.shape[1])


@dataclass
class Problem:
    name: str
    grid: Grid
    structure: Structure
    X: np.ndarray                       # (3, m) initial positions
    u: np.ndarray                       # (3, nz, ny, nx) initial velocity
    t0: float = 0.0


# ----------------------------------------------------------------------------
# Icosphere (level-k midpoint subdivision of the icosahedron).
# ----------------------------------------------------------------------------
def icosphere(level: int):
    """Unit-sphere vertices (V, 3), edges (E, 2) and faces (F, 3)."""
    p = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
             (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
             (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                v = verts[a] + verts[b]
                verts.append(v / np.linalg.norm(v))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    F = np.array(faces, dtype=np.int32)
    E = set()
    for a, b, c in faces:
        for u_, v_ in ((a, b), (b, c), (c, a)):
            E.add((min(u_, v_), max(u_, v_)))
    E = np.array(sorted(E), dtype=np.int32)
    return V, E, F


def _empty_structure(X0: np.ndarray) -> Structure:
    return Structure(X0=X0,
                     spring_ij=np.zeros((0, 2), np.int32), spring_k=np.zeros(0), spring_L0=np.zeros(0),
                     tether_i=np.zeros(0, np.int32), tether_k=np.zeros(0),
                     sheets=[], bend_b=np.zeros(0))


def sphere_problem(seed: int = 1, n: int = 32, level: int = 4, radius: float = 0.25,
                   stretch: float = 1.1, k: float = 1e4, dt: float = 1e-5,
                   rho: float = 1.0, mu: float = 0.02) -> Problem:
    """Elastic icosphere shell, stretched along x, relaxing in a periodic box.

    Markers are the subdivided icosphere's vertices, scaled to ``radius`` and
    centred at (0.5, 0.5, 0.5) plus a seeded jitter in (-0.05, 0.05)^3; the
    initial shape is stretched by ``stretch`` along x about that centre.
    Springs join mesh neighbours with rest length equal to the unstretched
    edge length.
    """
    V, E, F = icosphere(level)
    c = 0.5 + uniform(seed, 1, 3, -0.05, 0.05)
    Xr = c[:, None] + radius * V.T                    # unstretched (rest) shape
    X = Xr.copy()
    X[0] = c[0] + stretch * (Xr[0] - c[0])
    L0 = np.linalg.norm(Xr[:, E[:, 1]] - Xr[:, E[:, 0]], axis=0)
    st = _empty_structure(X.copy())
    st.spring_ij = E.astype(np.int32)
    st.spring_k = np.full(len(E), float(k))
    st.spring_L0 = L0
    st.faces = F
    grid = Grid(n=(n, n, n), h=1.0 / n, rho=rho, mu=mu, dt=dt)
    u = np.zeros((3, n, n, n))
    return Problem("sphere", grid, st, X.copy(), u)


# ----------------------------------------------------------------------------
# Synthetic cochlea: helicoidal membrane ribbon inside a tube of wall markers.
# ----------------------------------------------------------------------------
HELIX_R = 0.22          # cm, radius of the membrane's centre line about the axis
HELIX_TURNS = 2.5
BM_LENGTH = 3.5         # cm
HELIX_Z0 = 0.22         # cm
TUBE_RADIUS = 0.1       # cm
BM_W_BASE = 0.01        # cm
BM_W_APEX = 0.05        # cm


def helix_c() -> float:
    """Rise per radian c = p/(2 pi) such that 2.5 turns have arclength 3.5 cm."""
    per_turn = BM_LENGTH / HELIX_TURNS
    return math.sqrt((per_turn / (2.0 * math.pi)) ** 2 - HELIX_R ** 2)


def helix_frame(s: np.ndarray, z0: float = HELIX_Z0):
    """Centre line point C(s), unit tangent T, radial unit e_r and B = T x e_r."""
    c = helix_c()
    q = math.sqrt(HELIX_R ** 2 + c ** 2)
    th = s / q
    C = np.stack([0.5 + HELIX_R * np.cos(th), 0.5 + HELIX_R * np.sin(th), z0 + c * th])
    T = np.stack([-HELIX_R * np.sin(th), HELIX_R * np.cos(th), np.full_like(th, c)]) / q
    er = np.stack([np.cos(th), np.sin(th), np.zeros_like(th)])
    B = np.cross(T.T, er.T).T
    B /= np.linalg.norm(B, axis=0)
    return C, T, er, B


def flat_spiral_frame(s: np.ndarray, length: float = BM_LENGTH, z0: float = 0.25, r_apex: float = 0.08,
                      turns: float = 2.5):
    """A centre line that lies in the plane z = z0: the Archimedean spiral
    r = r_apex + a phi about (0.5, 0.5), phi in [0, 2 pi turns], with a chosen
    so that its arclength is `length`.  s is arclength from the base (the
    outer end, s = 0) to the apex (the inner end, s = length).  Returns C(s),
    the unit tangent T (base to apex), the in-plane unit normal e_r = z x T
    (outward) and B = T x e_r = z, like helix_frame."""
    Phi = 2.0 * math.pi * turns

    def sigma(r, a):
        # arclength from the apex to radius r: the integral of sqrt(r^2 + a^2) / a dr
        def F(x):
            return (x * np.sqrt(x * x + a * a) + a * a * np.arcsinh(x / a)) / (2.0 * a)
        return F(r) - F(r_apex)

    lo, hi = 1e-6, 1.0
    for _ in range(200):                              # a: total arclength equals length
        mid = 0.5 * (lo + hi)
        if sigma(r_apex + mid * Phi, mid) < length:
            lo = mid
        else:
            hi = mid
    a = 0.5 * (lo + hi)
    target = length - np.asarray(s, dtype=np.float64)
    rl = np.full(target.shape, r_apex)
    rh = np.full(target.shape, r_apex + a * Phi)
    for _ in range(100):                              # r(s): invert the arclength
        rm = 0.5 * (rl + rh)
        below = sigma(rm, a) < target
        rl = np.where(below, rm, rl)
        rh = np.where(below, rh, rm)
    r = 0.5 * (rl + rh)
    th = (r - r_apex) / a
    C = np.stack([0.5 + r * np.cos(th), 0.5 + r * np.sin(th), np.full_like(th, z0)])
    dC = np.stack([a * np.cos(th) - r * np.sin(th), a * np.sin(th) + r * np.cos(th), np.zeros_like(th)])
    T = -dC / np.linalg.norm(dC, axis=0)
    er = np.stack([-T[1], T[0], np.zeros_like(th)])
    B = np.cross(T.T, er.T).T
    return C, T, er, B


def bm_width(s: np.ndarray, length: float = BM_LENGTH, widths=(BM_W_BASE, BM_W_APEX)) -> np.ndarray:
    w_base, w_apex = widths
    return w_base + (w_apex - w_base) * (s / length)


def graded_stiffness(s: np.ndarray, b_base: float = 1.0, b_apex: float = 1e-3,
                     length: float = BM_LENGTH) -> np.ndarray:
    """Bending stiffness graded exponentially from b_base (s=0) to b_apex (s=L)."""
    return b_base * (b_apex / b_base) ** (s / length)


def cochlea_problem(seed: int = 2, n: int = 128, bm=(512, 48), walls=(1000, 200),
                    n_fibers: int = 0, freq: float = 1000.0, dt: float = 5e-6,
                    n_seg: int = 64, k_trans: float = 1e4, k_wall: float = 1e6,
                    k_edge: float = 1e6, amp: float = 1e-4, perturb: float = 0.0,
                    rho: float = 1.0, mu: float = 0.02, name: str = "cochlea",
                    length: float = BM_LENGTH, z0: float = HELIX_Z0, nz: int | None = None,
                    frame=None, widths=(BM_W_BASE, BM_W_APEX), tube_radius: float = TUBE_RADIUS) -> Problem:
    """Helicoidal membrane ribbon (n1 x n2 markers) + tethered tube walls.

    Membrane marker (i, a): arclength s_i = i*L/(n1-1), width offset
    w_a = -W(s_i)/2 + a*W(s_i)/(n2-1) along the radial direction.  Rows are
    grouped into ``n_seg`` stiffness segments; segment stiffness is the graded
    profile at the segment centre, times (1 + perturb*xi) with xi ~ N(0,1)
    from the seed when ``perturb`` > 0.  Transverse springs join (i,a)-(i,a+1)
    with rest length equal to the initial distance; the two long edges are
    tethered.  Wall markers sit on a tube of radius `tube_radius` about the
    centre line on an (s, psi) lattice and are tethered.  Fibers join a uniformly
    chosen membrane marker to a wall marker of the nearest tube ring at a
    uniformly chosen angle, with log-uniform stiffness in [1e2, 1e5] dyn/cm.
    The membrane is `length` cm long on a helix of fixed radius and pitch
    (2.5 turns for 3.5 cm) starting at height z0, or along `frame(s)` (a
    centre line with the same outputs as helix_frame) when given; its width
    grows linearly between `widths` (base, apex); the grid is n x n x nz.
    """
    if frame is None:
        frame = lambda s_: helix_frame(s_, z0)
    n1, n2 = bm
    ns, npsi = walls
    nz = n if nz is None else nz
    ds = length / (n1 - 1)
    s_rows = np.arange(n1) * ds
    C, T, er, B = frame(s_rows)
    W = bm_width(s_rows, length, widths)
    a = np.arange(n2)
    w = -W[:, None] / 2.0 + a[None, :] * (W[:, None] / (n2 - 1))       # (n1, n2)
    Xbm = C[:, :, None] + er[:, :, None] * w[None, :, :]                # (3, n1, n2)
    Xbm = Xbm.reshape(3, n1 * n2)
    nbm = n1 * n2
    normal0 = np.repeat(B, n2, axis=1)                                  # membrane normal

    s_w = np.arange(ns) * (length / (ns - 1))
    Cw, Tw, erw, Bw = frame(s_w)
    psi = 2.0 * math.pi * np.arange(npsi) / npsi
    Xw = (Cw[:, :, None] + tube_radius * (erw[:, :, None] * np.cos(psi)[None, None, :]
                                          + Bw[:, :, None] * np.sin(psi)[None, None, :]))
    Xw = Xw.reshape(3, ns * npsi)
    X0 = np.concatenate([Xbm, Xw], axis=1)

    # transverse springs (i, a) - (i, a+1)
    ii, aa = np.meshgrid(np.arange(n1), np.arange(n2 - 1), indexing="ij")
    si = (ii * n2 + aa).ravel()
    sj = si + 1
    springs = [np.stack([si, sj], 1)]
    ks = [np.full(len(si), float(k_trans))]
    # fibers
    if n_fibers > 0:
        fi = np.minimum((uniform(seed, 11, n_fibers) * nbm).astype(np.int64), nbm - 1)
        s_f = (fi // n2) * ds
        ring = np.clip(np.rint(s_f / length * (ns - 1)).astype(np.int64), 0, ns - 1)
        l = np.minimum((uniform(seed, 12, n_fibers) * npsi).astype(np.int64), npsi - 1)
        fj = nbm + ring * npsi + l
        springs.append(np.stack([fi, fj], 1))
        ks.append(10.0 ** uniform(seed, 13, n_fibers, 2.0, 5.0))
    sij = np.concatenate(springs).astype(np.int32)
    sk = np.concatenate(ks)
    sL0 = np.linalg.norm(X0[:, sij[:, 1]] - X0[:, sij[:, 0]], axis=0)

    edge = np.concatenate([np.arange(n1) * n2, np.arange(n1) * n2 + (n2 - 1)])
    wall = np.arange(nbm, nbm + ns * npsi)
    ti = np.concatenate([edge, wall]).astype(np.int32)
    tk = np.concatenate([np.full(len(edge), float(k_edge)), np.full(len(wall), float(k_wall))])

    seg_of_row = (np.arange(n1) * n_seg) // n1
    s_centre = np.array([s_rows[seg_of_row == q].mean() for q in range(n_seg)])
    bend_b = graded_stiffness(s_centre, length=length)
    if perturb:
        bend_b = bend_b * (1.0 + perturb * normal(seed, 21, n_seg))
    sheet = Sheet(first=0, n1=n1, n2=n2, ds=ds, dw=W / (n2 - 1), seg_of_row=seg_of_row.astype(np.int32))

    h = 1.0 / n
    C0, T0, _, _ = frame(np.zeros(1))
    forcing = Forcing(center=C0[:, 0].copy(), direction=T0[:, 0].copy(), radius=tube_radius,
                      half_len=2.0 * h, amp=amp, omega=2.0 * math.pi * freq)
    centerline = (np.arange(n1) * n2 + n2 // 2).astype(np.int32)
    st = Structure(X0=X0, spring_ij=sij, spring_k=sk, spring_L0=sL0, tether_i=ti, tether_k=tk,
                   sheets=[sheet], bend_b=bend_b, forcing=forcing, normal0=normal0, n_membrane=nbm,
                   centerline=centerline)
    grid = Grid(n=(n, n, nz), h=h, rho=rho, mu=mu, dt=dt)
    u = np.zeros((3, nz, n, n))
    return Problem(name, grid, st, X0.copy(), u)


def with_windows(problem: Problem, n_w: int = 24, half: float = 0.04, radius: float = 0.035,
                 offset: float = 0.06, sep: float = 0.05, k_w: float = 1e4, k_fix: float = 1e6,
                 force_amp: float = 1e-3, freq: float | None = None) -> Problem:
    """The problem plus the oval and round windows (Section 4): two identical
    n_w x n_w square grids of half-width `half` cm, perpendicular to the
    membrane's tangent at its base, `offset` cm before the base and `sep` cm
    to either side of the membrane plane (oval on the +B side).  Grid points
    farther than `radius` from the grid centre are tethered at k_fix (the
    bony rim); every pair of grid neighbours with a free point between them
    is a spring of stiffness k_w and rest length the grid spacing (constant
    compliance).  The oval window's free points carry the external force
    force_amp cos(omega t) along the window normal (the stapes load; omega
    from the problem's tone unless `freq` is given); the round window is
    unforced."""
    st = problem.structure
    m0 = st.m
    C0, T0, er0, B0 = helix_frame(np.zeros(1), _base_z0(problem))
    c0, t0, e0, b0 = C0[:, 0], T0[:, 0], er0[:, 0], B0[:, 0]
    g = np.linspace(-half, half, n_w)
    gu, gv = np.meshgrid(g, g, indexing="ij")                   # (n_w, n_w), u along e_r, v along B
    free = (gu ** 2 + gv ** 2 <= radius ** 2).ravel()
    pts, springs, tethers, forced = [], [], [], []
    for w, side in enumerate((+1.0, -1.0)):                    # oval (+B), round (-B)
        centre = c0 - offset * t0 + side * sep * b0
        P = centre[:, None] + e0[:, None] * gu.ravel()[None, :] + b0[:, None] * gv.ravel()[None, :]
        base = m0 + w * n_w * n_w
        pts.append(P)
        idx = np.arange(n_w * n_w).reshape(n_w, n_w)
        for a_, b_ in ((idx[:-1, :], idx[1:, :]), (idx[:, :-1], idx[:, 1:])):
            a_, b_ = a_.ravel(), b_.ravel()
            keep = free[a_] | free[b_]
            springs.append(np.stack([a_[keep] + base, b_[keep] + base], 1))
        tethers.append(np.nonzero(~free)[0] + base)
        if side > 0:
            forced.append(np.nonzero(free)[0] + base)
    X0 = np.concatenate([st.X0] + pts, axis=1)
    wsij = np.concatenate(springs).astype(np.int32)
    sij = np.concatenate([st.spring_ij, wsij]).astype(np.int32)
    sk = np.concatenate([st.spring_k, np.full(len(wsij), float(k_w))])
    sL0 = np.concatenate([st.spring_L0, np.full(len(wsij), float(g[1] - g[0]))])
    wt = np.concatenate(tethers).astype(np.int32)
    ti = np.concatenate([st.tether_i, wt]).astype(np.int32)
    tk = np.concatenate([st.tether_k, np.full(len(wt), float(k_fix))])
    fi = np.concatenate(forced).astype(np.int32)
    omega = st.forcing.omega if freq is None else 2.0 * math.pi * freq
    mf = MarkerForcing(index=fi, direction=np.repeat(t0[:, None], len(fi), axis=1), amp=force_amp, omega=omega)
    st2 = dataclasses.replace(st, X0=X0, spring_ij=sij, spring_k=sk, spring_L0=sL0, tether_i=ti, tether_k=tk,
                              marker_forcing=mf)
    return dataclasses.replace(problem, name=problem.name + "+windows", structure=st2, X=X0.copy())


def _base_z0(problem: Problem) -> float:
    """Height of the helix start: the first centre-line marker's (its radial
    offset is horizontal)."""
    st = problem.structure
    if st.centerline is not None and len(st.centerline):
        return float(st.X0[2, st.centerline[0]])
    return HELIX_Z0


# ----------------------------------------------------------------------------
# Named workloads (the sizes the project measures and checks on).
# ----------------------------------------------------------------------------
def sphere32() -> Problem:
    """Icosphere shell (2,562 markers, 7,680 springs) on a 32^3 grid, FP64 parity case."""
    return sphere_problem(seed=1, n=32)


# Time step of the cochlea workloads: the paper's own 30 ns (Section 5).  With
# 1e6 dyn/cm tethers on wall markers about h/2 apart, the explicit coupling
# has a collective frequency near sqrt(6.7 k / (rho h^3)): about 3.7e6 1/s at
# h = 1/128 and 1.1e7 1/s at h = 1/256, so 5 us or 2.5 us steps would give
# omega*dt of 19 and 26 (unstable), while 30 ns gives 0.1 and 0.3.
COCHLEA_DT = 3e-8


def cochlea128(seed: int = 2) -> Problem:
    """128^3 grid, 512x48 membrane, 200k wall markers, 1 kHz forcing, dt = 30 ns."""
    return cochlea_problem(seed=seed, n=128, bm=(512, 48), walls=(1000, 200), freq=1000.0,
                           dt=COCHLEA_DT, name="cochlea128")


def cochlea256(seed: int = 3) -> Problem:
    """256^3 grid, 2048x192 membrane + 600k wall markers (993,216) + 20k fibers, 4 kHz, dt = 30 ns."""
    return cochlea_problem(seed=seed, n=256, bm=(2048, 192), walls=(2000, 300), n_fibers=20000,
                           freq=4000.0, dt=COCHLEA_DT, name="cochlea256")


def cochlea128_adjoint(seed: int = 5) -> Problem:
    """The gradient workload: 128^3 grid, 512x48 membrane in 64 stiffness
    segments (graded profile, unperturbed: the target), 200k wall markers,
    1 kHz forcing, dt = 30 ns."""
    return cochlea_problem(seed=seed, n=128, bm=(512, 48), walls=(1000, 200), freq=1000.0,
                           dt=COCHLEA_DT, name="cochlea128_adjoint")


def tone_sweep(seed: int = 4, n_instances: int = 48, f_lo: float = 200.0, f_hi: float = 12000.0) -> list:
    """Independent instances of a tone sweep: grid sizes from {64, 96, 128}^3
    and membranes from {256x24, 512x48}, each chosen per instance from the
    seed; forcing frequencies log-spaced from f_lo to f_hi; 200k tethered
    wall markers, dt = 30 ns and the other parameters of the 128^3 cochlea."""
    grids = (64, 96, 128)
    bms = ((256, 24), (512, 48))
    gi = np.minimum((uniform(seed, 71, n_instances) * len(grids)).astype(int), len(grids) - 1)
    bi = np.minimum((uniform(seed, 72, n_instances) * len(bms)).astype(int), len(bms) - 1)
    freqs = f_lo * (f_hi / f_lo) ** (np.arange(n_instances) / max(1, n_instances - 1))
    out = []
    for i in range(n_instances):
        n = grids[gi[i]]
        out.append(cochlea_problem(seed=seed * 1000 + i, n=n, bm=bms[bi[i]], walls=(1000, 200),
                                   freq=float(freqs[i]), dt=COCHLEA_DT, name=f"tone{i}_{n}"))
    return out


def perturbed_stiffness(problem: Problem, seed: int, scale: float = 0.1) -> np.ndarray:
    """The graded bending stiffness times (1 + scale * xi), xi ~ N(0, 1) per segment."""
    b = np.asarray(problem.structure.bend_b, dtype=np.float64)
    return b * (1.0 + scale * normal(seed, 51, len(b)))


def cochlea_halfcube(seed: int = 6) -> Problem:
    """The paper's production grid shape, 256 x 256 x 128 (one mesh width):
    a 1.75 cm membrane (1.25 turns) of 1024 x 192 markers from z = 0.11 cm,
    1000 x 300 wall markers, 10,000 fibers, 4 kHz, dt = 30 ns."""
    return cochlea_problem(seed=seed, n=256, nz=128, bm=(1024, 192), walls=(1000, 300), n_fibers=10000,
                           freq=4000.0, dt=COCHLEA_DT, length=1.75, z0=0.11, name="cochlea_halfcube")


# The paper's half-cube model (Section 4): packed into 1 cm x 1 cm x 0.5 cm,
# its membrane flat (the spiral lies in one plane), 256 x 256 x 128 points.
HALFCUBE_FLAT_WIDTHS = (0.015, 0.056)   # cm: about 150 um at the stapes to 560 um at the helicotrema
HALFCUBE_FLAT_TUBE = 0.05               # cm: turns of the flat spiral lie 0.114 cm apart


def cochlea_halfcube_flat(seed: int = 9) -> Problem:
    """The paper's half-cube shape: 256 x 256 x 128 grid, a flat 3.5 cm
    membrane of 2048 x 192 markers on a 2.5-turn planar spiral in the plane
    z = 0.25 cm, width 0.015 -> 0.056 cm, 2000 x 160 wall markers on a tube of
    radius 0.05 cm (713,216 markers), 20,000 fibers, 4 kHz, dt = 30 ns."""
    return cochlea_problem(seed=seed, n=256, nz=128, bm=(2048, 192), walls=(2000, 160), n_fibers=20000,
                           freq=4000.0, dt=COCHLEA_DT, name="cochlea_halfcube_flat",
                           frame=lambda s_: flat_spiral_frame(s_, BM_LENGTH, z0=0.25),
                           widths=HALFCUBE_FLAT_WIDTHS, tube_radius=HALFCUBE_FLAT_TUBE)


def cochlea_windows(seed: int = 8, n: int = 128) -> Problem:
    """The 128^3 cochlea with its oval and round windows (48 x 48 grids,
    the oval one driven by a 1 kHz normal load)."""
    p = cochlea_problem(seed=seed, n=n, bm=(512, 48), walls=(1000, 200), freq=1000.0, dt=COCHLEA_DT,
                        name=f"cochlea{n}")
    return with_windows(p, n_w=48)


def cochlea_small(seed: int = 7, n: int = 32, bm=(64, 12), walls=(120, 40), n_fibers: int = 64,
                  freq: float = 2000.0, dt: float = 2.5e-6) -> Problem:
    """A scaled-down cochlea for parity tests that the oracle finishes in seconds."""
    return cochlea_problem(seed=seed, n=n, bm=bm, walls=walls, n_fibers=n_fibers, freq=freq,
                           dt=dt, n_seg=8, name=f"cochlea{n}")


def membrane_bump(problem: Problem, amplitude: float = 1e-4, k: int = 3) -> np.ndarray:
    """(3, m) displacement: the membrane pushed along its rest normal by
    amplitude * sin(k pi s / L) (s the arclength), everything else at rest."""
    st = problem.structure
    sh = st.sheets[0]
    D = np.zeros_like(st.X0)
    s = np.repeat(np.arange(sh.n1) / (sh.n1 - 1), sh.n2)
    M = st.n_membrane
    D[:, :M] = amplitude * np.sin(k * math.pi * s)[None, :] * st.normal0[:, :M]
    return D


def with_bend_scale(problem: Problem, scale: float) -> Problem:
    """The same problem with every segment's bending stiffness times scale."""
    st = dataclasses.replace(problem.structure, bend_b=np.asarray(problem.structure.bend_b) * scale)
    return dataclasses.replace(problem, structure=st)


# ----------------------------------------------------------------------------
# Random fields and marker clouds for unit-level parity cases.
# ----------------------------------------------------------------------------
def random_velocity(seed: int, n, amp: float = 1.0, modes: int = 6, noise: float = 0.0) -> np.ndarray:
    """(3, nz, ny, nx) field: a few random Fourier modes plus optional white noise."""
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    kk = np.floor(uniform(seed, 31, 9 * modes, -3, 4)).astype(int).reshape(3, modes, 3)
    ph = uniform(seed, 32, 3 * modes, 0, 2 * math.pi).reshape(3, modes)
    am = normal(seed, 33, 3 * modes).reshape(3, modes)
    for c in range(3):
        for q in range(modes):
            kx, ky, kz = kk[c, q]
            u[c] += am[c, q] * np.cos(2 * math.pi * (kx * x + ky * y + kz * z) + ph[c, q])
    if noise:
        u += noise * normal(seed, 34, u.size).reshape(u.shape)
    return amp * u


def random_markers(seed: int, m: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """(3, m) positions uniform in [lo, hi)^3."""
    return uniform(seed, 41, 3 * m, lo, hi).reshape(3, m)


def random_forces(seed: int, m: int) -> np.ndarray:
    return normal(seed, 42, 3 * m).reshape(3, m)
