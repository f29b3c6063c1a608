"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
values of the delta kernel, brute-force sums with no stencil logic, a dense
direct solve of the discrete Navier-Stokes system built from the difference
operators' definitions, exact decay factors, invariants (total force,
adjointness, divergence, mean mode), hand-computed force values and library
routines (numpy's FFT and stable argsort).  The cases are chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_math_0301321_gb300 import synth


class G:
    """Minimal grid description."""

    def __init__(self, n, h=None, rho=1.0, mu=0.02, dt=1e-5):
        self.n = tuple(n)
        self.h = (1.0 / n[0]) if h is None else h
        self.rho, self.mu, self.dt = rho, mu, dt


# ----------------------------------------------------------------------------
# phi (Section 3.2, definition of delta_h)
# ----------------------------------------------------------------------------
def test_phi_closed_values():
    # phi(0) = (3 + 1)/8; phi(1) = (3 - 2 + 1)/8; phi(2) = 1/2 - phi(0);
    # phi(1/2) = (3 - 1 + sqrt(2))/8; phi(3/2) = 1/2 - phi(1/2); |r| >= 2 -> 0.
    cases = {0.0: 0.5, 1.0: 0.25, -1.0: 0.25, 2.0: 0.0, -2.0: 0.0, 0.5: (2 + math.sqrt(2)) / 8,
             -0.5: (2 + math.sqrt(2)) / 8, 1.5: (2 - math.sqrt(2)) / 8, -1.5: (2 - math.sqrt(2)) / 8,
             2.5: 0.0, -3.0: 0.0}
    for r, v in cases.items():
        assert abs(oracle.phi(r) - v) <= 1e-16, (r, oracle.phi(r), v)


def test_phi_moment_identities():
    # Properties of Peskin's construction: partition of unity, zero first moment,
    # sum of squares 3/8, even and odd sums 1/2 each, for every shift r.
    r = np.linspace(0.0, 1.0, 10001)[:-1]
    j = np.arange(-3, 4)
    P = oracle.phi(r[:, None] - j[None, :])
    assert np.abs(P.sum(1) - 1.0).max() < 1e-15
    assert np.abs(((r[:, None] - j[None, :]) * P).sum(1)).max() < 1e-15
    assert np.abs((P ** 2).sum(1) - 0.375).max() < 1e-15
    assert np.abs(P[:, (j % 2) == 0].sum(1) - 0.5).max() < 1e-15
    assert np.abs(P[:, (j % 2) == 1].sum(1) - 0.5).max() < 1e-15
    # continuity at |r| = 1 from both branches, and support [-2, 2]
    assert abs(oracle.phi(1.0 - 1e-12) - oracle.phi(1.0 + 1e-12)) < 1e-11
    assert oracle.phi(2.0 + 1e-12) == 0.0


# ----------------------------------------------------------------------------
# Spreading and interpolation (Eqs. discreteF, discreteX)
# ----------------------------------------------------------------------------
def _brute_spread(g, X, f):
    """F at every node as a sum over 27 periodic images of f delta_h, no stencil."""
    nx, ny, nz = g.n
    h = g.h
    L = np.array([nx * h, ny * h, nz * h])
    F = np.zeros((3, nz, ny, nx))
    idx = [np.arange(nx), np.arange(ny), np.arange(nz)]
    for l in range(X.shape[1]):
        for img in np.ndindex(3, 3, 3):
            shift = (np.array(img) - 1) * L
            w = [oracle.phi((h * idx[a] - X[a, l] - shift[a]) / h) for a in range(3)]
            d = w[2][:, None, None] * w[1][None, :, None] * w[0][None, None, :] / h ** 3
            for c in range(3):
                F[c] += f[c, l] * d
    return F


@pytest.mark.parametrize("n", [(8, 8, 8), (8, 12, 10)])
def test_spread_matches_bruteforce(n):
    g = G(n, h=1.0 / 8)
    L = np.array(n) / 8.0
    X = synth.random_markers(5, 8) * L[:, None]
    X[:, 0] = [0.0, 0.0, 0.0]                        # a marker exactly on a node
    X[:, 1] = [L[0] - 1e-13, 0.5 * L[1], 1e-13]      # on the periodic seam
    f = synth.random_forces(6, 8)
    F = oracle.spread(g, X, f)
    Fb = _brute_spread(g, X, f)
    assert np.abs(F - Fb).max() <= 1e-13 * np.abs(Fb).max()


def test_spread_conserves_total_force():
    g = G((16, 16, 16))
    X = synth.random_markers(7, 200)
    f = synth.random_forces(8, 200)
    F = oracle.spread(g, X, f)
    tot = F.reshape(3, -1).sum(1) * g.h ** 3
    assert np.abs(tot - f.sum(1)).max() <= 1e-13 * np.abs(f).sum()


def test_interp_constant_and_linear_fields():
    g = G((16, 16, 16))
    X = synth.random_markers(9, 100, 0.3, 0.7)       # stencils never wrap
    h = g.h
    z, y, x = np.meshgrid(np.arange(16) * h, np.arange(16) * h, np.arange(16) * h, indexing="ij")
    u = np.stack([np.full_like(x, 2.5), 1.0 + 3.0 * x, -2.0 + 0.5 * y - 4.0 * z])
    U = oracle.interp(g, X, u)
    assert np.abs(U[0] - 2.5).max() < 1e-14
    assert np.abs(U[1] - (1.0 + 3.0 * X[0])).max() < 1e-14
    assert np.abs(U[2] - (-2.0 + 0.5 * X[1] - 4.0 * X[2])).max() < 1e-14


@pytest.mark.parametrize("n", [(16, 16, 16), (12, 8, 20)])
def test_spread_interp_adjoint(n):
    g = G(n, h=1.0 / 16)
    L = np.array(n) / 16.0
    X = synth.random_markers(10, 300) * L[:, None]
    f = synth.random_forces(11, 300)
    u = synth.random_velocity(12, n, noise=1.0)
    lhs = (oracle.spread(g, X, f) * u).sum() * g.h ** 3
    rhs = (f * oracle.interp(g, X, u)).sum()
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(f).sum() * np.abs(u).max())


def test_bin_sort_matches_stable_argsort():
    g = G((16, 12, 8), h=1.0 / 16)
    X = synth.random_markers(13, 2000) * (np.array([16, 12, 8]) / 16.0)[:, None]
    X[:, :50] = X[:, 50:100]                          # duplicate keys
    X[0, 100:110] = -0.01                             # negative coordinates wrap
    key, perm = oracle.bin_sort(g, X)
    b = np.floor(X * (1.0 / g.h)).astype(np.int64)
    i, j, k = b[0] % 16, b[1] % 12, b[2] % 8
    # tiles of 8^3 cells (2 x 2 x 1 tiles here), tile-major then cell order
    tile = ((k // 8) * 2 + j // 8) * 2 + i // 8
    kk = tile * 512 + ((k % 8) * 8 + j % 8) * 8 + i % 8
    assert np.array_equal(key, kk)
    assert np.array_equal(perm, np.argsort(kk // 512, kind="stable"))


# ----------------------------------------------------------------------------
# The DFT used by the fluid solve
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 12, 16, 30, 32])
def test_dft1_matches_naive_sum(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    naive = np.array([np.sum(a * np.exp(-2j * np.pi * ((j * k) % n) / n)) for k in range(n)])
    assert np.abs(oracle.dft1(a, -1) - naive).max() <= 1e-14 * max(1.0, np.abs(naive).max())
    naive_inv = np.array([np.sum(a * np.exp(2j * np.pi * ((j * k) % n) / n)) for k in range(n)])
    assert np.abs(oracle.dft1(a, +1) - naive_inv).max() <= 1e-14 * max(1.0, np.abs(naive_inv).max())


@pytest.mark.parametrize("n", [(8, 8, 8), (12, 6, 10), (96, 4, 4)])
def test_dft3_matches_numpy_and_parseval(n):
    g = G(n)
    rng = np.random.default_rng(1)
    a = rng.standard_normal(n[::-1]) + 1j * rng.standard_normal(n[::-1])
    A = oracle.dft3(g, a, -1)
    assert np.abs(A - np.fft.fftn(a)).max() <= 1e-13 * np.abs(A).max()
    assert abs((np.abs(A) ** 2).sum() / a.size - (np.abs(a) ** 2).sum()) <= 1e-12 * (np.abs(a) ** 2).sum()
    back = oracle.dft3(g, A, +1) / a.size
    assert np.abs(back - a).max() <= 1e-13


# ----------------------------------------------------------------------------
# The fluid solve (Eqs. discreteNS1-2)
# ----------------------------------------------------------------------------
def _shift(n, axis, d):
    """Dense matrix of u -> u(c + d e_axis) on a periodic (nz, ny, nx) grid."""
    nx, ny, nz = n
    Gn = nx * ny * nz
    S = np.zeros((Gn, Gn))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                src = [i, j, k]
                src[axis] = (src[axis] + d) % n[axis]
                S[(k * ny + j) * nx + i, (src[2] * ny + src[1]) * nx + src[0]] = 1.0
    return S


@pytest.mark.parametrize("n", [(4, 4, 4), (6, 6, 6), (4, 6, 8)])
def test_solve_equals_dense_direct_solve(n):
    # The linear system of Eqs. (discreteNS1)-(discreteNS2), assembled from the
    # definitions of D+, D-, D0 (Eqs. differenceOpsFirst..Last) and solved by
    # least squares: the velocity is unique even though p is not.
    g = G(n, h=0.1, rho=1.3, mu=0.7, dt=0.05)
    nx, ny, nz = n
    Gn = nx * ny * nz
    I = np.eye(Gn)
    Dp = [(_shift(n, a, 1) - I) / g.h for a in range(3)]
    Dm = [(I - _shift(n, a, -1)) / g.h for a in range(3)]
    D0 = [(_shift(n, a, 1) - _shift(n, a, -1)) / (2 * g.h) for a in range(3)]
    Lap = sum(Dp[a] @ Dm[a] for a in range(3))
    A = np.zeros((4 * Gn, 4 * Gn))
    for c in range(3):
        A[c * Gn:(c + 1) * Gn, c * Gn:(c + 1) * Gn] = g.rho / g.dt * I - g.mu * Lap
        A[c * Gn:(c + 1) * Gn, 3 * Gn:] = D0[c]
        A[3 * Gn:, c * Gn:(c + 1) * Gn] = D0[c]
    w = synth.random_velocity(3, n, noise=1.0)
    b = np.concatenate([w.reshape(3, -1).ravel(), np.zeros(Gn)])
    sol = np.linalg.lstsq(A, b, rcond=None)[0]
    un, p = oracle.solve(g, w, want_p=True)
    assert np.abs(un.ravel() - sol[:3 * Gn]).max() <= 1e-11 * np.abs(sol[:3 * Gn]).max()
    # the oracle's pressure satisfies the momentum equation with its velocity
    res = A[:3 * Gn] @ np.concatenate([un.ravel(), p.ravel()]) - b[:3 * Gn]
    assert np.abs(res).max() <= 1e-10 * np.abs(b).max()


def _div0(u, h):
    return sum((np.roll(u[c], -1, axis=2 - c) - np.roll(u[c], 1, axis=2 - c)) / (2 * h) for c in range(3))


def test_solve_is_discretely_divergence_free():
    g = G((16, 16, 16), dt=1e-4)
    u = synth.random_velocity(4, g.n, noise=1.0)
    F = synth.random_velocity(5, g.n, amp=100.0, noise=1.0)
    un = oracle.fluid_solve(g, u, F)
    assert np.abs(_div0(un, g.h)).max() <= 1e-13 * np.abs(un).max() / g.h


@pytest.mark.parametrize("k", [1, 3, 7])
def test_shear_mode_decays_by_exact_factor(k):
    # u = sin(2 pi k y) e_x has zero advection (u_x is constant along x and
    # u_y = u_z = 0) and zero divergence, so one step multiplies it by
    # 1 / (1 + (mu dt / rho)(4/h^2) sin^2(pi k / N)).
    n = 16
    g = G((n, n, n), rho=1.0, mu=0.5, dt=1e-3)
    y = np.arange(n) * g.h
    u = np.zeros((3, n, n, n))
    u[0] = np.sin(2 * math.pi * k * y)[None, :, None]
    un = oracle.fluid_solve(g, u, np.zeros_like(u))
    fac = 1.0 / (1.0 + g.mu * g.dt / g.rho * 4.0 / g.h ** 2 * math.sin(math.pi * k / n) ** 2)
    assert np.abs(un[0] - fac * u[0]).max() < 1e-14
    assert np.abs(un[1:]).max() < 1e-14


def test_shear_mode_converges_to_continuum_decay():
    # The continuum shear wave u = sin(2 pi k y) e_x decays as
    # exp(-(mu/rho)(2 pi k)^2 t).  Backward Euler in time and the 7-point
    # Laplacian in space err by O(dt + h^2): halving h and quartering dt
    # divides the error at a fixed time by about 4.
    k, T = 1, 0.02
    nu = 0.5
    errs = []
    for n, steps in ((16, 10), (32, 40)):
        g = G((n, n, n), rho=1.0, mu=nu, dt=T / steps)
        y = np.arange(n) * g.h
        u = np.zeros((3, n, n, n))
        u[0] = np.sin(2 * math.pi * k * y)[None, :, None]
        amp0 = u[0, 0, :, 0].copy()
        for _ in range(steps):
            u = oracle.fluid_solve(g, u, np.zeros_like(u))
        j = n // 4                       # y = 1/4, where sin = 1
        amp = u[0, 0, j, 0] / amp0[j]
        errs.append(abs(amp - math.exp(-nu * (2 * math.pi * k) ** 2 * T)))
    assert errs[0] < 1e-2
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_mean_mode_update():
    # The k = 0 mode: mean(u') = mean(u) + (dt/rho)(mean(F) - rho mean(A(u))).
    g = G((8, 8, 8), rho=1.2, mu=0.1, dt=1e-3)
    u = synth.random_velocity(6, g.n, noise=1.0)
    F = synth.random_velocity(7, g.n, amp=10.0, noise=1.0) + 3.0
    un = oracle.fluid_solve(g, u, F)
    A = oracle.advection(g, u)
    want = u.mean((1, 2, 3)) + g.dt / g.rho * (F.mean((1, 2, 3)) - g.rho * A.mean((1, 2, 3)))
    assert np.abs(un.mean((1, 2, 3)) - want).max() < 1e-13


def test_upwind_advection_hand_values():
    # 4^3 grid, h = 1/4.  u_x = i + 1 (i = x index), so D^- u_x = 4 except at
    # the periodic seam i = 0 where it is (1 - 4) * 4 = -12.
    g = G((4, 4, 4), h=0.25)
    i = np.arange(4)[None, None, :] * np.ones((4, 4, 4))
    u = np.zeros((3, 4, 4, 4))
    u[0] = i + 1.0
    A = oracle.advection(g, u)
    assert A[0, 0, 0, 2] == 3.0 * 4.0            # u_x = 3 > 0: 3 * (3 - 2) * 4
    assert A[0, 0, 0, 0] == 1.0 * (-12.0)        # wraps: 1 * (1 - 4) * 4
    assert np.all(A[1:] == 0.0)
    # reversed flow picks D^+: u_x = -(i + 1)
    u[0] = -(i + 1.0)
    A = oracle.advection(g, u)
    assert A[0, 0, 0, 2] == -3.0 * ((-4.0) - (-3.0)) * 4.0   # = 12
    assert A[0, 0, 0, 3] == -4.0 * ((-1.0) - (-4.0)) * 4.0   # wraps: = -48
    # u_y advected by u_x = 1: A_y = 1 * D_x^- u_y; u_y is constant along y
    u[0] = 1.0
    u[1] = i + 1.0
    A = oracle.advection(g, u)
    assert A[1, 0, 0, 2] == 4.0 and A[1, 0, 0, 0] == -12.0
    assert np.all(A[0] == 0.0)
    # a zero velocity component contributes nothing even across a jump
    u = np.zeros((3, 4, 4, 4))
    u[2] = np.arange(4)[:, None, None] * np.ones((4, 4, 4))   # u_z = k
    A = oracle.advection(g, u)
    assert A[2, 0, 0, 0] == 0.0                   # u_z = 0 at k = 0
    assert A[2, 2, 0, 0] == 2.0 * (2.0 - 1.0) * 4.0


@pytest.mark.parametrize("n", [(6, 5, 4), (8, 8, 8)])
def test_upwind_advection_identities_on_general_fields(n):
    """The upwind term of Eq. (discreteNS1) on random fields of both signs.
    Flipping the velocity swaps every upwind choice, so
      A(u) + A(-u) = sum_d u_d (u_c(+e_d) - u_c(-e_d)) / h      (centred)
      A(u) - A(-u) = sum_d |u_d| (2 u_c - u_c(+e_d) - u_c(-e_d)) / h
    and A is homogeneous of degree 2 (scaling by 2 is exact in binary).
    The right-hand sides are formed with periodic shifts, independently of
    the oracle's branch logic: a wrong branch, sign, axis or shift fails."""
    g = G(n, h=0.125)
    u = synth.random_velocity(41, g.n, noise=1.0) - 0.3
    u[:, 1, 2, 3] = 0.0                      # exact zeros take neither branch
    Ap, Am = oracle.advection(g, u), oracle.advection(g, -u)
    cen = np.zeros_like(u)
    dif = np.zeros_like(u)
    for d, ax in ((0, 3), (1, 2), (2, 1)):   # x, y, z are the last three axes of [c][z][y][x]
        up = np.roll(u, -1, axis=ax)          # u(+e_d)
        dn = np.roll(u, 1, axis=ax)           # u(-e_d)
        cen += u[d] * (up - dn) / g.h
        dif += np.abs(u[d]) * (2 * u - up - dn) / g.h
    scale = np.abs(cen).max() + np.abs(dif).max()
    assert np.abs((Ap + Am) - cen).max() <= 1e-13 * scale
    assert np.abs((Ap - Am) - dif).max() <= 1e-13 * scale
    assert np.array_equal(oracle.advection(g, 2 * u), 4 * Ap)


# ----------------------------------------------------------------------------
# Marker forces
# ----------------------------------------------------------------------------
def _one_structure(X0, springs=(), tethers=(), sheet=None, bend_b=()):
    st = synth._empty_structure(np.asarray(X0, float))
    if springs:
        st.spring_ij = np.array([s[:2] for s in springs], np.int32)
        st.spring_k = np.array([s[2] for s in springs], float)
        st.spring_L0 = np.array([s[3] for s in springs], float)
    if tethers:
        st.tether_i = np.array([t[0] for t in tethers], np.int32)
        st.tether_k = np.array([t[1] for t in tethers], float)
    if sheet is not None:
        st.sheets = [sheet]
        st.bend_b = np.array(bend_b, float)
    return st


def test_force_hand_values():
    # spring: d = (0.03, 0.04, 0), r = 0.05, L0 = 0.04, k = 100 -> 100*0.01*(0.6, 0.8, 0)
    X = np.array([[0.0, 0.03], [0.0, 0.04], [0.0, 0.0]])
    st = oracle.Structure(_one_structure(X, springs=[(0, 1, 100.0, 0.04)]))
    D = np.zeros_like(X)
    f = oracle.forces(st, D)
    assert np.allclose(f[:, 0], [0.6, 0.8, 0.0], rtol=0, atol=1e-15)
    assert np.allclose(f[:, 1], [-0.6, -0.8, 0.0], rtol=0, atol=1e-15)
    assert abs(oracle.energy(st, D) - 0.5 * 100 * 0.01 ** 2) < 1e-14 * 0.005
    # the same spring reached by displacing marker 1 from (0.03, 0, 0)
    X0 = np.array([[0.0, 0.03], [0.0, 0.0], [0.0, 0.0]])
    st = oracle.Structure(_one_structure(X0, springs=[(0, 1, 100.0, 0.04)]))
    f = oracle.forces(st, np.array([[0.0, 0.0], [0.0, 0.04], [0.0, 0.0]]))
    assert np.allclose(f[:, 1], [-0.6, -0.8, 0.0], rtol=0, atol=1e-15)
    # tether: X - X0 = (1e-3, -2e-3, 0), k = 1e6
    X0 = np.array([[0.5], [0.5], [0.5]])
    st = oracle.Structure(_one_structure(X0, tethers=[(0, 1e6)]))
    f = oracle.forces(st, np.array([[1e-3], [-2e-3], [0.0]]))
    assert np.allclose(f[:, 0], [-1000.0, 2000.0, 0.0], rtol=1e-12, atol=0)
    # bending: three markers on a line (n1 = 3, n2 = 1), middle one moved by
    # delta in y: v - v0 = (0, -2 delta, 0); c = b dw / ds^3 = 2*0.5/0.001 = 1000
    ds = 0.1
    X0 = np.array([[0.0, ds, 2 * ds], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    sh = synth.Sheet(first=0, n1=3, n2=1, ds=ds, dw=np.array([0.5, 0.5, 0.5]), seg_of_row=np.zeros(3, np.int32))
    st = oracle.Structure(_one_structure(X0, sheet=sh, bend_b=[2.0]))
    D = np.zeros_like(X0)
    D[1, 1] = 1e-3
    f = oracle.forces(st, D)
    assert np.allclose(f[1], [2.0, -4.0, 2.0], rtol=1e-12, atol=0)
    assert np.abs(f[[0, 2]]).max() == 0.0
    assert abs(oracle.energy(st, D) - 0.5 * 1000 * (2e-3) ** 2) < 1e-15


def test_forces_are_energy_gradient_and_balanced():
    p = synth.cochlea_small()
    st = oracle.Structure(p.structure)
    X = 1e-3 * synth.random_forces(14, p.structure.m)        # displacement from X0
    f = oracle.forces(st, X)
    rng = np.random.default_rng(0)
    for _ in range(12):
        c, l = rng.integers(3), rng.integers(X.shape[1])
        eps = 1e-6
        Xp, Xm = X.copy(), X.copy()
        Xp[c, l] += eps
        Xm[c, l] -= eps
        fd = -(oracle.energy(st, Xp) - oracle.energy(st, Xm)) / (2 * eps)
        assert abs(fd - f[c, l]) <= 1e-6 * max(1.0, abs(f[c, l])), (c, l, fd, f[c, l])
    # internal forces (springs + bending) sum to zero; tethers excluded
    st_int = synth._empty_structure(p.structure.X0)
    st_int.spring_ij, st_int.spring_k, st_int.spring_L0 = (p.structure.spring_ij, p.structure.spring_k,
                                                           p.structure.spring_L0)
    st_int.sheets, st_int.bend_b = p.structure.sheets, p.structure.bend_b
    fi = oracle.forces(oracle.Structure(st_int), X)
    assert np.abs(fi.sum(1)).max() <= 1e-12 * np.abs(fi).sum()
    # and they depend on position differences only: a rigid translation of
    # the whole structure leaves them unchanged
    shift = np.array([0.013, -0.021, 0.0047])[:, None]
    ft = oracle.forces(oracle.Structure(st_int), X + shift)
    assert np.abs(ft - fi).max() <= 1e-9 * np.abs(fi).max()
    # zero at rest
    f0 = oracle.forces(st, np.zeros_like(p.structure.X0))
    assert np.abs(f0).max() <= 1e-9


def test_body_force_region():
    p = synth.cochlea_small()
    g, fo = p.grid, p.structure.forcing
    st = oracle.Structure(p.structure)
    F = oracle.body_force(g, st, 0.0)
    mag = g.rho * fo.amp * fo.omega
    nz_ = np.abs(F[0]) + np.abs(F[1]) + np.abs(F[2]) > 0
    assert nz_.sum() > 0
    h = g.h
    for (k, j, i) in zip(*np.nonzero(nz_)):
        d = h * np.array([i, j, k]) - fo.center
        along = d @ fo.direction
        assert abs(along) <= fo.half_len + 1e-15
        assert d @ d - along ** 2 <= fo.radius ** 2 + 1e-15
        assert np.allclose(F[:, k, j, i], mag * fo.direction, rtol=1e-14)
    # a quarter period later cos(omega t) = 0
    F2 = oracle.body_force(g, st, math.pi / (2 * fo.omega))
    assert np.abs(F2).max() <= 1e-12 * mag


# ----------------------------------------------------------------------------
# Whole-step invariants
# ----------------------------------------------------------------------------
def _volume(X, faces):
    a, b, c = X[:, faces[:, 0]], X[:, faces[:, 1]], X[:, faces[:, 2]]
    return float(np.einsum("ij,ij->j", a, np.cross(b.T, c.T).T).sum() / 6.0)


def test_sphere_volume_drift_small_and_shrinks_with_h():
    # Volume conservation (Section 3.3: material mesh about half the fluid mesh
    # width keeps fluid from leaking).  The enclosed volume drifts little, and
    # refining fluid and material meshes together (32^3 with the level-4
    # sphere, 64^3 with level 5) lowers the drift per unit of displacement.
    drift = {}
    for n, level in ((32, 4), (64, 5)):
        p = synth.sphere_problem(seed=1, n=n, level=level)
        st = oracle.Structure(p.structure)
        v0 = _volume(p.X, p.structure.faces)
        D, u, t = oracle.step(p.grid, st, np.zeros_like(p.X), p.u, 0.0, 10)
        X = p.structure.X0 + D
        moved = np.abs(D).max()
        assert moved > 1e-4                            # the shell moves
        drift[n] = abs(_volume(X, p.structure.faces) - v0) / v0 / moved
    assert drift[32] < 2e-2
    assert drift[64] < drift[32]


def test_stokes_mean_velocity_stays_zero():
    p = synth.sphere32()
    st = oracle.Structure(p.structure)
    D, u, t = oracle.step(p.grid, st, np.zeros_like(p.X), p.u, 0.0, 5, no_advection=True)
    assert np.abs(u).max() > 1e-3
    assert np.abs(u.mean((1, 2, 3))).max() <= 1e-13 * np.abs(u).max()


def test_response_is_linear_in_forcing():
    # Linear regime of the passive model: 10x forcing gives 10x displacement.
    disp = []
    for amp in (1e-4, 1e-3):
        p = synth.cochlea_problem(seed=7, n=32, bm=(64, 12), walls=(120, 40), n_seg=8, amp=amp,
                                  freq=2000.0, dt=2.5e-6)
        st = oracle.Structure(p.structure)
        D, u, t = oracle.step(p.grid, st, np.zeros_like(p.X), p.u, 0.0, 10, no_advection=True)
        disp.append(D)
    ratio = np.linalg.norm(disp[1]) / np.linalg.norm(disp[0])
    assert abs(ratio - 10.0) < 1e-2
    assert np.linalg.norm(disp[1] - 10 * disp[0]) <= 1e-3 * np.linalg.norm(disp[1])


def test_step_time_levels():
    # Section 3.2 steps 3-4: u^{n+1} is solved first, then interpolated at the
    # OLD positions X^n.  With no elastic links, no forcing and no advection,
    # u = A (sin 2 pi y, sin 2 pi x, 0) is divergence free and decays by the
    # exact factor of its wavenumber, so X^1 = X^0 + dt * interp(fac u^0, X^0).
    n = 16
    g = G((n, n, n), rho=1.0, mu=0.3, dt=2e-3)
    h = g.h
    z, y, x = np.meshgrid(np.arange(n) * h, np.arange(n) * h, np.arange(n) * h, indexing="ij")
    u0 = np.stack([np.sin(2 * math.pi * y), np.sin(2 * math.pi * x), np.zeros_like(x)]) * 5.0
    X0 = synth.random_markers(17, 40)
    st = oracle.Structure(synth._empty_structure(X0.copy()))
    D1, u1, t1 = oracle.step(g, st, np.zeros_like(X0), u0, 0.0, 1, no_advection=True)
    X1 = X0 + D1
    fac = 1.0 / (1.0 + g.mu * g.dt / g.rho * 4.0 / h ** 2 * math.sin(math.pi / n) ** 2)
    assert np.abs(u1 - fac * u0).max() < 1e-13
    assert np.abs(D1 - g.dt * oracle.interp(g, X0, fac * u0)).max() < 1e-15
    # interpolating at the new positions instead would be off by O(dt^2 |grad u| |u|)
    wrong = X0 + g.dt * oracle.interp(g, X1, fac * u0)
    assert np.abs(X1 - wrong).max() > 1e-6
    assert abs(t1 - g.dt) < 1e-18
