"""Pins of the oracle's reverse time step (CPU only).

The adjoint oracle is the transpose of the linearised forward step.  Each
building block is pinned to what fixes it independently of its own code:
phi' to the moment identities that follow from differentiating phi's
partition of unity, first moment and sum of squares (Section 3.2, definition of
delta_h), and every transpose to central finite differences of the pinned
FORWARD oracle (a directional derivative <lam, J dv> must equal <J^T lam, dv>).
The whole reverse step is checked the same way against one and two forward
steps, with and without advection, so a dropped term, a wrong sign, a wrong
1/h^3 or a transposed operand fails.
"""
import numpy as np
import pytest

import oracle
from paper_math_0301321_gb300 import synth


def _rng(seed):
    return np.random.default_rng(seed)


def _bounded_velocity(g, rng, scale=1.0):
    """Velocity whose components stay at least 0.5*scale away from zero, so
    that no upwind branch switches inside a finite-difference stencil."""
    nx, ny, nz = g.n
    mag = 0.5 + 0.5 * rng.random((3, nz, ny, nx))
    sign = np.where(rng.random((3, nz, ny, nx)) < 0.5, -1.0, 1.0)
    return scale * mag * sign


# ---------------------------------------------------------------------------
# phi'
# ---------------------------------------------------------------------------
def test_phi_d_moment_identities():
    """d/dr of sum_i phi(r-i) = 1, sum_i (r-i) phi(r-i) = 0 and
    sum_i phi(r-i)^2 = 3/8 give sum phi' = 0, sum (r-i) phi' = -1 and
    sum phi phi' = 0 at every r."""
    for r in np.linspace(0.0, 1.0, 41):
        d = r - np.arange(-3, 5)
        pd = oracle.phi_d(d)
        p = oracle.phi(d)
        assert abs(pd.sum()) < 1e-14
        assert abs((d * pd).sum() + 1.0) < 1e-14
        assert abs((p * pd).sum()) < 1e-14


def test_phi_d_closed_values_and_fd():
    # phi'(r) = (-2 + (2 - 4|r|)/sqrt(1 + 4|r| - 4 r^2)) sign(r) / 8 on |r| <= 1
    assert oracle.phi_d(0.0) == 0.0
    assert abs(oracle.phi_d(0.5) + 0.25) < 1e-16
    assert abs(oracle.phi_d(1.0) + 0.5) < 1e-16
    assert abs(oracle.phi_d(-1.5) - 0.25) < 1e-16
    assert oracle.phi_d(2.0) == 0.0 and oracle.phi_d(2.5) == 0.0
    r = np.linspace(-2.4, 2.4, 963)
    eps = 1e-6
    fd = (oracle.phi(r + eps) - oracle.phi(r - eps)) / (2 * eps)
    assert np.max(np.abs(fd - oracle.phi_d(r))) < 1e-6   # O(eps) at the kinks of phi''


# ---------------------------------------------------------------------------
# building blocks against finite differences of the forward oracle
# ---------------------------------------------------------------------------
def test_interp_grad_is_derivative_of_interp():
    g = synth.Grid(n=(8, 6, 10), h=0.125, rho=1.0, mu=0.02, dt=1e-4)
    rng = _rng(11)
    m = 40
    X = rng.random((3, m)) * np.array([[1.0], [0.75], [1.25]])
    u = rng.standard_normal((3, 10, 6, 8))
    v = rng.standard_normal((3, m))
    dX = rng.standard_normal((3, m))
    eps = 1e-6 * g.h
    fd = ((oracle.interp(g, X + eps * dX, u) - oracle.interp(g, X - eps * dX, u)) / (2 * eps) * v).sum()
    an = (oracle.interp_grad(g, X, u, v) * dX).sum()
    assert abs(fd - an) < 1e-7 * abs(an)
    # the scale argument multiplies and the result accumulates into out
    an2 = (oracle.interp_grad(g, X, u, v, scale=-2.5) * dX).sum()
    assert abs(an2 + 2.5 * an) < 1e-12 * abs(an)


def test_spread_derivative_via_interp_grad():
    """d/dX <lam, S(X) f> = h^-3 interp_grad(lam, f): the spreading half of
    the position sensitivity uses the same kernel as interpolation."""
    g = synth.Grid(n=(8, 8, 8), h=0.125, rho=1.0, mu=0.02, dt=1e-4)
    rng = _rng(12)
    m = 25
    X = rng.random((3, m))
    f = rng.standard_normal((3, m))
    lam = rng.standard_normal((3, 8, 8, 8))
    dX = rng.standard_normal((3, m))
    eps = 1e-6 * g.h
    fd = ((oracle.spread(g, X + eps * dX, f) - oracle.spread(g, X - eps * dX, f)) * lam).sum() / (2 * eps)
    an = (oracle.interp_grad(g, X, lam, f, scale=g.h ** -3) * dX).sum()
    assert abs(fd - an) < 1e-7 * abs(an)


def test_advection_adjoint_transposes_linearisation():
    g = synth.Grid(n=(6, 8, 10), h=0.1, rho=1.0, mu=0.02, dt=1e-4)
    rng = _rng(13)
    u = _bounded_velocity(g, rng)
    du = rng.standard_normal(u.shape)
    lam = rng.standard_normal(u.shape)
    eps = 1e-4          # the upwind term is quadratic between sign switches
    jvp = (oracle.advection(g, u + eps * du) - oracle.advection(g, u - eps * du)) / (2 * eps)
    lhs = (lam * jvp).sum()
    rhs = (oracle.advection_adjoint(g, u, lam) * du).sum()
    assert abs(lhs - rhs) < 1e-10 * np.abs(lam * jvp).sum()


def test_advection_adjoint_zero_velocity_components():
    """Where u_k = 0 the upwind term has no branch: neither the coefficient
    nor the difference contributes (the forward reading of u_k = 0)."""
    g = synth.Grid(n=(4, 4, 4), h=0.25, rho=1.0, mu=0.02, dt=1e-4)
    u = np.zeros((3, 4, 4, 4))
    lam = _rng(14).standard_normal(u.shape)
    assert np.all(oracle.advection_adjoint(g, u, lam) == 0.0)


def _small_structure(seed=7, D_scale=1e-4):
    p = synth.cochlea_small(seed=seed)
    st = oracle.Structure(p.structure)
    rng = _rng(seed + 100)
    D = D_scale * rng.standard_normal(st.X0.shape)
    return p, st, D, rng


def test_forces_lin_is_symmetric_jacobian():
    p, st, D, rng = _small_structure()
    lam = rng.standard_normal(D.shape)
    dD = rng.standard_normal(D.shape)
    eps = 1e-7
    jvp = (oracle.forces(st, D + eps * dD) - oracle.forces(st, D - eps * dD)) / (2 * eps)
    K_dD = oracle.forces_lin(st, D, dD)
    assert np.max(np.abs(jvp - K_dD)) < 1e-6 * np.max(np.abs(K_dD))
    a = (lam * K_dD).sum()
    b = (oracle.forces_lin(st, D, lam) * dD).sum()
    assert abs(a - b) < 1e-12 * np.abs(lam * K_dD).sum()


def test_forces_lin_sphere_springs():
    p = synth.sphere32()
    st = oracle.Structure(p.structure)
    rng = _rng(21)
    D = 1e-3 * rng.standard_normal(st.X0.shape)
    dD = rng.standard_normal(D.shape)
    eps = 1e-7
    jvp = (oracle.forces(st, D + eps * dD) - oracle.forces(st, D - eps * dD)) / (2 * eps)
    K_dD = oracle.forces_lin(st, D, dD)
    assert np.max(np.abs(jvp - K_dD)) < 1e-6 * np.max(np.abs(K_dD))


def test_forces_dbend_is_stiffness_derivative():
    p, st, D, rng = _small_structure()
    lam = rng.standard_normal(D.shape)
    gb = oracle.forces_dbend(st, D, lam)
    b0 = st.bend_b.copy()
    assert len(gb) == len(b0) and np.all(np.abs(gb) > 0)
    for s in range(len(b0)):
        eps = 0.5 * b0[s]                               # f is linear in b
        bp, bm = b0.copy(), b0.copy()
        bp[s] += eps
        bm[s] -= eps
        fp = oracle.forces(oracle.Structure(p.structure, bend_b=bp), D)
        fm = oracle.forces(oracle.Structure(p.structure, bend_b=bm), D)
        fd = (lam * (fp - fm)).sum() / (2 * eps)
        assert abs(fd - gb[s]) < 1e-7 * abs(gb[s])


def test_solve_is_symmetric():
    """The spectral solve L (Eqs. discreteNS1-2) is real symmetric, which the
    reverse step uses in place of its transpose."""
    g = synth.Grid(n=(6, 4, 8), h=0.1, rho=1.0, mu=0.02, dt=1e-4)
    rng = _rng(15)
    a = rng.standard_normal((3, 8, 4, 6))
    b = rng.standard_normal((3, 8, 4, 6))
    lhs = (a * oracle.solve(g, b)).sum()
    rhs = (oracle.solve(g, a) * b).sum()
    assert abs(lhs - rhs) < 1e-13 * np.sqrt((a * a).sum() * (b * b).sum()) * g.dt


# ---------------------------------------------------------------------------
# the whole reverse step against finite differences of forward steps
# ---------------------------------------------------------------------------
def _state(p, st, rng, u_scale):
    """A uniform flow plus a perturbation of 0.3 of its smallest component:
    after a step (which projects the perturbation) every component keeps its
    sign, so no upwind branch switches within a finite-difference stencil in
    either step of a two-step check."""
    mean = u_scale * np.array([1.0, -0.8, 0.9])
    nx, ny, nz = p.grid.n
    u = mean[:, None, None, None] + 0.3 * 0.8 * u_scale * (2 * rng.random((3, nz, ny, nx)) - 1)
    D = 1e-4 * rng.standard_normal(st.X0.shape)
    return u, D


def _directions(st, u, D, rng):
    du = (2 * rng.random(u.shape) - 1) * 0.1 * np.abs(u).min()
    dD = rng.standard_normal(D.shape) * 1e-4
    db = rng.standard_normal(len(st.bend_b)) * st.bend_b
    return du, dD, db


@pytest.mark.parametrize("no_advection", [False, True])
def test_adjoint_step_matches_fd_of_step(no_advection):
    p, st, _, rng = _small_structure(seed=7)
    g = p.grid
    u, D = _state(p, st, rng, 50.0)
    t = 1.3e-4
    a = rng.standard_normal(u.shape)
    c = rng.standard_normal(D.shape)
    du, dD, db = _directions(st, u, D, rng)

    def J(u_, D_, b_):
        s_ = oracle.Structure(p.structure, bend_b=b_)
        D1, u1, _ = oracle.step(g, s_, D_, u_, t, 1, no_advection=no_advection)
        # J = <a, u^{n+1}> + <c, D^{n+1} - D^n>: the increment isolates the
        # non-identity part of dJ/dD
        return (a * u1).sum() + (c * (D1 - D_)).sum()

    lu0, lD0, gb = oracle.adjoint_step(g, st, D, u, t, a, c, no_advection=no_advection)
    lD0 = lD0 - c
    b0 = st.bend_b.copy()
    # steps: J is quadratic in u between upwind switches and affine in b
    # within one step, so those take large steps (small rounding error)
    for name, eps, (vu, vD, vb), an in (
            ("u", 1e-2, (du, 0 * dD, 0 * db), (lu0 * du).sum()),
            ("D", 1e-3, (0 * du, dD, 0 * db), (lD0 * dD).sum()),
            ("b", 1.0, (0 * du, 0 * dD, db), (gb * db).sum())):
        fd = (J(u + eps * vu, D + eps * vD, b0 + eps * vb) - J(u - eps * vu, D - eps * vD, b0 - eps * vb)) / (2 * eps)
        assert abs(fd - an) < 1e-8 * abs(an), (name, fd, an)


def test_adjoint_two_steps_chain():
    """Two reverse steps in a row, each about its own forward state (u^n, D^n,
    t^n), give the gradient of a function of the state two steps later."""
    p, st, _, rng = _small_structure(seed=8)
    g = p.grid
    u0, D0 = _state(p, st, rng, 20.0)
    t0 = 0.0
    a = rng.standard_normal(u0.shape)
    c = rng.standard_normal(D0.shape)
    du, dD, db = _directions(st, u0, D0, rng)
    b0 = st.bend_b.copy()

    def J(u_, D_, b_):
        s_ = oracle.Structure(p.structure, bend_b=b_)
        D2, u2, _ = oracle.step(g, s_, D_, u_, t0, 2)
        return (a * u2).sum() + (c * (D2 - D_)).sum()

    D1, u1, t1 = oracle.step(g, st, D0, u0, t0, 1)
    lu1, lD1, gb1 = oracle.adjoint_step(g, st, D1, u1, t1, a, c)
    lu0, lD0, gb0 = oracle.adjoint_step(g, st, D0, u0, t0, lu1, lD1)
    lD0 = lD0 - c
    gb = gb0 + gb1
    # J is close to affine in b over two steps, so b takes a large step
    # (the b-sensitivity is small against J, and rounding dominates below)
    for name, eps, vu, vD, vb, an in (("u", 1e-2, du, 0 * dD, 0 * db, (lu0 * du).sum()),
                                      ("D", 1e-3, 0 * du, dD, 0 * db, (lD0 * dD).sum()),
                                      ("b", 1e-1, 0 * du, 0 * dD, db, (gb * db).sum())):
        fd = (J(u0 + eps * vu, D0 + eps * vD, b0 + eps * vb) - J(u0 - eps * vu, D0 - eps * vD, b0 - eps * vb)) / (2 * eps)
        assert abs(fd - an) < 1e-7 * abs(an), (name, fd, an)


def test_adjoint_step_sphere_springs_only():
    """A closed spring shell with no bending or tethers: grad_b is empty and
    the position sensitivity comes from springs, spreading and interpolation."""
    p = synth.sphere_problem(n=16, level=2, seed=3)
    st = oracle.Structure(p.structure)
    g = p.grid
    rng = _rng(31)
    u = _bounded_velocity(g, rng, 5.0)
    D = 1e-3 * rng.standard_normal(st.X0.shape)
    a = rng.standard_normal(u.shape)
    c = rng.standard_normal(D.shape)
    lu0, lD0, gb = oracle.adjoint_step(g, st, D, u, 0.0, a, c)
    assert gb.size == 0
    dD = 1e-3 * rng.standard_normal(D.shape)

    def J(D_):
        D1, u1, _ = oracle.step(g, st, D_, u, 0.0, 1)
        return (a * u1).sum() + (c * (D1 - D_)).sum()

    eps = 1e-4
    fd = (J(D + eps * dD) - J(D - eps * dD)) / (2 * eps)
    an = ((lD0 - c) * dD).sum()
    assert abs(fd - an) < 3e-8 * abs(an)
