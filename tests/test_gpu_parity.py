"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Bars: FP64 contexts within 1e-12 relative (norm-wise), FP32 contexts within
2e-5 relative per call / per step from an identical state; the bin sort is
bit-exact.  Inputs are seeded and synthetic.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_math_0301321_gb300 import synth
from paper_math_0301321_gb300.binding import Context

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b.astype(np.float64))
    return float(np.linalg.norm(a.astype(np.float64) - b) / (nb if nb > 0 else 1.0))


def host(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


class Grid:
    def __init__(self, n, h=None, rho=1.0, mu=0.02, dt=1e-5):
        self.n = tuple(n)
        self.h = (1.0 / 32) if h is None else h
        self.rho, self.mu, self.dt = rho, mu, dt


def point_cloud(seed, n, m, h):
    """Markers uniform in the box plus a dense clump, exact nodes, seam and out-of-box points."""
    L = np.array(n, float) * h
    X = synth.random_markers(seed, m) * L[:, None]
    k = m // 4
    X[:, :k] = (np.array([3.3, 4.6, 5.1])[:, None] * h + synth.random_markers(seed + 1, k) * h * 0.9)
    X[:, k:k + 8] = np.round(X[:, k:k + 8] / h) * h                    # on nodes
    X[0, k + 8:k + 16] = L[0] - 1e-12                                   # at the seam
    X[:, k + 16:k + 24] += L[:, None]                                   # outside the box (wraps)
    X[1, k + 24:k + 32] -= L[1]
    return X


def structure_of(X):
    return synth._empty_structure(np.ascontiguousarray(X))


@pytest.mark.parametrize("n", [(32, 32, 32), (64, 32, 96)])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_bin_sort_bit_exact(ib, n, prec):
    g = Grid(n)
    X = point_cloud(1, n, 5000, g.h)
    ctx = Context(g, prec=prec)
    ctx.set_structure(structure_of(X))
    key, perm = ctx.bin_sort(X)
    okey, operm = oracle.bin_sort(g, X)
    assert np.array_equal(host(key), okey)
    assert np.array_equal(host(perm), operm)


@pytest.mark.parametrize("n,m", [((32, 32, 32), 3000), ((64, 32, 96), 6000), ((32, 32, 32), 1),
                                 ((256, 32, 64), 4000)])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_spread_matches_oracle(ib, n, m, prec):
    g = Grid(n)
    X = point_cloud(2, n, m, g.h) if m > 40 else synth.random_markers(2, m)
    f = synth.random_forces(3, m)
    ctx = Context(g, prec=prec)
    ctx.set_structure(structure_of(X))
    F = ctx.spread(X, f)
    Fo = oracle.spread(g, X, f)
    assert rel(F, Fo) <= TOL[prec]
    # repeated calls are bitwise identical
    F2 = ctx.spread(X, f)
    assert torch.equal(F, F2)


@pytest.mark.parametrize("n,m", [((32, 32, 32), 3000), ((64, 32, 96), 6000), ((32, 32, 32), 1),
                                 ((32, 32, 32), 20000)])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_interp_matches_oracle(ib, n, m, prec):
    """Includes one marker, and 20,000 markers whose dense clump (5,000 in one
    cell) makes a bin of several work items."""
    g = Grid(n)
    X = point_cloud(4, n, m, g.h) if m > 40 else synth.random_markers(4, m)
    u = synth.random_velocity(5, n, noise=0.5)
    ctx = Context(g, prec=prec)
    ctx.set_structure(structure_of(X))
    U = ctx.interp(X, u)
    Uo = oracle.interp(g, X, u)
    assert rel(U, Uo) <= TOL[prec]


@pytest.mark.parametrize("n", [(32, 32, 32), (64, 32, 96), (128, 64, 32), (256, 32, 32), (32, 256, 32),
                               (32, 32, 256)])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fluid_solve_matches_oracle(ib, n, prec):
    g = Grid(n, rho=1.0, mu=0.02, dt=1e-4)
    u = synth.random_velocity(6, n, amp=3.0, noise=0.3)
    F = synth.random_velocity(7, n, amp=1e4, noise=0.2)
    ctx = Context(g, prec=prec)
    un, p = ctx.fluid_solve(u, F, want_p=True)
    uo, po = oracle.fluid_solve(g, u, F, want_p=True)
    assert rel(un, uo) <= TOL[prec]
    assert rel(p, po) <= TOL[prec] * 10


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fluid_solve_stokes_and_host_pointers(ib, prec):
    g = Grid((32, 64, 32), rho=1.3, mu=0.5, dt=1e-3)
    u = synth.random_velocity(8, g.n, noise=1.0)
    F = synth.random_velocity(9, g.n, amp=100.0)
    ctx = Context(g, prec=prec, device=False, no_advection=True)
    un = ctx.fluid_solve(u, F)
    uo = oracle.fluid_solve(g, u, F, no_advection=True)
    assert rel(un, uo) <= TOL[prec]


def run_gpu(p, prec, nsteps, no_advection=False, D=None, u=None, t=0.0):
    """nsteps on the GPU from displacement D (from the reference X0) and velocity u."""
    ctx = Context(p.grid, prec=prec, no_advection=no_advection)
    ctx.set_structure(p.structure)
    ctx.set_state(p.u if u is None else u, None, t)
    ctx.set_displacement(np.zeros_like(p.structure.X0) if D is None else D)
    ctx.step(nsteps)
    uu, XX, tt = ctx.get_state()
    DD = ctx.get_displacement()
    ctx.close()
    return host(DD), host(uu), tt


def test_step_sphere_fp64_20_steps(ib):
    p = synth.sphere32()
    st = oracle.Structure(p.structure)
    D0 = np.zeros_like(p.X)
    Do, uo, to = oracle.step(p.grid, st, D0, p.u, 0.0, 20)
    Dg, ug, tg = run_gpu(p, "fp64", 20)
    assert rel(ug, uo) <= 1e-12
    assert rel(Dg, Do) <= 1e-12
    assert abs(tg - to) <= 1e-18


def test_step_cochlea_fp64(ib):
    p = synth.cochlea_small()
    st = oracle.Structure(p.structure)
    # start from a perturbed state so that every force term is active
    D = 1e-5 * synth.random_forces(21, p.structure.m)
    u = synth.random_velocity(22, p.grid.n, amp=1e-2)
    Do, uo, to = oracle.step(p.grid, st, D, u, 0.0, 5)
    Dg, ug, tg = run_gpu(p, "fp64", 5, D=D, u=u)
    assert rel(ug, uo) <= 1e-12
    assert rel(Dg - D, Do - D) <= 1e-12


@pytest.mark.parametrize("case", ["sphere", "cochlea"])
def test_step_fp32_per_step(ib, case):
    if case == "sphere":
        p = synth.sphere32()
        D, u = np.zeros_like(p.X), p.u
    else:
        p = synth.cochlea_small()
        D = 1e-5 * synth.random_forces(23, p.structure.m)
        u = synth.random_velocity(24, p.grid.n, amp=1e-2)
    st = oracle.Structure(p.structure)
    # advance a few oracle steps, then compare one step from that shared state
    Ds, us, ts = oracle.step(p.grid, st, D, u, 0.0, 3)
    Do, uo, to = oracle.step(p.grid, st, Ds, us, ts, 1)
    Dg, ug, tg = run_gpu(p, "fp32", 1, D=Ds, u=us, t=ts)
    assert rel(ug, uo) <= 2e-5
    assert rel(Dg - Ds, Do - Ds) <= 2e-5


def test_step_without_markers(ib):
    g = Grid((32, 32, 64), dt=1e-4)
    u = synth.random_velocity(25, g.n, amp=2.0, noise=0.1)
    X0 = np.zeros((3, 0))
    st = synth._empty_structure(X0)
    p = synth.Problem("fluid", synth.Grid(g.n, g.h, g.rho, g.mu, g.dt), st, X0, u)
    Do, uo, to = oracle.step(p.grid, oracle.Structure(st), X0, u, 0.0, 3)
    Dg, ug, tg = run_gpu(p, "fp64", 3)
    assert rel(ug, uo) <= 1e-12


def test_step_is_bitwise_reproducible(ib):
    p = synth.cochlea_small()
    D = 1e-5 * synth.random_forces(26, p.structure.m)
    a = run_gpu(p, "fp32", 4, D=D)
    b = run_gpu(p, "fp32", 4, D=D)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_positions_round_trip_through_state(ib):
    p = synth.cochlea_small()
    ctx = Context(p.grid, prec="fp64")
    ctx.set_structure(p.structure)
    X = p.X + 1e-3 * synth.random_forces(27, p.structure.m)
    ctx.set_state(None, X, 0.25)
    u, XX, t = ctx.get_state()
    assert t == 0.25
    assert np.abs(host(XX) - X).max() <= 4e-16
    assert np.abs(host(ctx.get_displacement()) - (X - p.X)).max() <= 4e-16


def test_state_transfer_pinned_host_buffers(ib):
    """A host-pointer context reads and writes page-locked caller buffers in
    place (no staging copy); positions, displacements and the stepped state
    equal the staged path's (pageable numpy buffers) bit for bit."""
    import ctypes as C
    from paper_math_0301321_gb300 import binding
    p = synth.cochlea_small()
    X = p.X + 1e-6 * synth.random_forces(27, p.structure.m)
    for prec in ("fp64", "fp32"):
        ref = Context(p.grid, prec=prec, device=False)
        ref.set_structure(p.structure)
        ref.set_state(p.u, X, 0.0)
        ref.step(2)
        _, X_ref, _ = ref.get_state()
        D_ref = ref.get_displacement()
        ref.close()

        ctx = Context(p.grid, prec=prec, device=False)
        ctx.set_structure(p.structure)
        Xp = torch.from_numpy(np.ascontiguousarray(X)).pin_memory()
        ctx.set_state(p.u, None, 0.0)
        binding._check(ctx.lib.ib_set_state(ctx.h, None, C.c_void_p(Xp.data_ptr()), 0.0))
        ctx.step(2)
        Xo = torch.zeros_like(Xp).pin_memory()
        Do = torch.zeros_like(Xp).pin_memory()
        t = C.c_double()
        binding._check(ctx.lib.ib_get_state(ctx.h, None, C.c_void_p(Xo.data_ptr()), C.byref(t)))
        binding._check(ctx.lib.ib_get_displacement(ctx.h, C.c_void_p(Do.data_ptr())))
        assert np.array_equal(Xo.numpy(), X_ref) and np.array_equal(Do.numpy(), D_ref)
        # displacements written from a pinned buffer come back unchanged
        Dp = torch.from_numpy(np.ascontiguousarray(D_ref)).pin_memory()
        binding._check(ctx.lib.ib_set_displacement(ctx.h, C.c_void_p(Dp.data_ptr())))
        assert np.array_equal(host(ctx.get_displacement()), D_ref) or prec == "fp32"
        ctx.close()


def _order_vs_oracle(g, X0, D, key, perm, internal):
    X = np.asarray(X0, np.float64) + D
    ko, po = oracle.bin_sort(g, X[:, internal])
    k = np.empty_like(ko)
    k[internal] = ko
    return np.array_equal(key, k), np.array_equal(perm, internal[po]), int((key != k).sum())


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_step_bin_sort_bit_exact_at_cell_faces(ib, prec):
    """The step forms its keys from the state X0 + D.  Markers whose reference
    positions sit on cell faces, displaced by a few units in the last place
    of the FP32 offset either way, and markers displaced by whole cells: the
    step's keys and tile order equal the oracle's sort of X0 + D bit for bit
    (in FP32 contexts the cell is decided in FP64 within rounding of a face)."""
    n = (32, 32, 64)
    g = Grid(n, h=1.0 / 32)
    m = 6000
    rng = np.random.default_rng(11)
    cells = rng.integers(0, 32, size=(3, m)).astype(np.float64)
    cells[2] = rng.integers(0, 64, size=m)
    X0 = cells * g.h
    X0[:, m // 2:] += rng.random((3, m - m // 2)) * g.h                # half off the faces
    # displacements: tiny multiples of h either way, a few whole cells, zero
    D = np.zeros((3, m))
    D[:, :m // 3] = rng.integers(-4, 5, size=(3, m // 3)) * (g.h * 2.0 ** -26)
    D[:, m // 3:m // 2] = rng.integers(-3, 4, size=(3, m // 2 - m // 3)) * g.h
    D[:, m // 2:] = 1e-7 * rng.standard_normal((3, m - m // 2))
    D = np.asarray(D, np.float32).astype(np.float64)                   # held exactly by FP32 contexts
    ctx = Context(g, prec=prec)
    ctx.set_structure(structure_of(X0))
    ctx.set_displacement(D)
    Dh = host(ctx.get_displacement())
    ctx.step(1)
    key, perm, internal = (host(o) for o in ctx.get_bin_order())
    ctx.close()
    ok_k, ok_p, nbad = _order_vs_oracle(g, X0, Dh, key, perm, internal)
    assert ok_k, nbad
    assert ok_p


def test_nonfinite_velocity_is_reported(ib):
    """A NaN in the velocity field reaches the markers through the solve and
    interpolation: the next ib_sync reports IB_ERR_NONFINITE and names it."""
    from paper_math_0301321_gb300.binding import IBError, IB_ERR_NONFINITE
    p = synth.sphere32()
    ctx = Context(p.grid, prec="fp32")
    ctx.set_structure(p.structure)
    u = np.array(p.u, np.float64)
    u[1, 5, 6, 7] = np.nan
    ctx.set_state(u, p.X, 0.0)
    ctx.step(1)
    with pytest.raises(IBError) as e:
        ctx.sync()
    assert e.value.status == IB_ERR_NONFINITE
    assert "velocity" in str(e.value)
    # the flag is cleared once reported; a finite state steps cleanly again
    ctx.set_state(p.u, p.X, 0.0)
    ctx.step(1)
    ctx.sync()
    ctx.close()


def test_bounded_wait_that_runs_out_is_reported(ib):
    """A bounded wait on an mbarrier that nothing arrives on runs out: the
    next ib_sync reports IB_ERR_TIMEOUT and clears the flag, and the context
    then steps bitwise as a context that never saw the failure."""
    from paper_math_0301321_gb300.binding import IBError, IB_ERR_ARG, IB_ERR_TIMEOUT
    p = synth.sphere32()

    def fresh():
        c = Context(p.grid, prec="fp32")
        c.set_structure(p.structure)
        c.set_state(p.u, p.X, 0.0)
        return c

    ref = fresh()
    ref.step(2)
    u_ref, X_ref, _ = (host(o) if not isinstance(o, float) else o for o in ref.get_state())
    ref.close()

    ctx = fresh()
    with pytest.raises(IBError) as e:
        ctx.check_bounded_wait(0)
    assert e.value.status == IB_ERR_ARG
    ctx.check_bounded_wait(1000)
    with pytest.raises(IBError) as e:
        ctx.sync()
    assert e.value.status == IB_ERR_TIMEOUT
    assert "bounded wait" in str(e.value)
    ctx.sync()
    ctx.step(2)
    u, X, _ = (host(o) if not isinstance(o, float) else o for o in ctx.get_state())
    ctx.close()
    assert np.array_equal(u, u_ref)
    assert np.array_equal(X, X_ref)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_nonfinite_position_is_reported(ib, prec):
    """A non-finite marker displacement is caught where the step forms the
    marker's cell (IB_ERR_NONFINITE, 'position'); the keys stay in range."""
    from paper_math_0301321_gb300.binding import IBError, IB_ERR_NONFINITE
    p = synth.sphere32()
    ctx = Context(p.grid, prec=prec)
    ctx.set_structure(p.structure)
    D = np.zeros_like(p.structure.X0)
    D[0, 17] = np.inf
    ctx.set_displacement(D)
    ctx.step(1)
    with pytest.raises(IBError) as e:
        ctx.sync()
    assert e.value.status == IB_ERR_NONFINITE
    assert "position" in str(e.value)
    ctx.close()
