"""GPU parity of the widened model: the oval and round windows with the
stapes load (external marker force), the centre-line probe with its
envelope, the half-cube grid 256 x 256 x 128, and the linear response of
the no-advection (Stokes) mode.  Bars: FP64 1e-12, FP32 2e-5 per step."""
import numpy as np
import pytest
import torch

import oracle
from paper_math_0301321_gb300 import synth
from paper_math_0301321_gb300.binding import Context, IBError

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def host(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def rounded(a, prec):
    return np.asarray(a, np.float32).astype(np.float64) if prec == "fp32" else np.asarray(a, np.float64)


def start_state(p, seed):
    D = synth.membrane_bump(p, 1e-7, 3) + 2e-8 * synth.normal(seed, 61, 3 * p.structure.m).reshape(3, -1)
    u = synth.random_velocity(seed, p.grid.n, amp=0.1, modes=6)
    return D, u


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_windows_step_matches_oracle(ib, prec):
    """Three steps of the small cochlea with both windows and the oval
    window's load, at a time where the load is near its peak."""
    p = synth.with_windows(synth.cochlea_small(seed=7), n_w=12, force_amp=5e-3)
    D, u = start_state(p, 31)
    D, u = rounded(D, prec), rounded(u, prec)
    t = 2.0e-5
    ctx = Context(p.grid, prec=prec)
    ctx.set_structure(p.structure)
    ctx.set_state(u, None, t)
    ctx.set_displacement(D)
    nsteps = 3 if prec == "fp64" else 1
    ctx.step(nsteps)
    ug, _, tg = ctx.get_state()
    Dg = host(ctx.get_displacement())
    st = oracle.Structure(p.structure)
    Do, uo, to = oracle.step(p.grid, st, D, u, t, nsteps)
    assert abs(tg - to) < 1e-15
    assert rel(host(ug), uo) <= TOL[prec]
    assert rel(Dg - D, Do - D) <= TOL[prec]
    # the windows moved (the load is on)
    w = slice(p.structure.m - 2 * 144, p.structure.m)
    assert np.abs(Do[:, w] - D[:, w]).max() > 0


def test_windows_structure_errors(ib):
    p = synth.with_windows(synth.cochlea_small(seed=7), n_w=8)
    bad = p.structure.marker_forcing
    bad.index = bad.index.copy()
    bad.index[1] = bad.index[0]                 # a repeated marker
    ctx = Context(p.grid, prec="fp64")
    with pytest.raises(IBError):
        ctx.set_structure(p.structure)


def test_probe_records_match_oracle(ib):
    """Centre-line normal displacement recorded every 3rd step on the device,
    against the oracle's states; the envelope is the running max |eta|; the
    ring keeps the newest records."""
    p = synth.cochlea_small(seed=9)
    D, u = start_state(p, 32)
    t = 1e-5
    cl = p.structure.centerline
    n0 = p.structure.normal0[:, cl]
    ctx = Context(p.grid, prec="fp64")
    ctx.set_structure(p.structure)
    ctx.set_state(u, None, t)
    ctx.set_displacement(D)
    ctx.set_probe(cl, n0, every=3, capacity=8)
    ctx.step(12)
    eta, times, env, produced = ctx.read_probe()
    assert produced == 4 and eta.shape == (4, len(cl))
    st = oracle.Structure(p.structure)
    Dn, un, tn = D, u, t
    ref, reft = [], []
    for k in range(1, 13):
        Dn, un, tn = oracle.step(p.grid, st, Dn, un, tn, 1)
        if k % 3 == 0:
            ref.append((Dn[:, cl] * n0).sum(0))
            reft.append(tn)
    ref = np.array(ref)
    assert rel(eta, ref) <= 1e-12
    assert np.allclose(times, reft, rtol=0, atol=1e-15)
    assert rel(env, np.abs(ref).max(0)) <= 1e-12
    # nothing new until more steps; then a small ring keeps the newest
    assert ctx.read_probe()[3] == 0
    ctx.set_probe(cl, n0, every=1, capacity=2)
    ctx.step(5)
    eta2, times2, _, produced2 = ctx.read_probe()
    assert produced2 == 5 and eta2.shape == (2, len(cl))
    assert times2[1] > times2[0]
    ctx.set_probe([], np.zeros((3, 0)))
    with pytest.raises(IBError):
        ctx.read_probe()


def test_stokes_mode_is_linear_in_the_load(ib):
    """With advection off the response to the windows' load is linear up to
    the geometric nonlinearity of moving markers, which is second order:
    doubling the load doubles the displacement history to a relative error
    that itself shrinks in proportion to the load."""
    base = synth.cochlea_small(seed=11)

    def run(amp):
        p = synth.with_windows(base, n_w=12, force_amp=amp)
        p.structure.forcing.amp = 0.0
        ctx = Context(p.grid, prec="fp64", no_advection=True)
        ctx.set_structure(p.structure)
        ctx.set_state(np.zeros((3,) + tuple(reversed(p.grid.n))), None, 0.0)
        ctx.step(20)
        D = host(ctx.get_displacement())
        ctx.close()
        return D

    dev = {}
    for amp in (1e-3, 1e-4):
        a, b = run(amp), run(2 * amp)
        assert np.abs(a).max() > 0
        dev[amp] = rel(b, 2 * a)
    assert dev[1e-3] < 1e-6
    assert dev[1e-4] < 0.2 * dev[1e-3], dev


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_half_cube_step_matches_oracle(ib, prec):
    """The paper's production grid shape, 256 x 256 x 128."""
    p = synth.cochlea_halfcube()
    D, u = start_state(p, 33)
    D, u = rounded(D, prec), rounded(u, prec)
    t = 2.0e-5
    ctx = Context(p.grid, prec=prec)
    ctx.set_structure(p.structure)
    ctx.set_state(u, None, t)
    ctx.set_displacement(D)
    ctx.step(1)
    ug, _, _ = ctx.get_state()
    Dg = host(ctx.get_displacement())
    ctx.close()
    Do, uo, _ = oracle.step(p.grid, oracle.Structure(p.structure), D, u, t, 1)
    assert rel(host(ug), uo) <= TOL[prec]
    assert rel(Dg - D, Do - D) <= TOL[prec]
