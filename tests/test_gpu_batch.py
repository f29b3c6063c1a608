"""Tile tuning, the autotuner and batched stepping (ib_set_tuning,
ib_autotune, ib_batch_*).

Tile shapes change only how work is split among blocks, never the
arithmetic of a grid point or a marker, so every tuning must give bitwise
the same step; a batch must advance each member exactly as stepping it
alone; the autotuner must leave the state where it found it.
"""
import numpy as np
import pytest
import torch

from paper_math_0301321_gb300 import synth
from paper_math_0301321_gb300.binding import Batch, Context, IBError

pytestmark = pytest.mark.gpu


def started(p, prec="fp32", seed=3):
    ctx = Context(p.grid, prec=prec)
    ctx.set_structure(p.structure)
    D = synth.membrane_bump(p, 1e-7, 3)
    u = synth.random_velocity(seed, p.grid.n, amp=0.1, modes=6)
    ctx.set_state(u, None, 1e-5)
    ctx.set_displacement(D)
    return ctx


def state_of(ctx):
    ctx.sync()
    u, _, t = ctx.get_state()
    return u.cpu().numpy(), ctx.get_displacement().cpu().numpy(), t


def same(a, b):
    return np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_every_tuning_gives_the_same_step(ib, prec):
    p = synth.cochlea_small(seed=7, n=64, bm=(128, 16), walls=(300, 60), n_fibers=100, dt=1e-6)
    ref = None
    variants = [(x, y, z) for x in (0, 1, 2) for y in (0, 1) for z in (0, 1)] if prec == "fp32" else [(0, 0, 0)]
    for (x, y, z) in variants:
        for mb in (0, 7, 152):
            ctx = started(p, prec)
            ctx.set_tuning(x, y, z, mb)
            assert ctx.get_tuning() == {"fft_x": x, "fft_y": y, "fft_z": z, "marker_blocks": mb}
            ctx.step(3)
            st = state_of(ctx)
            ctx.close()
            if ref is None:
                ref = st
            assert same(st, ref), (x, y, z, mb)


def test_tuning_rejects_bad_values(ib):
    p = synth.cochlea_small(seed=7)
    c32 = Context(p.grid, prec="fp32")
    c64 = Context(p.grid, prec="fp64")
    with pytest.raises(IBError):
        c32.set_tuning(3, 0, 0, 0)
    with pytest.raises(IBError):
        c32.set_tuning(0, 2, 0, 0)
    with pytest.raises(IBError):
        c32.set_tuning(0, 0, 0, -1)
    with pytest.raises(IBError):
        c64.set_tuning(1, 0, 0, 0)


def test_autotune_keeps_the_state(ib):
    p = synth.cochlea_small(seed=8, n=64, bm=(128, 16), walls=(300, 60), n_fibers=100, dt=1e-6)
    a = started(p)
    b = started(p)
    before = state_of(a)
    best = a.autotune(reps=3)
    assert set(best) == {"fft_x", "fft_y", "fft_z", "marker_blocks"}
    assert a.get_tuning() == best
    assert same(state_of(a), before)
    a.step(4)
    b.step(4)
    assert same(state_of(a), state_of(b))


@pytest.mark.parametrize("steps_per_launch", [1, 3])
def test_batch_equals_members_stepped_alone(ib, steps_per_launch):
    probs = [synth.cochlea_small(seed=11, n=32, dt=1e-6),
             synth.cochlea_small(seed=12, n=64, bm=(128, 16), walls=(300, 60), n_fibers=100, dt=1e-6),
             synth.cochlea_small(seed=13, n=96, bm=(96, 12), walls=(200, 40), n_fibers=50, dt=1e-6)]
    alone = []
    for p in probs:
        c = started(p)
        c.step(6)
        alone.append(state_of(c))
        c.close()
    ctxs = [started(p) for p in probs]
    b = Batch(ctxs, steps_per_launch=steps_per_launch)
    b.step(6)
    b.sync()
    for c, ref in zip(ctxs, alone):
        assert same(state_of(c), ref)
    if steps_per_launch == 3:
        with pytest.raises(IBError):
            b.step(4)                           # not a multiple of steps_per_launch
    b.close()


def test_batch_autotune_and_retune(ib):
    probs = [synth.cochlea_small(seed=21, n=32, dt=1e-6),
             synth.cochlea_small(seed=22, n=64, bm=(128, 16), walls=(300, 60), n_fibers=100, dt=1e-6)]
    ref = []
    for p in probs:
        c = started(p)
        c.step(5)
        ref.append(state_of(c))
        c.close()
    ctxs = [started(p) for p in probs]
    b = Batch(ctxs)
    b.autotune(reps=2)
    tunings = [c.get_tuning() for c in ctxs]
    assert tunings[0] == tunings[1]
    b.step(3)
    ctxs[1].set_tuning(1, 1, 1, 5)              # the batch graph goes stale and is recaptured
    b.step(2)
    b.sync()
    for c, r in zip(ctxs, ref):
        assert same(state_of(c), r)
    b.close()


def test_batch_rejects_bad_arguments(ib):
    p = synth.cochlea_small(seed=7)
    c = started(p)
    with pytest.raises(IBError):
        Batch([c, c])
    e = Context(p.grid, prec="fp32")          # no structure
    with pytest.raises(IBError):
        Batch([c, e])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_members_match_oracle(ib, prec):
    """A batch of three uneven members (32^3, 64^3 and 96^3 grids, different
    membranes, wall and fibre counts, tones) advanced in one graph launch per
    step: each member's state against the oracle's steps from the same state
    (bars: FP64 1e-12 over 2 steps, FP32 2e-5 over 1 step, norm-wise, and the
    largest element within 10x that of the field's largest value)."""
    import oracle
    probs = [synth.cochlea_small(seed=31, n=32, dt=1e-6, freq=1500.0),
             synth.cochlea_small(seed=32, n=64, bm=(128, 16), walls=(300, 60), n_fibers=100, dt=1e-6, freq=4000.0),
             synth.cochlea_small(seed=33, n=96, bm=(96, 12), walls=(200, 40), n_fibers=50, dt=1e-6, freq=800.0)]
    tol = {"fp64": 1e-12, "fp32": 2e-5}[prec]
    nsteps = 2 if prec == "fp64" else 1
    starts, ctxs = [], []
    for i, p in enumerate(probs):
        D = synth.membrane_bump(p, 1e-7, 3)
        u = synth.random_velocity(40 + i, p.grid.n, amp=0.1, modes=6)
        if prec == "fp32":
            D = np.asarray(D, np.float32).astype(np.float64)
            u = np.asarray(u, np.float32).astype(np.float64)
        t0 = 1e-5 * (i + 1)
        c = Context(p.grid, prec=prec)
        c.set_structure(p.structure)
        c.set_state(u, None, t0)
        c.set_displacement(D)
        starts.append((D, u, t0))
        ctxs.append(c)
    b = Batch(ctxs)
    b.step(nsteps)
    b.sync()
    for p, c, (D, u, t0) in zip(probs, ctxs, starts):
        ug, Dg, tg = state_of(c)
        Do, uo, to = oracle.step(p.grid, oracle.Structure(p.structure), D, u, t0, nsteps)
        assert abs(tg - to) < 1e-15
        du, dD = ug.astype(np.float64) - uo, (Dg - D) - (Do - D)
        assert np.linalg.norm(du) <= tol * np.linalg.norm(uo), (p.name, prec)
        assert np.linalg.norm(dD) <= tol * np.linalg.norm(Do - D), (p.name, prec)
        assert np.abs(du).max() <= 10 * tol * np.abs(uo).max(), (p.name, prec)
        assert np.abs(dD).max() <= 10 * tol * np.abs(Do - D).max(), (p.name, prec)
    b.close()
