"""Pins of the oracle's external marker force (the oval window's stapes
load, Section 4) and of the window geometry.

The force enters the fluid only through spreading, which conserves the total
force, and through the solve, whose mean (zero-wavenumber) mode is
rho u/dt + F divided by rho/dt: after one step from rest, with no body force
and no advection, the fluid momentum is exactly dt times the total marker
force at the step's start time.  So the momentum of the fluid pins the
force's magnitude, direction, the markers it acts on and its time argument
independently of the force code.
"""
import dataclasses
import math

import numpy as np

import oracle
from paper_math_0301321_gb300 import synth


def windows_only(n=32):
    """The windows of the small cochlea without the cochlea (and without its
    body force), so that at rest the only force is the oval window's load."""
    base = synth.cochlea_small(seed=7, n=n)
    full = synth.with_windows(base, n_w=12, freq=3000.0, force_amp=2e-3)
    st, m0 = full.structure, base.structure.m
    keep = np.arange(m0, st.m)
    remap = np.full(st.m, -1)
    remap[keep] = np.arange(len(keep))
    sp = np.all(remap[st.spring_ij] >= 0, axis=1)
    te = remap[st.tether_i] >= 0
    mf = st.marker_forcing
    st2 = dataclasses.replace(
        st, X0=st.X0[:, keep], spring_ij=remap[st.spring_ij[sp]].astype(np.int32), spring_k=st.spring_k[sp],
        spring_L0=st.spring_L0[sp], tether_i=remap[st.tether_i[te]].astype(np.int32), tether_k=st.tether_k[te],
        sheets=[], bend_b=np.zeros(0), forcing=synth.Forcing(), normal0=None, n_membrane=0, centerline=None,
        marker_forcing=dataclasses.replace(mf, index=remap[mf.index].astype(np.int32)))
    return dataclasses.replace(full, structure=st2, X=st2.X0.copy()), mf


def test_window_geometry():
    base = synth.cochlea_small(seed=7)
    p = synth.with_windows(base, n_w=12)
    st, m0 = p.structure, base.structure.m
    assert st.m == m0 + 2 * 144
    # rim points (outside the circle) are tethered, the rest are free; the oval
    # window's free points are the forced ones
    g = np.linspace(-0.04, 0.04, 12)
    gu, gv = np.meshgrid(g, g, indexing="ij")
    free = (gu ** 2 + gv ** 2 <= 0.035 ** 2).ravel()
    wt = st.tether_i[st.tether_i >= m0]
    assert len(wt) == 2 * int((~free).sum())
    assert np.array_equal(np.sort(st.marker_forcing.index), np.nonzero(free)[0] + m0)
    # the windows are flat plates perpendicular to the membrane's base tangent
    _, T0, _, _ = synth.helix_frame(np.zeros(1), synth.HELIX_Z0)
    for w in range(2):
        P = st.X0[:, m0 + 144 * w: m0 + 144 * (w + 1)]
        assert np.max(np.abs((P - P.mean(1, keepdims=True)).T @ T0[:, 0])) < 1e-15


def test_marker_force_momentum_after_one_step():
    p, mf = windows_only()
    st = oracle.Structure(p.structure)
    g = p.grid
    for t in (0.0, 1.7e-4, math.pi / (2 * mf.omega)):
        D = np.zeros_like(st.X0)
        u = np.zeros((3,) + tuple(reversed(g.n)))
        _, u1, _ = oracle.step(g, st, D, u, t, 1, no_advection=True)
        momentum = g.rho * u1.reshape(3, -1).sum(1) * g.h ** 3
        expected = g.dt * mf.amp * math.cos(mf.omega * t) * mf.direction.sum(1)
        scale = g.dt * mf.amp * len(mf.index)
        assert np.max(np.abs(momentum - expected)) <= 1e-12 * scale, (t, momentum, expected)
