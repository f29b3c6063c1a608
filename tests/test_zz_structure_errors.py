"""Corrupted structures are caught on the host and leave the context as it was.

ib_set_structure checks every link and lattice index before it touches the
context: a spring past the last marker or from a marker to itself, a tether
on a negative marker, a sheet row in a stiffness segment that does not exist.
Each returns IB_ERR_ARG, and the context keeps stepping its previous
structure, bitwise as a context that never saw the bad calls.
"""
import dataclasses

import numpy as np
import pytest

from paper_math_0301321_gb300 import synth
from paper_math_0301321_gb300.binding import Context

pytestmark = pytest.mark.gpu


def host(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def bad_structures(st):
    m = st.m
    past_end = st.spring_ij.copy()
    past_end[5, 1] = m
    self_loop = st.spring_ij.copy()
    self_loop[3, 1] = self_loop[3, 0]
    tether = st.tether_i.copy()
    tether[2] = -1
    seg = st.sheets[0].seg_of_row.copy()
    seg[0] = len(st.bend_b)
    sheet = dataclasses.replace(st.sheets[0], seg_of_row=seg)
    return [dataclasses.replace(st, spring_ij=past_end), dataclasses.replace(st, spring_ij=self_loop),
            dataclasses.replace(st, tether_i=tether), dataclasses.replace(st, sheets=[sheet] + st.sheets[1:])]


def test_bad_structures_are_rejected_and_the_context_keeps_its_own(ib):
    from paper_math_0301321_gb300.binding import IBError, IB_ERR_ARG
    p = synth.cochlea_small()
    st = p.structure

    ref = Context(p.grid, prec="fp64")
    ref.set_structure(st)
    ref.set_state(p.u, p.X, 0.0)
    ref.step(2)
    u_ref, X_ref, t_ref = ref.get_state()
    u_ref, X_ref = host(u_ref), host(X_ref)
    ref.close()

    ctx = Context(p.grid, prec="fp64")
    ctx.set_structure(st)
    ctx.set_state(p.u, p.X, 0.0)
    ctx.step(1)
    for bad in bad_structures(st):
        with pytest.raises(IBError) as e:
            ctx.set_structure(bad)
        assert e.value.status == IB_ERR_ARG
    ctx.step(1)
    u, X, t = ctx.get_state()
    ctx.close()
    assert t == t_ref
    assert np.array_equal(host(u), u_ref)
    assert np.array_equal(host(X), X_ref)
